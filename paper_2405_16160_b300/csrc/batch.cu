// Host side of the batched solver (qp_batch_* in include/pdhcg.h): packs
// the instances into flat device arrays, launches the persistent batch
// kernel (batch_kernels.cuh) and returns per-instance results.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/pdhcg.h"
#include "batch_kernels.cuh"
#include "host_csr.h"

using namespace pdhcg;

void pdhcg_set_last_error(const char* msg);

namespace {

void berror(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  pdhcg_set_last_error(buf);
}

#define BCUDA(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      berror("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return QP_ERR_CUDA;                                                                 \
    }                                                                                     \
  } while (0)

#define BTRY(call)              \
  do {                          \
    qp_status s_ = (call);      \
    if (s_ != QP_OK) return s_; \
  } while (0)

__global__ void k_batch_step_pow(double* t, int count) {
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < count;
       a += (long long)gridDim.x * blockDim.x)
    step_pow_entry(t, a);
}

__global__ void k_fill_f64(double* v, double a, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = a;
}

__global__ void k_to_float(const double* __restrict__ in, float* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = float(in[i]);
}

// Every instance's F from the caller's row-major n x k layout (uploaded as
// is) to the column-major one the solver reads, one destination entry per
// thread (coalesced writes).  The lowest id of an instance holding a
// non-finite entry goes to *bad (INT_MAX when there is none).
__global__ void k_F_colmajor(const BatchDesc* __restrict__ desc, int count,
                             const double* __restrict__ Frow, double* Fcol, long long total,
                             int* bad) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    // the owning instance: the last one with off_F <= e (instances without
    // F entries share their successor's offset and are skipped this way)
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (desc[mid].off_F <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchDesc d = desc[lo];
    const long long t = e - d.off_F;
    const long long l = t / d.n, j = t - l * d.n;
    const double v = Frow[d.off_F + j * d.k + l];
    Fcol[e] = v;
    if (!isfinite(v)) atomicMin(bad, lo);
  }
}

constexpr int kThreadChoices[] = {64, 128, 256, 512};
constexpr int kMaxBins = 4;

// Default block size of a bin: the smallest that keeps about 16 warps per
// SM resident, given the blocks per SM that its vector space in shared memory
// (smem bytes per block of the mixed adaptive layout, 0 for the global
// workspace) and the 128-register launch bounds allow, and at least n/8
// threads for the largest instance (n variables).  The batched kernel is
// latency-bound, so the warps per SM are what count (measured: 128 threads
// for n <= 400 at 4 blocks per SM).
int default_threads(int max_n, size_t smem) {
  const int per_sm_smem = 228 * 1024;
  for (int t : kThreadChoices) {
    const int by_regs = 65536 / (t * 128);
    const int by_smem = smem > 0 ? int(size_t(per_sm_smem) / (smem + 2048)) : by_regs;
    const int warps = std::min(by_regs, by_smem) * (t / 32);
    if (warps >= 16 && t >= std::min(512, max_n / 8)) return t;
  }
  return kThreadChoices[3];
}

}  // namespace

// Instances of similar size, solved by one launch on their own stream.
struct BatchBin {
  int count = 0;
  std::vector<int32_t> h_order;
  int32_t* order = nullptr;  // instance ids (device)
  int max_n = 1, max_m = 1, max_k = 1;
  // vector space of one block and its dynamic shared memory (0: global
  // workspace), for FP64 [0] and mixed [1] precision, each with the fixed
  // [0] and the adaptive [1] step size
  size_t block_doubles[2][2] = {{0, 0}, {0, 0}};
  size_t smem[2][2] = {{0, 0}, {0, 0}};
  int threads = 128;
  double* ws = nullptr;      // global workspace when the vectors do not fit shared memory
  size_t ws_doubles = 0;     // capacity of ws
  int* next = nullptr;       // work-queue counter
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

struct qp_batch {
  int device = 0;
  cudaStream_t stream = nullptr, user_stream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, t0 = nullptr, t1 = nullptr;
  qp_device_ctx ctx{};
  bool has_alloc = false;
  std::vector<std::pair<void*, size_t>> allocs;
  int32_t count = 0;
  int64_t n_total = 0, m_total = 0;
  int num_sms = 1;
  std::vector<BatchBin> bins;
  cudaEvent_t fork = nullptr;
  BatchDesc* desc = nullptr;
  double *F64 = nullptr, *qd64 = nullptr, *c = nullptr, *b = nullptr;
  double *Aval64 = nullptr, *Tval64 = nullptr;
  float *F32 = nullptr, *qd32 = nullptr, *Aval32 = nullptr, *Tval32 = nullptr;
  float *c32 = nullptr, *b32 = nullptr;
  int32_t *Arp = nullptr, *Acol = nullptr, *Trp = nullptr, *Tcol = nullptr;
  int32_t *Along = nullptr, *Tlong = nullptr;
  double *x0 = nullptr, *y0 = nullptr, *x_out = nullptr, *y_out = nullptr;
  double *lo = nullptr, *hi = nullptr;  // packed variable bounds (allocated on first use)
  float *lo32 = nullptr, *hi32 = nullptr;  // and their FP32 copies
  BatchResult* res = nullptr;
  double* step_pow = nullptr;  // step_decide's power table (kStepPowTable pairs)
  bool warm_set = false, solved = false, bounded = false;
  std::vector<BatchResult> h_res;
  std::vector<int64_t> h_off;  // instance i's variables: packed [h_off[i], h_off[i + 1])
};

namespace {

qp_status balloc(qp_batch* h, void** out, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  bytes = (bytes + 255) & ~size_t(255);
  void* ptr = nullptr;
  if (h->has_alloc) {
    ptr = h->ctx.alloc(bytes, h->ctx.user, h->ctx.stream);
    if (!ptr) {
      berror("device allocator callback returned NULL for %zu bytes", bytes);
      return QP_ERR_OOM;
    }
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    berror("cudaMalloc(%zu) failed", bytes);
    return QP_ERR_OOM;
  }
  h->allocs.emplace_back(ptr, bytes);
  *out = ptr;
  return QP_OK;
}

// Frees one allocation of the handle now (after the handle's stream is idle).
qp_status bfree(qp_batch* h, void* ptr) {
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    if (h->allocs[i].first != ptr) continue;
    BCUDA(cudaStreamSynchronize(h->stream));
    if (h->has_alloc)
      h->ctx.free(ptr, h->allocs[i].second, h->ctx.user, h->ctx.stream);
    else
      BCUDA(cudaFree(ptr));
    h->allocs.erase(h->allocs.begin() + long(i));
    return QP_OK;
  }
  berror("internal: freeing an unknown allocation");
  return QP_ERR_CUDA;
}

template <class T>
qp_status bupload(qp_batch* h, T** dst, const std::vector<T>& src) {
  BTRY(balloc(h, reinterpret_cast<void**>(dst), src.size() * sizeof(T)));
  if (!src.empty())
    BCUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice,
                          h->stream));
  return QP_OK;
}

// out = FP32 copy of in (n values), on the handle's stream.
qp_status convert_float(qp_batch* h, const double* in, float* out, size_t n) {
  if (n > 0) {
    const int grid = int(std::min<size_t>((n + 255) / 256, size_t(h->num_sms) * 8));
    k_to_float<<<grid, 256, 0, h->stream>>>(in, out, (long long)n);
    BCUDA(cudaGetLastError());
  }
  return QP_OK;
}

// f(i) for every i in [0, count), in contiguous ranges on up to `threads`
// host threads.
template <class F>
void host_parallel(int64_t count, int threads, F&& f) {
  parallel_ranges(count, threads, 1, [&](int, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) f(i);
  });
}

int host_threads() {
  return std::min(hw_threads(), 16);
}

// Host-to-device copies through pinned staging, shared by the batch handles
// of the process (two chunks per device, allocated on first use).  The
// sources, pieces laid out one after another in the destination, are packed
// into a chunk by several host threads and copied from there; a chunk's copy
// overlaps the packing of the next.  (A copy from pageable memory goes
// through the driver's own staging, about 10 GB/s on one thread.)  The
// sources may be freed on return.
struct HostPiece {
  const void* src;
  size_t bytes;
};

constexpr size_t kStageChunk = size_t(64) << 20;
constexpr int kStageDevices = 64;

struct Staging {
  std::mutex mu;
  char* buf[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
};

Staging& staging(int device) {
  static Staging s[kStageDevices];
  return s[device];
}

qp_status staged_upload(qp_batch* h, void* dst, const std::vector<HostPiece>& pieces) {
  std::vector<size_t> off(pieces.size() + 1, 0);
  for (size_t i = 0; i < pieces.size(); ++i) off[i + 1] = off[i] + pieces[i].bytes;
  const size_t total = off.back();
  if (total == 0) return QP_OK;
  if (h->device < 0 || h->device >= kStageDevices) {
    berror("device %d beyond the staging table", h->device);
    return QP_ERR_CUDA;
  }
  Staging& S = staging(h->device);
  std::lock_guard<std::mutex> lock(S.mu);
  for (int k = 0; k < 2; ++k) {
    if (!S.buf[k]) BCUDA(cudaMallocHost(&S.buf[k], kStageChunk));
    if (!S.done[k]) BCUDA(cudaEventCreateWithFlags(&S.done[k], cudaEventDisableTiming));
  }
  const int T = host_threads();
  int slot = 0;
  for (size_t start = 0; start < total; start += kStageChunk, slot ^= 1) {
    const size_t len = std::min(kStageChunk, total - start);
    BCUDA(cudaEventSynchronize(S.done[slot]));  // the chunk's previous copy has finished
    char* chunk = S.buf[slot];
    host_parallel(T, T, [&](int64_t t) {
      const size_t a = start + len * size_t(t) / size_t(T);
      const size_t e = start + len * size_t(t + 1) / size_t(T);
      size_t i = size_t(std::upper_bound(off.begin(), off.end(), a) - off.begin()) - 1;
      for (size_t pos = a; pos < e; ++i) {
        const size_t take = std::min(e, off[i + 1]) - pos;
        std::memcpy(chunk + (pos - start), static_cast<const char*>(pieces[i].src) + (pos - off[i]),
                    take);
        pos += take;
      }
    });
    BCUDA(cudaMemcpyAsync(static_cast<char*>(dst) + start, chunk, len, cudaMemcpyHostToDevice,
                          h->stream));
    BCUDA(cudaEventRecord(S.done[slot], h->stream));
  }
  return QP_OK;
}

// A grow-only pinned host buffer of the process for the packed arrays of a
// batch: qp_batch_create writes them there from its host threads and copies
// them to the device from there (a pinned source, no staging).  Its mutex is
// held until those copies have finished.
struct HostArena {
  std::mutex mu;
  char* p = nullptr;
  size_t cap = 0;
};

HostArena& host_arena() {
  static HostArena a;
  return a;
}

qp_status to_float(qp_batch* h, const double* in, float** out, size_t n) {
  BTRY(balloc(h, reinterpret_cast<void**>(out), n * sizeof(float)));
  return convert_float(h, in, *out, n);
}

qp_status begin(qp_batch* h) {
  BCUDA(cudaSetDevice(h->device));
  // the caller's stream; 0 is the legacy default stream (PyTorch's default)
  BCUDA(cudaEventRecord(h->ev_a, h->user_stream));
  BCUDA(cudaStreamWaitEvent(h->stream, h->ev_a, 0));
  return QP_OK;
}

qp_status finish(qp_batch* h) {
  BCUDA(cudaEventRecord(h->ev_b, h->stream));
  BCUDA(cudaStreamWaitEvent(h->user_stream, h->ev_b, 0));
  return QP_OK;
}

bool finite_all(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

template <class V, int NT>
qp_status launch_batch_nt(qp_batch* h, BatchBin& bin, BatchData<V> B) {
  const int ad = B.opt.step_mode == kStepAdaptive ? 1 : 0;
  const int mx = std::is_same<V, float>::value ? 1 : 0;
  const size_t smem = bin.smem[mx][ad], bd = bin.block_doubles[mx][ad];
  int occ = 0;
  BCUDA((BatchLaunch<V, NT>::prepare(smem, &occ)));
  if (occ < 1) {
    berror("batch kernel with %d threads and %zu bytes of shared memory cannot be resident", NT,
           smem);
    return QP_ERR_INVALID_ARG;
  }
  const int grid = std::max(1, std::min(B.count, occ * h->num_sms));
  B.adaptive = ad;
  if (smem == 0) {
    if (bin.ws_doubles < size_t(grid) * bd) {
      void* p = nullptr;
      BTRY(balloc(h, &p, size_t(grid) * bd * sizeof(double)));
      bin.ws = static_cast<double*>(p);
      bin.ws_doubles = size_t(grid) * bd;
    }
    B.ws = bin.ws;
    B.ws_stride = (long long)bd;
  }
  BCUDA((BatchLaunch<V, NT>::launch(grid, smem, bin.stream, B)));
  return QP_OK;
}

template <class V>
qp_status launch_batch(qp_batch* h, BatchBin& bin, const BatchData<V>& B, int threads) {
  switch (threads) {
    case 64: return launch_batch_nt<V, 64>(h, bin, B);
    case 128: return launch_batch_nt<V, 128>(h, bin, B);
    case 256: return launch_batch_nt<V, 256>(h, bin, B);
    case 512: return launch_batch_nt<V, 512>(h, bin, B);
  }
  berror("unsupported block size %d", threads);
  return QP_ERR_INVALID_ARG;
}

template <class V>
BatchData<V> batch_data(qp_batch* h, const BatchBin& bin, const V* F, const V* qd, const V* Av,
                        const V* Tv, const qp_options* o, int count) {
  BatchData<V> B{};
  B.desc = h->desc;
  B.order = bin.order;
  B.count = count;
  B.F = F;
  B.qd = qd;
  B.F64 = h->F64;
  B.qd64 = h->qd64;
  B.c = h->c;
  B.b = h->b;
  B.c32 = h->c32;
  B.b32 = h->b32;
  B.Arp = h->Arp;
  B.Acol = h->Acol;
  B.Aval = Av;
  B.Aval64 = h->Aval64;
  B.Trp = h->Trp;
  B.Tcol = h->Tcol;
  B.Tval = Tv;
  B.Tval64 = h->Tval64;
  B.Along = h->Along;
  B.Tlong = h->Tlong;
  B.x0 = h->x0;
  B.y0 = h->y0;
  B.warm = (o->warm_start == 1 && h->warm_set) ? 1 : 0;
  B.lo = h->bounded ? h->lo : nullptr;
  B.hi = h->bounded ? h->hi : nullptr;
  B.lo32 = h->bounded ? h->lo32 : nullptr;
  B.hi32 = h->bounded ? h->hi32 : nullptr;
  B.x_out = h->x_out;
  B.y_out = h->y_out;
  B.res = h->res;
  B.next = bin.next;
  DevOptions& d = B.opt;
  d.tol = o->tol;
  d.max_iter = o->max_iter;
  d.cg_mode = o->cg_mode;
  d.cg_fixed_n = o->cg_fixed_n;
  d.cg_max = o->cg_max;
  d.restart_mode = o->restart_mode;
  d.cg_eps_factor = o->cg_eps_factor;
  d.beta_suff = o->beta_suff;
  d.beta_nec = o->beta_nec;
  d.beta_art = o->beta_art;
  d.theta_pw = o->theta_pw;
  d.eps_zero = o->eps_zero;
  d.omega0 = o->omega0;
  d.eta_override = o->eta;
  d.pw_update = o->primal_weight_update;
  d.m_eq = 0;
  d.debug_flags = 0;
  d.barrier_timeout_ms = 0;
  d.step_mode = o->step_mode;
  B.pow_table = h->step_pow;
  B.power_iters = o->power_iters;
  B.eval_freq = o->eval_freq;
  B.max_n = bin.max_n;
  B.max_m = bin.max_m;
  B.max_k = bin.max_k;
  return B;
}

// One launch per bin, each with the bin's block size on the bin's stream,
// forked from and joined back into the handle's stream, over the first
// `limit` instances of each bin (limit <= 0: all, as in a solve; the tuner
// samples); the whole is timed with events.
qp_status run_batch(qp_batch* h, const qp_options* o, int limit, double* ms) {
  BCUDA(cudaEventRecord(h->t0, h->stream));
  BCUDA(cudaEventRecord(h->fork, h->stream));
  for (int bi = 0; bi < int(h->bins.size()); ++bi) {
    BatchBin& bin = h->bins[size_t(bi)];
    const int count = limit > 0 ? std::min(limit, bin.count) : bin.count;
    const int nt = bin.threads;
    BCUDA(cudaStreamWaitEvent(bin.stream, h->fork, 0));
    BCUDA(cudaMemsetAsync(bin.next, 0, sizeof(int), bin.stream));
    if (o->precision == QP_PREC_MIXED)
      BTRY(launch_batch<float>(
          h, bin, batch_data<float>(h, bin, h->F32, h->qd32, h->Aval32, h->Tval32, o, count),
          nt));
    else
      BTRY(launch_batch<double>(
          h, bin, batch_data<double>(h, bin, h->F64, h->qd64, h->Aval64, h->Tval64, o, count),
          nt));
    BCUDA(cudaEventRecord(bin.done, bin.stream));
    BCUDA(cudaStreamWaitEvent(h->stream, bin.done, 0));
  }
  BCUDA(cudaEventRecord(h->t1, h->stream));
  BCUDA(cudaEventSynchronize(h->t1));
  float f = 0.f;
  BCUDA(cudaEventElapsedTime(&f, h->t0, h->t1));
  if (ms) *ms = f;
  return QP_OK;
}

qp_status validate_batch_options(const qp_options* o) {
  if (!o || !(o->tol >= 0.0) || o->max_iter < 0 || o->eval_freq < 1 || o->eval_freq > 4096 ||
      (o->cg_mode != QP_CG_ADAPTIVE && o->cg_mode != QP_CG_FIXED) || o->cg_fixed_n < 0 ||
      o->cg_max < 1 ||
      (o->restart_mode != QP_RESTART_ADAPTIVE && o->restart_mode != QP_RESTART_NONE) ||
      o->power_iters < 1 || o->power_iters > 100000 || !(o->eps_zero >= 0.0) ||
      !(o->theta_pw >= 0.0 && o->theta_pw <= 1.0) ||
      (o->precision != QP_PREC_FP64 && o->precision != QP_PREC_MIXED) ||
      (o->step_mode != QP_STEP_FIXED && o->step_mode != QP_STEP_ADAPTIVE)) {
    berror("invalid option value");
    return QP_ERR_INVALID_ARG;
  }
  return QP_OK;
}

qp_status create_batch(qp_batch* h, int32_t count, const qp_instance* inst) {
  std::vector<BatchDesc> desc(static_cast<size_t>(count));
  // 1. Every instance on its own, on host threads: the checks, whether A is
  // canonical (else a canonical copy), its entry count and the long rows of
  // A and A' (A' is built in step 3).  The lowest failing instance gives the
  // error.
  struct Prep {
    HostCsr A;  // the canonical copy, only where A is not canonical
    bool copy = false;
    int64_t nnz = 0;
    int32_t n_along = 0, n_tlong = 0;
  };
  std::vector<Prep> prep(static_cast<size_t>(count));
  std::vector<std::string> err(static_cast<size_t>(count));
  std::atomic<int32_t> first_bad(INT32_MAX);
  auto fail = [&](int32_t i, std::string why) {
    err[size_t(i)] = std::move(why);
    int32_t cur = first_bad.load();
    while (i < cur && !first_bad.compare_exchange_weak(cur, i)) {
    }
  };
  static const int32_t kZeroRowptr[1] = {0};
  // the CSR of instance i's A as used (the caller's arrays or the copy)
  auto a_view = [&](int32_t i) {
    const qp_instance& q = inst[i];
    const Prep& P = prep[size_t(i)];
    if (P.copy) return view_of(P.A);
    return CsrView{q.m, q.n, q.m > 0 ? q.A_rowptr : kZeroRowptr, q.A_col, q.A_val};
  };
  const int nth = host_threads();
  host_parallel(nth, nth, [&](int64_t t) {
    std::vector<int32_t> colcount;  // this thread's, reused across its instances
    for (int64_t ii = int64_t(count) * t / nth; ii < int64_t(count) * (t + 1) / nth; ++ii) {
      const int32_t i = int32_t(ii);
      if (i > first_bad.load()) return;
      const qp_instance& q = inst[i];
      if (q.n < 1 || q.m < 0 || q.m_eq < 0 || q.m_eq > q.m || q.k < 0 || !q.qd || !q.c ||
          (q.k > 0 && !q.F) || (q.m > 0 && (!q.b || !q.A_rowptr))) {
        fail(i, "bad sizes or NULL arrays");
        continue;
      }
      std::string why;
      bool canonical = true;
      if (q.m > 0 && !csr_check(q.m, q.n, q.A_rowptr, q.A_col, q.A_val, &why, &canonical)) {
        fail(i, "A: " + why);
        continue;
      }
      // (F is checked on the device, where it is transposed)
      if (!finite_all(q.qd, size_t(q.n)) || !finite_all(q.c, size_t(q.n)) ||
          (q.m > 0 && !finite_all(q.b, size_t(q.m)))) {
        fail(i, "a value is not finite");
        continue;
      }
      Prep& P = prep[size_t(i)];
      if (!canonical) {
        P.A = csr_canonical(q.m, q.n, q.A_rowptr, q.A_col, q.A_val);
        P.copy = true;
      }
      const CsrView V = a_view(i);
      P.nnz = V.nnz();
      for (int32_t r = 0; r < q.m; ++r)
        P.n_along += V.rowptr[r + 1] - V.rowptr[r] > kBatchLongRow;
      colcount.assign(size_t(q.n), 0);
      for (int64_t k = 0; k < P.nnz; ++k) colcount[size_t(V.col[k])]++;
      for (int32_t j = 0; j < q.n; ++j) P.n_tlong += colcount[size_t(j)] > kBatchLongRow;
    }
  });
  if (first_bad.load() < count) {
    berror("instance %d: %s", first_bad.load(), err[size_t(first_bad.load())].c_str());
    return QP_ERR_INVALID_ARG;
  }
  // 2. Offsets of every instance in the packed arrays (instance order).
  int64_t n_total = 0, m_total = 0, F_total = 0, arp = 0, ann = 0, trp = 0, tnn = 0;
  int32_t al = 0, tl = 0;
  for (int32_t i = 0; i < count; ++i) {
    const qp_instance& q = inst[i];
    const Prep& P = prep[size_t(i)];
    BatchDesc& d = desc[size_t(i)];
    d.n = q.n;
    d.m = q.m;
    d.m_eq = q.m_eq;
    d.k = q.k;
    d.off_n = n_total;
    d.off_m = m_total;
    d.off_F = F_total;
    d.off_Arp = arp;
    d.off_Ann = ann;
    d.off_Trp = trp;
    d.off_Tnn = tnn;
    d.off_Along = al;
    d.off_Tlong = tl;
    d.n_Along = P.n_along;
    d.n_Tlong = P.n_tlong;
    n_total += q.n;
    m_total += q.m;
    F_total += int64_t(q.n) * q.k;
    arp += int64_t(q.m) + 1;
    ann += P.nnz;
    trp += int64_t(q.n) + 1;
    tnn += P.nnz;
    al += d.n_Along;
    tl += d.n_Tlong;
  }
  h->n_total = n_total;
  h->m_total = m_total;
  h->h_off.resize(size_t(count) + 1);
  for (int32_t i = 0; i < count; ++i) h->h_off[size_t(i)] = desc[size_t(i)].off_n;
  h->h_off[size_t(count)] = n_total;
  // bins: instances sorted by n (largest first), cut into equal-count groups
  std::vector<int32_t> ids(static_cast<size_t>(count));
  for (int32_t i = 0; i < count; ++i) ids[size_t(i)] = i;
  std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b2) {
    return desc[size_t(a)].n > desc[size_t(b2)].n;
  });
  int smem_optin = 0;
  BCUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  const size_t static_smem = sizeof(DevState) + 512 / 32 * 13 * sizeof(double) + 64;
  const int nbins = std::min(kMaxBins, int(count));
  h->bins.resize(size_t(nbins));
  for (int bi = 0; bi < nbins; ++bi) {
    BatchBin& bin = h->bins[size_t(bi)];
    const size_t lo = size_t(count) * size_t(bi) / size_t(nbins);
    const size_t hi = size_t(count) * size_t(bi + 1) / size_t(nbins);
    bin.h_order.assign(ids.begin() + long(lo), ids.begin() + long(hi));
    bin.count = int(bin.h_order.size());
    for (int32_t id : bin.h_order) {
      bin.max_n = std::max(bin.max_n, desc[size_t(id)].n);
      bin.max_m = std::max(bin.max_m, desc[size_t(id)].m);
      bin.max_k = std::max(bin.max_k, desc[size_t(id)].k);
    }
    for (int ad = 0; ad < 2; ++ad) {
      bin.block_doubles[0][ad] =
          batch_block_doubles(bin.max_n, bin.max_m, bin.max_k, false, ad != 0);
      bin.block_doubles[1][ad] = batch_block_doubles_mixed(bin.max_n, bin.max_m, bin.max_k);
      for (int mx = 0; mx < 2; ++mx) {
        const size_t need = bin.block_doubles[mx][ad] * sizeof(double);
        bin.smem[mx][ad] = need + static_smem <= size_t(smem_optin) ? need : 0;
      }
    }
    bin.threads = default_threads(bin.max_n, bin.smem[1][1]);
    BCUDA(cudaStreamCreateWithFlags(&bin.stream, cudaStreamNonBlocking));
    BCUDA(cudaEventCreateWithFlags(&bin.done, cudaEventDisableTiming));
    BTRY(bupload(h, &bin.order, bin.h_order));
    BTRY(balloc(h, reinterpret_cast<void**>(&bin.next), sizeof(int)));
  }
  BCUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  BTRY(bupload(h, &h->desc, desc));
  // F: the caller's row-major arrays copied as they are, then transposed and
  // checked on the device
  BTRY(balloc(h, reinterpret_cast<void**>(&h->F64), size_t(F_total) * sizeof(double)));
  if (F_total > 0) {
    double* Frow = nullptr;
    int* bad = nullptr;
    BTRY(balloc(h, reinterpret_cast<void**>(&Frow), size_t(F_total) * sizeof(double)));
    BTRY(balloc(h, reinterpret_cast<void**>(&bad), sizeof(int)));
    std::vector<HostPiece> fp;
    for (int32_t i = 0; i < count; ++i)
      if (inst[i].k > 0) fp.push_back({inst[i].F, size_t(inst[i].n) * size_t(inst[i].k) * 8});
    BTRY(staged_upload(h, Frow, fp));
    const int big = INT_MAX;
    BCUDA(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    const int grid = int(std::min<int64_t>((F_total + 255) / 256, int64_t(h->num_sms) * 8));
    k_F_colmajor<<<grid, 256, 0, h->stream>>>(h->desc, count, Frow, h->F64, (long long)F_total,
                                              bad);
    BCUDA(cudaGetLastError());
    int first_bad = INT_MAX;
    BCUDA(cudaMemcpyAsync(&first_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BCUDA(cudaStreamSynchronize(h->stream));
    BTRY(bfree(h, Frow));
    if (first_bad != INT_MAX) {
      berror("instance %d: a value is not finite", first_bad);
      return QP_ERR_INVALID_ARG;
    }
  }
  // 3. The packed arrays, written by the host threads into the pinned arena
  // (A as used, A' by a stable transpose, the vectors, the long-row lists),
  // then copied to the device from there.
  {
    struct Arr {
      void** dst;
      size_t bytes;
      size_t off = 0;
    };
    Arr arrs[] = {{reinterpret_cast<void**>(&h->qd64), size_t(n_total) * 8},
                  {reinterpret_cast<void**>(&h->c), size_t(n_total) * 8},
                  {reinterpret_cast<void**>(&h->b), size_t(m_total) * 8},
                  {reinterpret_cast<void**>(&h->Arp), size_t(arp) * 4},
                  {reinterpret_cast<void**>(&h->Acol), size_t(ann) * 4},
                  {reinterpret_cast<void**>(&h->Aval64), size_t(ann) * 8},
                  {reinterpret_cast<void**>(&h->Trp), size_t(trp) * 4},
                  {reinterpret_cast<void**>(&h->Tcol), size_t(tnn) * 4},
                  {reinterpret_cast<void**>(&h->Tval64), size_t(tnn) * 8},
                  {reinterpret_cast<void**>(&h->Along), size_t(al) * 4},
                  {reinterpret_cast<void**>(&h->Tlong), size_t(tl) * 4}};
    size_t total = 0;
    for (Arr& x : arrs) {
      x.off = total;
      total += (x.bytes + 255) & ~size_t(255);
    }
    HostArena& H = host_arena();
    std::lock_guard<std::mutex> lock(H.mu);
    if (H.cap < total) {
      const size_t cap = std::max(total, H.cap * 2);
      if (H.p) BCUDA(cudaFreeHost(H.p));
      H.p = nullptr;
      H.cap = 0;
      BCUDA(cudaHostAlloc(reinterpret_cast<void**>(&H.p), cap, cudaHostAllocPortable));
      H.cap = cap;
    }
    double* qd = reinterpret_cast<double*>(H.p + arrs[0].off);
    double* cc = reinterpret_cast<double*>(H.p + arrs[1].off);
    double* bb = reinterpret_cast<double*>(H.p + arrs[2].off);
    int32_t* Arp = reinterpret_cast<int32_t*>(H.p + arrs[3].off);
    int32_t* Acol = reinterpret_cast<int32_t*>(H.p + arrs[4].off);
    double* Av = reinterpret_cast<double*>(H.p + arrs[5].off);
    int32_t* Trp = reinterpret_cast<int32_t*>(H.p + arrs[6].off);
    int32_t* Tcol = reinterpret_cast<int32_t*>(H.p + arrs[7].off);
    double* Tv = reinterpret_cast<double*>(H.p + arrs[8].off);
    int32_t* Along = reinterpret_cast<int32_t*>(H.p + arrs[9].off);
    int32_t* Tlong = reinterpret_cast<int32_t*>(H.p + arrs[10].off);
    host_parallel(count, nth, [&](int64_t ii) {
      const int32_t i = int32_t(ii);
      const qp_instance& q = inst[i];
      const BatchDesc& d = desc[size_t(i)];
      const CsrView V = a_view(i);
      const size_t nz = size_t(prep[size_t(i)].nnz);
      std::memcpy(qd + d.off_n, q.qd, size_t(q.n) * 8);
      std::memcpy(cc + d.off_n, q.c, size_t(q.n) * 8);
      if (q.m > 0) std::memcpy(bb + d.off_m, q.b, size_t(q.m) * 8);
      std::memcpy(Arp + d.off_Arp, V.rowptr, (size_t(q.m) + 1) * 4);
      if (nz > 0) {
        std::memcpy(Acol + d.off_Ann, V.col, nz * 4);
        std::memcpy(Av + d.off_Ann, V.val, nz * 8);
      }
      int32_t* tr = Trp + d.off_Trp;
      csr_transpose(q.m, q.n, V.rowptr, V.col, V.val, tr, Tcol + d.off_Tnn, Tv + d.off_Tnn);
      int32_t* la = Along + d.off_Along;
      for (int32_t r = 0; r < q.m; ++r)
        if (V.rowptr[r + 1] - V.rowptr[r] > kBatchLongRow) *la++ = r;
      int32_t* lt = Tlong + d.off_Tlong;
      for (int32_t r = 0; r < q.n; ++r)
        if (tr[r + 1] - tr[r] > kBatchLongRow) *lt++ = r;
    });
    for (Arr& x : arrs) {
      BTRY(balloc(h, x.dst, x.bytes));
      if (x.bytes > 0)
        BCUDA(cudaMemcpyAsync(*x.dst, H.p + x.off, x.bytes, cudaMemcpyHostToDevice, h->stream));
    }
    BCUDA(cudaStreamSynchronize(h->stream));  // the arena is free again after this
  }
  BTRY(to_float(h, h->F64, &h->F32, size_t(F_total)));
  BTRY(to_float(h, h->qd64, &h->qd32, size_t(n_total)));
  BTRY(to_float(h, h->Aval64, &h->Aval32, size_t(ann)));
  BTRY(to_float(h, h->Tval64, &h->Tval32, size_t(tnn)));
  BTRY(to_float(h, h->c, &h->c32, size_t(n_total)));
  BTRY(to_float(h, h->b, &h->b32, size_t(m_total)));
  for (double** v : {&h->x0, &h->x_out}) {
    BTRY(balloc(h, reinterpret_cast<void**>(v), size_t(h->n_total) * sizeof(double)));
    BCUDA(cudaMemsetAsync(*v, 0, size_t(h->n_total) * sizeof(double), h->stream));
  }
  for (double** v : {&h->y0, &h->y_out}) {
    BTRY(balloc(h, reinterpret_cast<void**>(v), size_t(h->m_total) * sizeof(double)));
    BCUDA(cudaMemsetAsync(*v, 0, size_t(h->m_total) * sizeof(double), h->stream));
  }
  BTRY(balloc(h, reinterpret_cast<void**>(&h->res), size_t(count) * sizeof(BatchResult)));
  BTRY(balloc(h, reinterpret_cast<void**>(&h->step_pow), size_t(2) * kStepPowTable * sizeof(double)));
  k_batch_step_pow<<<h->num_sms * 4, 256, 0, h->stream>>>(h->step_pow, kStepPowTable);
  BCUDA(cudaGetLastError());
  BCUDA(cudaStreamSynchronize(h->stream));  // the host staging vectors die here
  return QP_OK;
}

}  // namespace

extern "C" {

qp_status qp_batch_create(qp_batch** out, int32_t count, const qp_instance* inst,
                          const qp_device_ctx* ctx, uint32_t flags) {
  if (!out) {
    berror("out is NULL");
    return QP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (count < 1 || !inst || flags != 0) {
    berror("bad batch: count %d, flags %u", count, flags);
    return QP_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    berror("no CUDA device visible");
    return QP_ERR_NO_DEVICE;
  }
  qp_batch* h = new qp_batch();
  h->count = count;
  cudaGetDevice(&h->device);
  if (ctx) {
    h->ctx = *ctx;
    h->has_alloc = ctx->alloc && ctx->free;
    h->user_stream = static_cast<cudaStream_t>(ctx->stream);
  }
  qp_status s = QP_OK;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&h->t0) != cudaSuccess || cudaEventCreate(&h->t1) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    berror("stream/event creation failed");
    s = QP_ERR_CUDA;
  }
  if (s == QP_OK) s = begin(h);
  if (s == QP_OK) s = create_batch(h, count, inst);
  if (s == QP_OK) s = finish(h);
  if (s != QP_OK) {
    qp_batch_destroy(h);
    return s;
  }
  *out = h;
  return QP_OK;
}

void qp_batch_destroy(qp_batch* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& a : h->allocs) {
    if (h->has_alloc)
      h->ctx.free(a.first, a.second, h->ctx.user, h->ctx.stream);
    else
      cudaFree(a.first);
  }
  for (BatchBin& bin : h->bins) {
    if (bin.stream) cudaStreamSynchronize(bin.stream);
    if (bin.done) cudaEventDestroy(bin.done);
    if (bin.stream) cudaStreamDestroy(bin.stream);
  }
  for (cudaEvent_t e : {h->ev_a, h->ev_b, h->t0, h->t1, h->fork})
    if (e) cudaEventDestroy(e);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

qp_status qp_batch_solve(qp_batch* h, const qp_options* o, double* device_ms) {
  if (!h) return QP_ERR_INVALID_ARG;
  BTRY(validate_batch_options(o));
  BTRY(begin(h));
  h->solved = false;
  double ms = 0.0;
  BTRY(run_batch(h, o, 0, &ms));
  h->h_res.resize(size_t(h->count));
  BCUDA(cudaMemcpyAsync(h->h_res.data(), h->res, size_t(h->count) * sizeof(BatchResult),
                        cudaMemcpyDeviceToHost, h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  if (device_ms) *device_ms = ms;
  h->solved = true;
  return finish(h);
}

qp_status qp_batch_results(const qp_batch* h, qp_instance_result* out) {
  if (!h || !out) return QP_ERR_INVALID_ARG;
  if (!h->solved) {
    berror("no successful batch solve");
    return QP_ERR_NOT_SOLVED;
  }
  for (int32_t i = 0; i < h->count; ++i) {
    const BatchResult& r = h->h_res[size_t(i)];
    qp_instance_result& o = out[i];
    o.termination = r.termination;
    o.returned_avg = r.returned_avg;
    o.iterations = r.iterations;
    o.cg_steps = r.cg_steps;
    o.restarts = r.restarts;
    o.r_primal = r.kkt[0];
    o.r_dual = r.kkt[1];
    o.r_gap = r.kkt[2];
    o.relkkt = r.kkt[3];
    o.primal_obj = r.kkt[4];
    o.dual_obj = r.kkt[5];
    o.eta = r.eta;
    o.omega = r.omega;
    o.norm_A = r.norm_A;
    o.attempts = r.attempts;
  }
  return QP_OK;
}

qp_status qp_batch_solution(const qp_batch* hc, double* x, double* y) {
  if (!hc) return QP_ERR_INVALID_ARG;
  if (!hc->solved) {
    berror("no successful batch solve");
    return QP_ERR_NOT_SOLVED;
  }
  qp_batch* h = const_cast<qp_batch*>(hc);
  BTRY(begin(h));
  if (x && h->n_total > 0)
    BCUDA(cudaMemcpyAsync(x, h->x_out, size_t(h->n_total) * sizeof(double),
                          cudaMemcpyDeviceToHost, h->stream));
  if (y && h->m_total > 0)
    BCUDA(cudaMemcpyAsync(y, h->y_out, size_t(h->m_total) * sizeof(double),
                          cudaMemcpyDeviceToHost, h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  return finish(h);
}

qp_status qp_batch_set_warm_start(qp_batch* h, const double* x0, const double* y0) {
  if (!h) return QP_ERR_INVALID_ARG;
  // the check on host threads: warm starts of whole batches are millions of values
  std::atomic<bool> ok(true);
  const int nth = host_threads();
  host_parallel(nth, nth, [&](int64_t t) {
    const int64_t N = h->n_total, M = h->m_total;
    if (x0 && !finite_all(x0 + N * t / nth, size_t(N * (t + 1) / nth - N * t / nth))) ok = false;
    if (y0 && !finite_all(y0 + M * t / nth, size_t(M * (t + 1) / nth - M * t / nth))) ok = false;
  });
  if (!ok.load()) {
    berror("warm start holds a non-finite value");
    return QP_ERR_INVALID_ARG;
  }
  BTRY(begin(h));
  const size_t nb = size_t(h->n_total) * sizeof(double), mb = size_t(h->m_total) * sizeof(double);
  if (x0)
    BTRY(staged_upload(h, h->x0, {{x0, nb}}));
  else
    BCUDA(cudaMemsetAsync(h->x0, 0, nb, h->stream));
  if (mb) {
    if (y0)
      BTRY(staged_upload(h, h->y0, {{y0, mb}}));
    else
      BCUDA(cudaMemsetAsync(h->y0, 0, mb, h->stream));
  }
  BCUDA(cudaStreamSynchronize(h->stream));
  h->warm_set = true;
  return finish(h);
}

}  // extern "C"

namespace {

// The bounds of every instance: lo_of(i) / hi_of(i) give instance i's n_i
// values or NULL (that side unbounded); any_lo / any_hi: some instance has
// that side.  The checks run on host threads over the caller's arrays (the
// lowest bad packed variable is reported); the values go through the pinned
// staging chunks straight from those arrays.
template <class LoOf, class HiOf>
qp_status set_bounds_impl(qp_batch* h, LoOf lo_of, HiOf hi_of, bool any_lo, bool any_hi) {
  const int64_t N = h->n_total;
  const int32_t count = h->count;
  std::atomic<int64_t> bad(N);
  std::atomic<bool> any(false);
  const int nth = host_threads();
  host_parallel(nth, nth, [&](int64_t t) {
    bool fin = false;
    for (int64_t ii = int64_t(count) * t / nth; ii < int64_t(count) * (t + 1) / nth; ++ii) {
      const int32_t i = int32_t(ii);
      const double* lo = any_lo ? lo_of(i) : nullptr;
      const double* hi = any_hi ? hi_of(i) : nullptr;
      if (!lo && !hi) continue;
      const int64_t o = h->h_off[size_t(i)], n = h->h_off[size_t(i) + 1] - o;
      for (int64_t v = 0; v < n; ++v) {
        const double l = lo ? lo[v] : -INFINITY, u = hi ? hi[v] : INFINITY;
        if (std::isnan(l) || std::isnan(u) || l > u || l == INFINITY || u == -INFINITY) {
          int64_t cur = bad.load();
          while (o + v < cur && !bad.compare_exchange_weak(cur, o + v)) {
          }
          break;
        }
        fin = fin || std::isfinite(l) || std::isfinite(u);
      }
    }
    if (fin) any = true;
  });
  if (bad.load() < N) {
    const int64_t j = bad.load();
    const int32_t i = int32_t(std::upper_bound(h->h_off.begin(), h->h_off.end(), j) -
                              h->h_off.begin()) - 1;
    const int64_t v = j - h->h_off[size_t(i)];
    const double* lo = any_lo ? lo_of(i) : nullptr;
    const double* hi = any_hi ? hi_of(i) : nullptr;
    berror("invalid bounds at packed variable %lld: [%g, %g]", (long long)j,
           lo ? lo[v] : -INFINITY, hi ? hi[v] : INFINITY);
    return QP_ERR_INVALID_ARG;
  }
  BTRY(begin(h));
  h->solved = false;
  h->bounded = false;  // set again only once both arrays hold the new bounds
  if (any.load()) {
    if (!h->lo) BTRY(balloc(h, reinterpret_cast<void**>(&h->lo), size_t(N) * sizeof(double)));
    if (!h->hi) BTRY(balloc(h, reinterpret_cast<void**>(&h->hi), size_t(N) * sizeof(double)));
    if (!h->lo32) BTRY(balloc(h, reinterpret_cast<void**>(&h->lo32), size_t(N) * sizeof(float)));
    if (!h->hi32) BTRY(balloc(h, reinterpret_cast<void**>(&h->hi32), size_t(N) * sizeof(float)));
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, int64_t(h->num_sms) * 8)));
    int64_t max_n = 0;
    for (int32_t i = 0; i < count; ++i)
      max_n = std::max(max_n, h->h_off[size_t(i) + 1] - h->h_off[size_t(i)]);
    // the pieces of one side, an instance without it read from a run of the fill value
    auto upload_side = [&](auto of, bool present, double fill, double* dst) -> qp_status {
      if (!present) {
        k_fill_f64<<<grid, 256, 0, h->stream>>>(dst, fill, (long long)N);
        return QP_OK;
      }
      const std::vector<double> fills(size_t(std::max<int64_t>(max_n, 1)), fill);
      std::vector<HostPiece> pieces(static_cast<size_t>(count));
      for (int32_t i = 0; i < count; ++i) {
        const double* v = of(i);
        pieces[size_t(i)] = {v ? static_cast<const void*>(v) : fills.data(),
                             size_t(h->h_off[size_t(i) + 1] - h->h_off[size_t(i)]) * sizeof(double)};
      }
      BTRY(staged_upload(h, dst, pieces));
      BCUDA(cudaStreamSynchronize(h->stream));  // fills dies with this call
      return QP_OK;
    };
    BTRY(upload_side(lo_of, any_lo, -INFINITY, h->lo));
    BTRY(upload_side(hi_of, any_hi, INFINITY, h->hi));
    BTRY(convert_float(h, h->lo, h->lo32, size_t(N)));
    BTRY(convert_float(h, h->hi, h->hi32, size_t(N)));
    BCUDA(cudaStreamSynchronize(h->stream));
    h->bounded = true;
  }
  return finish(h);
}

}  // namespace

extern "C" {

qp_status qp_batch_set_bounds(qp_batch* h, const double* lo, const double* hi) {
  if (!h) return QP_ERR_INVALID_ARG;
  const std::vector<int64_t>& off = h->h_off;
  return set_bounds_impl(
      h, [&](int32_t i) { return lo + off[size_t(i)]; },
      [&](int32_t i) { return hi + off[size_t(i)]; }, lo != nullptr, hi != nullptr);
}

qp_status qp_batch_set_bounds_each(qp_batch* h, const double* const* lo, const double* const* hi) {
  if (!h) return QP_ERR_INVALID_ARG;
  return set_bounds_impl(
      h, [&](int32_t i) { return lo[i]; }, [&](int32_t i) { return hi[i]; }, lo != nullptr,
      hi != nullptr);
}

qp_status qp_batch_set_threads(qp_batch* h, int32_t threads) {
  if (!h) return QP_ERR_INVALID_ARG;
  bool ok = threads == 0;
  for (int t : kThreadChoices) ok = ok || t == threads;
  if (!ok) {
    berror("unsupported block size %d", threads);
    return QP_ERR_INVALID_ARG;
  }
  for (BatchBin& bin : h->bins)
    bin.threads = threads == 0 ? default_threads(bin.max_n, bin.smem[1][1]) : threads;
  return QP_OK;
}

qp_status qp_batch_tune(qp_batch* h, const qp_options* o, int32_t sample_count,
                        int32_t sample_iters, int32_t* threads_out) {
  if (!h || sample_count < 1 || sample_iters < 1) return QP_ERR_INVALID_ARG;
  BTRY(validate_batch_options(o));
  qp_options t = *o;
  t.max_iter = std::min<int64_t>(o->max_iter, sample_iters);
  BTRY(begin(h));
  // The bins run concurrently and share the SMs, so each candidate is timed
  // on the whole batch: one bin at a time tries every block size with the
  // others at their current choice (coordinate search, largest bin first).
  for (int bi = 0; bi < int(h->bins.size()); ++bi) {
    BatchBin& bin = h->bins[size_t(bi)];
    double best = INFINITY;
    int best_t = bin.threads;
    for (int threads : kThreadChoices) {
      bin.threads = threads;
      double ms = 0.0;
      qp_status s = run_batch(h, &t, sample_count, &ms);
      if (s == QP_ERR_INVALID_ARG) continue;  // this block size cannot be resident
      BTRY(s);
      if (ms < best) {
        best = ms;
        best_t = threads;
      }
    }
    bin.threads = best_t;
  }
  h->solved = false;  // the sample runs overwrote the outputs
  if (threads_out) *threads_out = h->bins.front().threads;
  return finish(h);
}

}  // extern "C"
