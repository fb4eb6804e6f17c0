// qp_norm_A_static: the ||A||_2 power-iteration estimate of qp_norm_A for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a controller that must run under a
// device-memory budget fixed at start-up (for instance a model-predictive
// control loop re-solving QPs every few milliseconds), code running while
// another framework owns all device memory through its own arena, or code
// that must not trigger the device-wide synchronisation an allocation can
// cause.  This entry point takes its work vectors from a file-scope static
// device array instead, so it allocates nothing.  The array is part of the
// loaded module: every GPU that loads this library holds it until the
// process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "../../include/pdhcg.h"

void pdhcg_set_last_error(const char* msg);  // defined with qp_last_error

namespace {

constexpr int kBlock = 256;

constexpr int kMaxDevices = 64;
constexpr int kMaxBlocks = 148 * 8;  // cap on every launch below: partial-sum slots
constexpr size_t kScratchDoubles = size_t(QP_NORM_A_STATIC_MAX_DOUBLES);

// Layout per call: v[n] | w[n] | u[m] | partial sums[kMaxBlocks] | lambda[1].
__device__ __align__(256) double g_norm_scratch[kScratchDoubles];

struct DeviceSetup {
  std::once_flag once;
  double* scratch = nullptr;  // device address of g_norm_scratch on this device
  int sms = 0;
  cudaError_t err = cudaSuccess;
};
DeviceSetup g_setup[kMaxDevices];

struct Csr {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  int32_t rows;
};

__device__ __forceinline__ long long tid_global() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long threads_global() { return (long long)gridDim.x * blockDim.x; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum; thread 0 writes it to *out.
__device__ __forceinline__ void block_sum(double v, double* out) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double x = lane < int(blockDim.x >> 5) ? sh[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) *out = x;
  }
}

// G lanes per row; the whole warp walks the same row blocks.
template <int G, class F>
__device__ __forceinline__ void rows_loop(const Csr& M, const double* v, F&& f) {
  constexpr int kRows = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  const long long gw = tid_global() >> 5, nw = threads_global() >> 5;
  for (long long base = gw * kRows; base < M.rows; base += nw * kRows) {
    const int i = int(base) + lane / G;
    double s = 0.0;
    if (i < M.rows) {
      const int e = __ldg(M.rowptr + i + 1);
      for (int k = __ldg(M.rowptr + i) + sub; k < e; k += G)
        s = fma(__ldg(M.val + k), v[__ldg(M.col + k)], s);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i < M.rows && sub == 0) f(i, s);
  }
}

// Row-group SpMV out = M v; with part != nullptr also per-block sums of out_i^2.
template <int G>
__global__ void __launch_bounds__(kBlock) k_ns_spmv(Csr M, const double* v, double* out,
                                                    double* part) {
  double acc = 0.0;
  rows_loop<G>(M, v, [&](int i, double s) {
    out[i] = s;
    acc = fma(s, s, acc);
  });
  if (part) block_sum(acc, part + blockIdx.x);
}

__global__ void k_ns_start(double* v, int n) {
  const double v0 = 1.0 / sqrt((double)n);
  for (long long i = tid_global(); i < n; i += threads_global()) v[i] = v0;
}

// v = w / lambda with lambda = ||w||_2 from the partial sums (summed in one
// fixed order by every block); block 0 keeps lambda.
__global__ void k_ns_scale(const double* w, double* v, int n, const double* part, int gp,
                           double* lam_out) {
  __shared__ double s_lam;
  if (threadIdx.x < 32) {
    double x = 0.0;
    for (int i = threadIdx.x; i < gp; i += 32) x += part[i];
    x = warp_sum(x);
    if (threadIdx.x == 0) s_lam = sqrt(x);
  }
  __syncthreads();
  const double lam = s_lam;
  const double inv_lam = lam > 0.0 ? 1.0 / lam : 0.0;
  for (long long i = tid_global(); i < n; i += threads_global()) v[i] = w[i] * inv_lam;
  if (blockIdx.x == 0 && threadIdx.x == 0) *lam_out = lam;
}

__global__ void k_ns_finish(const double* lam, double* out) { *out = sqrt(*lam); }

int lanes_per_row(int64_t nnz, int64_t rows) {
  const double avg = rows > 0 ? double(nnz) / double(rows) : 0.0;
  if (avg <= 24.0) return 1;
  if (avg <= 64.0) return 4;
  if (avg <= 256.0) return 8;
  return 32;
}

template <class F>
bool with_g(int G, F&& f) {
  switch (G) {
    case 1: f(std::integral_constant<int, 1>{}); return true;
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 8: f(std::integral_constant<int, 8>{}); return true;
    case 32: f(std::integral_constant<int, 32>{}); return true;
  }
  return false;
}

int grid_for(int64_t rows, int G, int sms) {
  const int64_t per_block = int64_t(kBlock / 32) * (32 / G);
  const int64_t g = (rows + per_block - 1) / per_block;
  return int(std::max<int64_t>(1, std::min<int64_t>({g, int64_t(sms) * 8, kMaxBlocks})));
}

}  // namespace

extern "C" qp_status qp_norm_A_static(int32_t m, int32_t n, int64_t nnz,
                                      const int32_t* A_rowptr, const int32_t* A_col,
                                      const double* A_val, const int32_t* At_rowptr,
                                      const int32_t* At_col, const double* At_val,
                                      int32_t iters, double* norm_out, void* stream) {
  if (m < 0 || n <= 0 || nnz < 0 || iters < 1 || !norm_out || !A_rowptr || !At_rowptr ||
      (nnz > 0 && (!A_col || !A_val || !At_col || !At_val))) {
    pdhcg_set_last_error("qp_norm_A_static: invalid size or NULL pointer");
    return QP_ERR_INVALID_ARG;
  }
  const size_t need = 2 * size_t(n) + size_t(m) + size_t(kMaxBlocks) + 1;
  if (need > kScratchDoubles) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "qp_norm_A_static: 2n + m = %lld exceeds the static scratch limit %lld",
                  (long long)(2 * size_t(n) + size_t(m)),
                  (long long)(kScratchDoubles - kMaxBlocks - 1));
    pdhcg_set_last_error(msg);
    return QP_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    pdhcg_set_last_error("qp_norm_A_static: no usable current CUDA device");
    return QP_ERR_NO_DEVICE;
  }
  // Once per device, with that device current: resolve the array's device
  // address (a host-side stand-in is not a device pointer) and the SM count.
  DeviceSetup& ds = g_setup[dev];
  std::call_once(ds.once, [&] {
    ds.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&ds.scratch), g_norm_scratch);
    if (ds.err == cudaSuccess)
      ds.err = cudaDeviceGetAttribute(&ds.sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (ds.err != cudaSuccess || !ds.scratch) {
    cudaGetLastError();
    pdhcg_set_last_error("qp_norm_A_static: cudaGetSymbolAddress of the static scratch failed");
    return QP_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* v = ds.scratch;
  double* w = v + n;
  double* u = w + n;
  double* part = u + m;
  double* lam = part + kMaxBlocks;
  // Every slot read below is written earlier in the same call (v by
  // k_ns_start, u and w by the products, the first `gn` partial sums by the
  // A' product, lambda by k_ns_scale), so nothing needs clearing.
  const Csr A{A_rowptr, A_col, A_val, m};
  const Csr At{At_rowptr, At_col, At_val, n};
  const int Ga = lanes_per_row(nnz, m), Gt = lanes_per_row(nnz, n);
  const int gm = grid_for(std::max(m, 1), Ga, ds.sms), gn = grid_for(n, Gt, ds.sms);
  const int gv = grid_for(n, 1, ds.sms);
  k_ns_start<<<gv, kBlock, 0, s>>>(v, n);
  for (int t = 0; t < iters; ++t) {
    with_g(Ga, [&](auto g) {
      k_ns_spmv<decltype(g)::value><<<gm, kBlock, 0, s>>>(A, v, u, nullptr);
    });
    with_g(Gt, [&](auto g) {
      k_ns_spmv<decltype(g)::value><<<gn, kBlock, 0, s>>>(At, u, w, part);
    });
    k_ns_scale<<<gv, kBlock, 0, s>>>(w, v, n, part, gn, lam);
  }
  k_ns_finish<<<1, 1, 0, s>>>(lam, norm_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    pdhcg_set_last_error(cudaGetErrorString(e));
    return QP_ERR_CUDA;
  }
  return QP_OK;
}
