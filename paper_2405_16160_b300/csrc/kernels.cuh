// Device side of the B300 restarted-PDHCG solver (arXiv 2405.16160).
//
// One PDHCG iteration (Algorithm 1 loop body) is three launches:
//   k_cg    cooperative, persistent: the whole inexact CG solve of
//           (Q + I/tau) x = x/tau - c - A'y (Section 2), grid barriers between
//           the SpMV and the vector phases;
//   k_dual  A x+ fused with the projected dual step, the A x cache and the
//           running average of y (Algorithm 1, y-update and averages);
//   k_atv   A' y+ (explicit transpose) fused with the running average of x.
// Every eval_freq iterations: k_spmv (Q x, Q x~, A x~, A' y~), k_kkt_n, k_kkt_m
// (relKKT terms of Section 4 for the current iterate and the average),
// k_control (one warp:
// termination and the restart tests), k_restart_n / k_restart_m /
// k_restart_finish (restart to the candidate and the primal-weight update).
//
// Every vector kernel is templated on the value type T:
//   T = double  the FP64 path (the parity reference on the GPU);
//   T = float   the mixed path: FP32 matrix values, iterates and SpMV
//               arithmetic.  Dot products use exact FP32 products and
//               compensated (double-float) sums up to the block, and FP64
//               across blocks; every scalar of the method (alpha, beta, tau,
//               sigma, omega, eps, relKKT, restart tests) is FP64.  x is held
//               as the restart point x_a (a compensated FP32 pair, fixed for
//               an epoch) plus the FP32 displacement dx, and the iteration
//               runs on dx with b - A x_a in place of b; y and its average
//               are compensated pairs.  A column of A shared by millions of
//               rows would otherwise move all of their dual steps at once
//               each time its FP32 value stepped by an ulp.
// This GPU's FP64 pipe runs at ~1/58 of FP32, so the mixed path keeps FP64
// instructions out of the per-iteration element work (long-row segment sums
// aside, which are a small part of any SpMV).
//
// Reductions never use floating-point atomics: each block writes partials,
// and every consumer reduces them in one fixed order, so results do not
// depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <math_constants.h>
#include <stdint.h>

#include <type_traits>

#include "state.cuh"

namespace pdhcg {

constexpr int kBlock = 256;
constexpr int kCgBlock = 768;  // persistent CG kernel: fewer, larger blocks
constexpr int kPartStride = 16;  // doubles per block in the multi-value partial buffers

// Which entries of the relKKT partial buffers are maxima (bit set) or sums.
constexpr unsigned kKktNMaxMask = 0b0010011100111u;  // 13 entries, see k_kkt_n
constexpr unsigned kKktMMaxMask = 0b1011011u;      // 7 entries, see k_kkt_m

// Rows with more than kLongRow entries are "long": a pre-pass splits them
// into segments of kSegLen entries, one warp per segment, sums each row's
// segments in index order (long_val), and the row kernels read that value.
constexpr int kLongRow = 4096;
constexpr int kSegLen = 2048;

// Rows longer than med_min (and at most kLongRow) are "medium": the row
// kernels leave them to one whole warp each, after the regular rows, so that
// a skewed row-length distribution (a few rows of thousands of entries among
// rows of a handful) does not stall a warp's other row groups.
// How the row kernels hand rows to warps (a runtime choice per matrix and
// precision, picked by qp_tune): rows in groups of 32/G across the whole grid
// in turn; each warp a contiguous range of its own, the same size for every
// warp to within one group; or each block a contiguous range whose groups
// its warps take in turn.
constexpr int kRowsGridStride = 0;
constexpr int kRowsWarpRange = 1;
constexpr int kRowsBlockRange = 2;

template <class T>
struct CsrT {
  const int32_t* rowptr;
  const int32_t* col;
  const T* val;
  int32_t rows;
  const int32_t* long_rows = nullptr;  // ascending ids of the long rows
  const T* long_val = nullptr;         // their products, from the pre-pass
  int32_t nlong = 0;
  const int32_t* med_rows = nullptr;   // ascending ids of the medium rows
  int32_t nmed = 0;
  int32_t med_min = 0x7fffffff;
  int32_t layout = kRowsWarpRange;
};

// Segment table of a matrix's long rows: segment s covers entries
// [seg_begin[s], seg_end[s]); long row r owns segments [seg_ptr[r], seg_ptr[r+1]).
struct LongRows {
  const int32_t* seg_begin = nullptr;
  const int32_t* seg_end = nullptr;
  const int32_t* seg_ptr = nullptr;
  int32_t nseg = 0, nlong = 0;
};


// Grid barrier state.  Barrier number g (gen before it) publishes its value
// (a reduced total, or 0) in slot[g % 2], which holds kSlotOpen while the
// barrier is open; waiting blocks poll that slot, so one load both releases
// them and hands them the value.  The host resets the barrier with
// reset_barrier-style memsets: count 0, gen 0, both slots kSlotOpen.
constexpr unsigned long long kSlotOpen = ~0ull;

struct alignas(128) GridBarrier {
  unsigned int count;
  unsigned int pad0[31];
  unsigned int gen;  // barriers completed, read by a kernel at its start
  unsigned int pad1[31];
  unsigned long long slot[2];
  unsigned long long pad2[14];
  double extra[16];  // totals 2..K of a K-value barrier (written before the slot's release)
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}


__device__ __forceinline__ long long grid_tid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long grid_threads() { return (long long)gridDim.x * blockDim.x; }

// Correctly rounded, never-contracted arithmetic for both value types.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <class T>
constexpr bool kSplit = std::is_same<T, float>::value;

// The CG and BB scalars from their FP64 totals, derived by thread 0 of every
// block right after a grid barrier while the block waits.  FP32 values: in
// FP32, the precision they are applied in (an FP64 division or square root
// is dozens of cycles per instruction on B300's narrow FP64 pipe, on the
// critical path of every barrier).  FP64 values: in FP64, rounded as the
// oracle rounds them.
template <class T>
__device__ __forceinline__ T ratio(double a, double b) {  // a / b
  if constexpr (kSplit<T>)
    return float(a) / float(b);
  else
    return a / b;
}
template <class T>
__device__ __forceinline__ T inv_ratio(double a, double b) {  // 1 / (a / b)
  if constexpr (kSplit<T>)
    return float(b) / float(a);
  else
    return 1.0 / (a / b);
}
template <class T>
__device__ __forceinline__ bool scaled_norm_le(double scale, double sq, double bound) {
  // scale * sqrt(sq) <= bound
  if constexpr (kSplit<T>)
    return float(scale) * sqrtf(float(sq)) <= float(bound);
  else
    return scale * sqrt(sq) <= bound;
}

// 16 bytes of consecutive vector entries (4 floats or 2 doubles), so that the
// streaming vector phases load and store 128 bits at a time.
template <class T>
struct alignas(16) Pack16 {
  static constexpr int N = 16 / int(sizeof(T));
  T v[N];
};


// Dot-product accumulators.  AccD: plain FP64.  AccF: an exact FP32 product
// (two-product via FMA) added into a double-float pair (two-sum), i.e. about
// 48 significant bits without touching the FP64 pipe.
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void merge_shfl(int o) { s += shfl_xor(s, o); }
  __device__ __forceinline__ double value() const { return s; }
};

struct AccF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add2(float a, float ae) {
    const float s = __fadd_rn(hi, a);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, ae));
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    add2(p, fmaf(a, b, -p));
  }
  __device__ __forceinline__ void merge_shfl(int o) {
    const float h = shfl_xor(hi, o), l = shfl_xor(lo, o);
    add2(h, l);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <class T>
struct Acc;
template <>
struct Acc<double> {
  using type = AccD;
};
template <>
struct Acc<float> {
  using type = AccF;
};


template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_xor(v, o));
  return v;
}

template <class A>
__device__ __forceinline__ void warp_merge(A& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a.merge_shfl(o);
}

// Block reduction of KM maxima (of non-negative values, in T) and KS sums
// (accumulators); thread 0 writes out[0..KM) = maxima, out[KM..KM+KS) = sums,
// as doubles.  Only one value per warp is ever widened to FP64.
template <int KM, int KS, class T, class A>
__device__ __forceinline__ void block_reduce_ms(const T* mx, A* sm, double* out) {
  __shared__ double sh[(KM + KS) > 0 ? KM + KS : 1][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const T v = warp_max(mx[k]);
    if (lane == 0) sh[k][wid] = (double)v;
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    warp_merge(sm[k]);
    if (lane == 0) sh[KM + k][wid] = sm[k].value();
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < KM + KS; ++k) {
      double x = lane < nwarps ? sh[k][lane] : 0.0;
      x = k < KM ? warp_max(x) : warp_sum(x);
      if (lane == 0) out[k] = x;
    }
  }
  __syncthreads();
}

template <class A>
__device__ __forceinline__ void block_sum_store(A a, double* out) {
  block_reduce_ms<0, 1, double, A>(nullptr, &a, out);
}

// Per-block partial of a dot product inside the persistent CG kernel.  FP64:
// the double sum.  FP32: the double-float pair stored in the same 8 bytes, so
// the grid-wide combine also stays on the FP32 pipe.
__device__ __forceinline__ void block_dot_store(AccD a, double* out) { block_sum_store(a, out); }

__device__ __forceinline__ void block_dot_store(AccF a, double* out) {
  __shared__ float2 sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  warp_merge(a);
  if (lane == 0) sh[wid] = make_float2(a.hi, a.lo);
  __syncthreads();
  if (wid == 0) {
    AccF b;
    if (lane < int(blockDim.x >> 5)) {
      b.hi = sh[lane].x;
      b.lo = sh[lane].y;
    }
    warp_merge(b);
    if (lane == 0) *reinterpret_cast<float2*>(out) = make_float2(b.hi, b.lo);
  }
  __syncthreads();
}

// Fixed-order reductions of block partials by a whole block.  A grid-wide
// total is read right after a grid barrier or by the last block to finish,
// so it sits on the critical path: every thread issues its loads together
// (one round trip to L2 instead of one per partial a lane would walk), then
// the warps combine by xor shuffles and warp 0 combines the warps in index
// order.  The order depends only on the partial count and blockDim, so the
// result is the same on every run and in every block that computes it.
//
// Row i of the partials is part + i * stride with K entries; bit k of maxmask
// marks entry k as a maximum (of non-negative values), the others are sums.
// Every thread gets the totals.
template <int K, int RB = (K > 4 ? 2 : 4)>
__device__ __forceinline__ void block_reduce_rows(const double* part, int nrows, int stride,
                                                  unsigned maxmask, double (&out)[K]) {
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int base = threadIdx.x; base < nrows; base += RB * blockDim.x) {
    double v[RB][K];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const int i = base + j * int(blockDim.x);
#pragma unroll
      for (int k = 0; k < K; ++k) v[j][k] = i < nrows ? __ldcg(part + size_t(i) * stride + k) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
      for (int k = 0; k < K; ++k)
        acc[k] = ((maxmask >> k) & 1u) ? fmax(acc[k], v[j][k]) : acc[k] + v[j][k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double x = ((maxmask >> k) & 1u) ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < nwarps ? sh[k][lane] : 0.0;
      x = ((maxmask >> k) & 1u) ? warp_max(x) : warp_sum(x);
      if (lane == 0) sh[k][0] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = sh[k][0];
  __syncthreads();
}

// The total of n block_dot_store partials.  FP64: their plain sum.  FP32:
// the double-float pairs added two-sum style, on the FP32 pipe.  RB loads in
// flight per thread (1 where n <= blockDim, as in the persistent CG grid).
template <int RB>
__device__ __forceinline__ double block_total_dot(const double* p, int n, AccD) {
  double t[1];
  block_reduce_rows<1, RB>(p, n, 1, 0u, t);
  return t[0];
}

template <int RB>
__device__ __forceinline__ double block_total_dot(const double* p, int n, AccF) {
  __shared__ float2 sh[32];
  __shared__ double s_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  AccF a;
  for (int base = threadIdx.x; base < n; base += RB * blockDim.x) {
    float2 v[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const int i = base + j * int(blockDim.x);
      v[j] = i < n ? __ldcg(reinterpret_cast<const float2*>(p) + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < RB; ++j) a.add2(v[j].x, v[j].y);
  }
  warp_merge(a);
  if (lane == 0) sh[wid] = make_float2(a.hi, a.lo);
  __syncthreads();
  if (wid == 0) {
    AccF b;
    if (lane < int(blockDim.x >> 5)) {
      b.hi = sh[lane].x;
      b.lo = sh[lane].y;
    }
    warp_merge(b);
    if (lane == 0) s_tot = b.value();
  }
  __syncthreads();
  const double v = s_tot;
  __syncthreads();
  return v;
}


// KS sums per block in the layout of block_dot_store: for AccF each total is
// a double-float pair in its 8-byte slot, so the consumer also combines them
// on the FP32 pipe; for AccD plain doubles.  Thread 0 writes out[0..KS).
template <int KS, class A>
__device__ __forceinline__ void block_pairs_store(A (&a)[KS], double* out) {
  if constexpr (std::is_same<A, AccF>::value) {
    __shared__ float2 sh[KS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      warp_merge(a[k]);
      if (lane == 0) sh[k][wid] = make_float2(a[k].hi, a[k].lo);
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        AccF b;
        if (lane < int(blockDim.x >> 5)) {
          b.hi = sh[k][lane].x;
          b.lo = sh[k][lane].y;
        }
        warp_merge(b);
        if (lane == 0) reinterpret_cast<float2*>(out)[k] = make_float2(b.hi, b.lo);
      }
    }
    __syncthreads();
  } else {
    block_reduce_ms<0, KS, double, AccD>(nullptr, a, out);
  }
}

// The totals of nrows rows of K block_pairs_store partials (row r at
// part + r * K), combined in index order by the whole block; every thread
// gets them.  AccF: double-float pairs on the FP32 pipe; AccD: doubles.
template <int K, class A>
__device__ __forceinline__ void block_pairs_total(const double* part, int nrows, double (&out)[K]) {
  if constexpr (std::is_same<A, AccF>::value) {
    __shared__ float2 sh[K][32];
    __shared__ double s_out[K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    AccF acc[K];
    const float2* p2 = reinterpret_cast<const float2*>(part);
    // rows t, t + blockDim, t + 2 blockDim, ... in that order, eight rows'
    // loads in flight at once (a row past the end adds an exact zero)
    constexpr int RB = 8;
    for (int base = threadIdx.x; base < nrows; base += RB * int(blockDim.x)) {
      float2 v[RB][K];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int r = base + j * int(blockDim.x);
#pragma unroll
        for (int k = 0; k < K; ++k)
          v[j][k] = r < nrows ? __ldcg(p2 + size_t(r) * K + k) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k].add2(v[j][k].x, v[j][k].y);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      warp_merge(acc[k]);
      if (lane == 0) sh[k][wid] = make_float2(acc[k].hi, acc[k].lo);
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        AccF b;
        if (lane < int(blockDim.x >> 5)) {
          b.hi = sh[k][lane].x;
          b.lo = sh[k][lane].y;
        }
        warp_merge(b);
        if (lane == 0) s_out[k] = b.value();
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = s_out[k];
    __syncthreads();
  } else {
    block_reduce_rows<K>(part, nrows, K, 0u, out);
  }
}

// Barrier over all blocks of a co-resident grid that can also reduce one
// partial per block (block_dot_store layout) to a total.  Each block's
// thread 0 holds the barrier number in gen_local (grid_gen at the kernel's
// start, then advanced by every barrier).  Arriving: after the block's
// __syncthreads, thread 0 counts with an acquire-release add, which makes
// the block's writes visible to whoever acquires the count after it (no
// separate fence).  The block that arrives last sums the partials in index order
// (block_total_dot, so the value does not depend on which block is last),
// re-opens the next barrier's slot, resets the count and publishes the total
// in this barrier's slot with release order; the others poll that slot.  One
// block reads the partials instead of every block, so their L2 lines are not
// read by the whole grid at once, and the waiting blocks get the total with
// the same load that releases them.
//
// on_total(total) runs in thread 0 of every block once the total is known,
// before the block's closing barrier: the place to derive the method's FP64
// scalars once per block and share them through shared memory (the FP64
// pipe of B300 runs at 1/58 of FP32, so a division or square root evaluated
// by every thread of a persistent grid costs microseconds).
//
// Every wait is bounded: after opt.barrier_timeout_ms (globaltimer) or 2^27
// polls the block records kErrBarrierTimeout and the kernel winds down; a
// block that sees the error flag stops waiting too.  Returns false on error.
__device__ __forceinline__ unsigned int grid_gen(GridBarrier* bar) {
  unsigned int g = 0u;
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(bar->gen);
    g = gen.load(cuda::memory_order_acquire);
  }
  return g;
}

// K > 1: K totals per barrier (block_pairs_store layout, K per block); the
// last block publishes the first in the slot and the others in the barrier's
// extra line, which block 0 alone reads after the slot releases it (the
// other blocks see 0 for them: one dependent L2 load fewer on their way
// out).
template <class A, int K = 1, class F>
__device__ __forceinline__ bool grid_sync_sum(GridBarrier* bar, DevState* st, int timeout_ms,
                                              bool never_release, unsigned int& gen_local,
                                              const double* part, F&& on_total) {
  __shared__ int s_ok, s_last;
  __syncthreads();
  const unsigned int g = gen_local;
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar->count);
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> slot(bar->slot[g & 1u]);
  if (threadIdx.x == 0) {
    const unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    s_last = arrived == gridDim.x - 1 && !never_release;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {  // the whole last block (the branch is uniform)
    double t[K];
    if constexpr (K == 1) {
      t[0] = part ? block_total_dot<1>(part, gridDim.x, A()) : 0.0;
    } else {
      block_pairs_total<K, A>(part, gridDim.x, t);
    }
    if (threadIdx.x == 0) {
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> next(
          bar->slot[(g + 1u) & 1u]);
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(bar->gen);
      unsigned long long bits = (unsigned long long)__double_as_longlong(t[0]);
      if (bits == kSlotOpen) bits = 0x7ff8000000000000ull;  // a NaN either way
      t[0] = __longlong_as_double((long long)bits);
#pragma unroll
      for (int k = 1; k < K; ++k) bar->extra[k - 1] = t[k];
      next.store(kSlotOpen, cuda::memory_order_relaxed);
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.store(g + 1u, cuda::memory_order_relaxed);
      slot.store(bits, cuda::memory_order_release);
      on_total(static_cast<const double*>(t));
    }
  } else if (threadIdx.x == 0) {
    cuda::atomic_ref<int, cuda::thread_scope_device> err(st->err);
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = (unsigned long long)timeout_ms * 1000000ull;
    unsigned int polls = 0;
    unsigned long long v;
    while ((v = slot.load(cuda::memory_order_acquire)) == kSlotOpen) {
      if (err.load(cuda::memory_order_relaxed) != 0) {
        s_ok = 0;
        break;
      }
      if ((++polls & 255u) == 0u) {
        if (global_ns() - t0 > limit || polls > (1u << 27)) {
          err.fetch_or(kErrBarrierTimeout, cuda::memory_order_relaxed);
          s_ok = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    if (s_ok) {
      double t[K];
      t[0] = __longlong_as_double((long long)v);
#pragma unroll
      for (int k = 1; k < K; ++k) t[k] = blockIdx.x == 0 ? __ldcg(&bar->extra[k - 1]) : 0.0;
      on_total(static_cast<const double*>(t));
    }
  }
  if (threadIdx.x == 0) gen_local = g + 1u;
  __syncthreads();
  return s_ok != 0;
}

// The plain barrier: no partials to reduce.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, DevState* st, int timeout_ms,
                                          bool never_release, unsigned int& gen_local) {
  return grid_sync_sum<AccD>(bar, st, timeout_ms, never_release, gen_local, nullptr,
                             [](const double*) {});
}

// Row-group CSR SpMV: G lanes share a row (G in {1,2,4,8,16,32}); all 32 lanes
// of a warp walk the same number of row blocks, so the group shuffles never
// diverge.  Each lane takes the entries k, k+G, k+2G, ... of its row, four per
// trip: the four column and value loads are issued first, then the four
// gathers, then the four FMAs in entry order (slots past the row end add an
// exact zero), so memory latency is paid once per four entries while the sum
// is the plain strided one.  The group reduces with xor shuffles, so a row's
// sum does not depend on the launch configuration.  f(i, sum, leader) is
// called by every lane of the group; `leader` is lane 0 of the group.
constexpr int kUnroll = 4;

template <int G, class T>
__device__ __forceinline__ T row_dot(const CsrT<T>& M, const T* v, int b, int e, int sub) {
  T s = T(0);
  for (int k = b + sub; k < e; k += kUnroll * G) {
    int c[kUnroll];
    T a[kUnroll], xv[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) {
      const int kk = k + j * G;
      c[j] = kk < e ? __ldg(M.col + kk) : -1;
      a[j] = kk < e ? __ldg(M.val + kk) : T(0);
    }
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) xv[j] = c[j] >= 0 ? v[c[j]] : T(0);
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) s = fma(a[j], xv[j], s);
  }
  return s;
}

// Index of long row i in M.long_rows (binary search; only called for long rows).
template <class T>
__device__ __forceinline__ int long_slot(const CsrT<T>& M, int i) {
  int lo = 0, hi = M.nlong - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(M.long_rows + mid) < i)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The row kernels' template parameter GM is the group size G, plus kMedRows
// when the matrix has medium rows (so that matrices without them run the
// plain row loop).
constexpr int kMedRows = 64;

// blocks: how many blocks of the grid (the first ones) share the rows; by
// default the whole grid.
template <int GM, class T, class F>
__device__ __forceinline__ void spmv_rows(const CsrT<T>& M, const T* v, F&& f, int blocks = 0) {
  constexpr int G = GM & (kMedRows - 1);
  constexpr bool kMed = (GM & kMedRows) != 0;
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int nb = blocks > 0 ? blocks : int(gridDim.x);
  const long long gw = grid_tid() >> 5;
  const long long nw = ((long long)nb * blockDim.x) >> 5;
  int start, end, step;  // the warp's row groups: base = start, start + step, ... < end
  if (M.layout == kRowsGridStride) {
    start = int(gw) * kRowsPerWarp;
    end = M.rows;
    step = int(nw) * kRowsPerWarp;
  } else if (M.layout == kRowsWarpRange) {
    start = int((long long)M.rows * gw / nw);
    end = int((long long)M.rows * (gw + 1) / nw);
    step = kRowsPerWarp;
  } else {
    const int wpb = int(blockDim.x >> 5);
    start = int((long long)M.rows * blockIdx.x / nb) + int(threadIdx.x >> 5) * kRowsPerWarp;
    end = int((long long)M.rows * (blockIdx.x + 1) / nb);
    step = wpb * kRowsPerWarp;
  }
  for (int base = start; base < end; base += step) {
    const int i = base + lane / G;
    T s = T(0);
    bool own = i < end;
    if (own) {
      const int b = __ldg(M.rowptr + i), e = __ldg(M.rowptr + i + 1);
      if (e - b > kLongRow) {
        if (sub == 0) s = M.long_val[long_slot(M, i)];
      } else if (kMed && e - b > M.med_min) {
        own = false;  // a medium row: taken by a whole warp below
      } else {
        s = row_dot<G>(M, v, b, e, sub);
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += shfl_xor(s, o);
    if (own) f(i, s, sub == 0);
  }
  if constexpr (kMed) {
    for (long long w = gw; w < M.nmed; w += nw) {
      const int i = __ldg(M.med_rows + w);
      T s = row_dot<32>(M, v, __ldg(M.rowptr + i), __ldg(M.rowptr + i + 1), lane);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
      f(i, s, lane == 0);
    }
  }
}

// Rows handed out in chunks: a block takes chunk after chunk of kChunkRows
// rows from *counter (an atomic, zero at the launch; the kernel's last block
// puts it back to zero) until none is left, so the SMs that run faster take
// more of them and the launch ends with the slowest SM's last chunk rather
// than with its fixed share.  A chunk's rows go to the block's warps as in
// the block-range layout; chunk_end(c) runs once a chunk is done (the place
// to store the chunk's partial sums: they are indexed by chunk, so the sums
// do not depend on which block took which chunk).  Medium rows are left to
// the caller (spmv_rows' second loop), long rows read the segment pass.
constexpr int kChunkRows = 512;

template <int GM, class T, class F, class E>
__device__ __forceinline__ void spmv_rows_chunked(const CsrT<T>& M, const T* v,
                                                  unsigned int* counter, F&& f, E&& chunk_end) {
  constexpr int G = GM & (kMedRows - 1);
  constexpr bool kMed = (GM & kMedRows) != 0;
  constexpr int kRowsPerWarp = 32 / G;
  __shared__ int s_chunk;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int wpb = int(blockDim.x >> 5);
  const int nchunks = (M.rows + kChunkRows - 1) / kChunkRows;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = int(atomicAdd(counter, 1u));
    __syncthreads();
    const int c = s_chunk;
    if (c >= nchunks) break;
    const int end = min(M.rows, (c + 1) * kChunkRows);
    for (int base = c * kChunkRows + int(threadIdx.x >> 5) * kRowsPerWarp; base < end;
         base += wpb * kRowsPerWarp) {
      const int i = base + lane / G;
      T sum = T(0);
      bool own = i < end;
      if (own) {
        const int b = __ldg(M.rowptr + i), e = __ldg(M.rowptr + i + 1);
        if (e - b > kLongRow) {
          if (sub == 0) sum = M.long_val[long_slot(M, i)];
        } else if (kMed && e - b > M.med_min) {
          own = false;  // a medium row: taken by a whole warp in the caller's pass
        } else {
          sum = row_dot<G>(M, v, b, e, sub);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sum += shfl_xor(sum, o);
      if (own) f(i, sum, sub == 0);
    }
    chunk_end(c);  // synchronises the block before s_chunk is written again
  }
}

// The medium rows of M (a whole warp each), over the first `blocks` blocks
// of the grid: spmv_rows' second loop on its own.
template <int GM, class T, class F>
__device__ __forceinline__ void spmv_medium_rows(const CsrT<T>& M, const T* v, F&& f,
                                                 int blocks) {
  if constexpr ((GM & kMedRows) != 0) {
    const int lane = threadIdx.x & 31;
    const long long gw = grid_tid() >> 5;
    const long long nw = ((long long)blocks * blockDim.x) >> 5;
    for (long long w = gw; w < M.nmed; w += nw) {
      const int i = __ldg(M.med_rows + w);
      T sum = row_dot<32>(M, v, __ldg(M.rowptr + i), __ldg(M.rowptr + i + 1), lane);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += shfl_xor(sum, o);
      f(i, sum, lane == 0);
    }
  }
}

// Segment sum of a long row by a whole warp (the warp's total, for every
// lane), with the sum carried beyond FP32.  A row of millions of entries
// would otherwise pick up an FP32 rounding error that grows with its length,
// on exactly the coordinates (high-degree columns of A, i.e. long rows of A')
// where the scaled residual is smallest.  FP32 values: each product is
// formed exactly (two-product) and summed in double-float on the FP32 pipe
// (FP64 arithmetic runs at 1/58 of FP32 here); FP64 values: plain FP64.
template <class T>
__device__ __forceinline__ double row_dot_wide(const CsrT<T>& M, const T* v, int b, int e,
                                               int lane) {
  typename Acc<T>::type s;
  for (int k = b + lane; k < e; k += kUnroll * 32) {
    int c[kUnroll];
    T a[kUnroll], xv[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) {
      const int kk = k + j * 32;
      c[j] = kk < e ? __ldg(M.col + kk) : -1;
      a[j] = kk < e ? __ldg(M.val + kk) : T(0);
    }
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) xv[j] = c[j] >= 0 ? v[c[j]] : T(0);
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) s.add_prod(a[j], xv[j]);
  }
  warp_merge(s);
  return s.value();
}

// Long-row pre-pass, phase 1: one warp per segment (grid-stride over warps).
// Each segment is summed beyond FP32 (row_dot_wide).
template <class T>
__device__ __forceinline__ void long_segments(const CsrT<T>& M, const T* v, const LongRows& L,
                                              T* seg_part) {
  const int lane = threadIdx.x & 31;
  const long long nw = grid_threads() >> 5;
  for (long long sg = grid_tid() >> 5; sg < L.nseg; sg += nw) {
    const int e = __ldg(L.seg_end + sg);
    const double s = row_dot_wide(M, v, __ldg(L.seg_begin + sg), e, lane);
    if (lane == 0) seg_part[sg] = T(s);
  }
}

// Phase 2: one warp per long row sums its segments in index order (in FP64).
template <class T>
__device__ __forceinline__ void long_finish(const LongRows& L, const T* seg_part, T* long_val) {
  const int lane = threadIdx.x & 31;
  const long long nw = grid_threads() >> 5;
  for (long long r = grid_tid() >> 5; r < L.nlong; r += nw) {
    double s = 0.0;
    const int e = __ldg(L.seg_ptr + r + 1);
    // four loads in flight per lane; the additions keep the order k, k+32, ...
    for (int k = __ldg(L.seg_ptr + r) + lane; k < e; k += 4 * 32) {
      double v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = k + 32 * j < e ? (double)__ldcg(seg_part + k + 32 * j) : 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) s += v[j];
    }
    s = warp_sum(s);
    if (lane == 0) long_val[r] = T(s);
  }
}

// v_trial (may be null): the vector to read instead of v after an accepted
// attempt of the adaptive step (the trial y, before it is committed).
template <class T>
__global__ void __launch_bounds__(kBlock) k_long_segments(CsrT<T> M, const T* __restrict__ v,
                                                          LongRows L, T* seg_part,
                                                          const T* __restrict__ v_trial = nullptr,
                                                          const DevState* st = nullptr) {
  const bool trial = v_trial != nullptr && st->iter_active && st->accepted;
  long_segments(M, trial ? v_trial : v, L, seg_part);
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_long_finish(LongRows L, const T* seg_part,
                                                        T* long_val) {
  long_finish(L, seg_part, long_val);
}

// Block partial of r0'r0, and the grid total written by the last block to
// finish (ticket counter, reset by that block) into part[gridDim.x], so the
// CG kernel reads one value.  The summation order is fixed: the last block
// reduces all partials in index order.
// blocks: the blocks taking part (the first ones; default the whole grid).
// The "last block finishes" ticket: called by thread 0 after the block's
// __syncthreads, it counts the block with an acquire-release add, which
// publishes the block's writes to the block that counts last and lets that
// block see every other block's (no separate fences).  True for the block
// that takes the last of n tickets.
__device__ __forceinline__ bool take_ticket(unsigned int* ticket, unsigned int n) {
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> t(*ticket);
  return t.fetch_add(1u, cuda::memory_order_acq_rel) == n - 1u;
}

template <class A>
__device__ __forceinline__ void store_and_finish_dot(A acc, double* part, unsigned int* ticket,
                                                     int blocks = 0) {
  __shared__ int s_last;
  const int nb = blocks > 0 ? blocks : int(gridDim.x);
  block_dot_store(acc, part + blockIdx.x);
  if (threadIdx.x == 0) s_last = take_ticket(ticket, unsigned(nb));
  __syncthreads();
  if (s_last) {  // the whole last block (the branch is uniform)
    const double total = block_total_dot<4>(part, nb, A());
    if (threadIdx.x == 0) {
      part[nb] = total;
      *ticket = 0u;  // for the next launch (ordered by the kernel boundary)
    }
  }
}

// ------------------------------------------------------------- CG (Section 2)
// Inexact CG on (Q + I/tau) x = x^k/tau - c - A'y^k warm-started at x^k.  Its
// initial residual simplifies to r0 = -(Q x^k + c + A'y^k); the kernel that
// produces A'y^k (k_atv, or k_prepare after a set-up, evaluation or restart)
// also forms r0 = p0 and r0'r0 (one value, r0r0) from a tracked qx = Q x.
// Two grid barriers per CG step:
//   [A] gather r: Q r.  First step (p = r): Qp = Q r.  Later steps:
//       Qp = Q r + beta Qp and p = r + beta p, formed row by row in the
//       product's epilogue; then q = Qp + p/tau and p'q.          | barrier
//   [B] x += a p, qx += a Qp, r -= a q, r'r.                       | barrier
// The product of a continued step reads r, which is complete after [B]'s
// barrier, instead of the new p, which would need a separate pass and a
// third barrier; Q p = Q r + beta Q p_old is the same vector in exact
// arithmetic (textbook CG's p = r + beta p_old, multiplied by Q), so alpha,
// beta and the iterates are those of textbook CG up to rounding.  Each step
// costs one product with Q.  With the adaptive step size the iteration
// counters wait for the accept/reject decision that k_dual's last block
// takes.  Every dot product is FP64-accurate for both value types; alpha,
// beta and the stop test are derived from them in the value type's precision
// (ratio, scaled_norm_le).  part holds 2 * gridDim.x doubles.
// Resident CG blocks per SM: two of 768 threads, 48 warps per SM at 40
// registers a thread (65536 / (768 * 2)), the warps of three 512-thread
// blocks with a third fewer blocks arriving at every grid barrier (measured
// slightly faster); four blocks of 512 would need 32 registers and spill.
constexpr int kCgBlocksPerSm = 2;

// Adaptive step size: the attempt's primal move from its saved start (x_save,
// qx_save), ||x+ - x||^2 and (x+ - x)'(Q x+ - Q x).  The CG kernel sums them
// in each step's phase B and totals them in that step's closing barrier;
// block 0 writes the last step's two totals to part[0..1].  The BB kernel
// sums them in a pass after its last step into part[2 * block] (block
// partials).  k_dual's last block combines them with its own sums.
// part == nullptr: fixed step.
template <class T>
struct StepStart {
  const T* x_save = nullptr;
  const T* qx_save = nullptr;
  double* part = nullptr;
};

template <class T, class A>
__device__ __forceinline__ void step_start_sums(const StepStart<T>& ss, const T* x, const T* qx,
                                                int n) {
  A acc[2];
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const T dx = x[i] - ss.x_save[i], dq = qx[i] - ss.qx_save[i];
    acc[0].add_prod(dx, dx);
    acc[1].add_prod(dx, dq);
  }
  block_pairs_store<2>(acc, ss.part + 2 * size_t(blockIdx.x));
}

template <int G, class T>
__global__ void __launch_bounds__(kCgBlock, kCgBlocksPerSm)
    k_cg(CsrT<T> Q, LongRows LQ, T* qseg, T* qlong, T* x, T* r, T* p, T* q, T* qx,
         const double* r0r0, double* part, DevState* st, GridBarrier* bar, int n,
         StepStart<T> ss) {
  using A = typename Acc<T>::type;
  const bool active = running(st) && st->attempts < st->opt.max_iter;
  if (!active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iter_active = 0;
    return;
  }
  // Every read of st happens before the first barrier; block 0 writes the
  // counters only after the last one.  The FP64 scalars (tau, eps, r'r,
  // alpha, beta, the stop test) live in thread 0 of each block, which shares
  // what the other threads need through shared memory.
  const int mode = st->opt.cg_mode, nfix = st->opt.cg_fixed_n, cgmax = st->opt.cg_max;
  const bool adaptive_step = st->opt.step_mode == kStepAdaptive;
  const int tmo = st->opt.barrier_timeout_ms;
  bool never_release = (st->opt.debug_flags & kDebugBarrierNeverReleases) != 0u;
  __shared__ double s_tau, s_eps, s_rr;  // thread 0's
  __shared__ double s_mv[2];             // the latest step's primal move sums (block 0's totals)
  __shared__ T s_inv_tau, s_coef;        // 1/tau; alpha, then beta
  __shared__ int s_flag;                 // skip / numerical error / stop
  if (threadIdx.x == 0) {
    s_mv[0] = 0.0;  // no step: x is the attempt's start
    s_mv[1] = 0.0;
    s_tau = st->tau;
    s_eps = mode == kCgAdaptive ? st->eps + st->opt.cg_eps_factor * st->relkkt_last : st->eps;
    s_rr = __ldcg(r0r0);
    s_inv_tau = T(1.0 / s_tau);
    s_flag = (mode == kCgFixed && nfix <= 0) || s_rr == 0.0;
  }
  __syncthreads();
  const T inv_tau = s_inv_tau;
  const bool skip = s_flag != 0;
  double* part_pq = part;                 // one partial per block
  double* part_rr = part + gridDim.x;     // three per block: r'r and the move sums
  const long long t0 = grid_tid(), nt = grid_threads();
  unsigned int gen = grid_gen(bar);
  // adaptive step: the primal move's sums of the latest step, per thread
  A mv[2];
  const bool move_sums = ss.part != nullptr;

  int steps = 0;
  bool numerr = false;
  T beta = T(0);  // 0 in the first step, where p = r
  while (!skip) {
    if (LQ.nlong > 0) {
      // long rows of Q: segment sums, then per-row totals, before the row pass
      long_segments(Q, r, LQ, qseg);
      if (!grid_sync(bar, st, tmo, never_release, gen)) return;
      never_release = false;
      long_finish(LQ, qseg, qlong);
      if (!grid_sync(bar, st, tmo, false, gen)) return;
    }
    A acc;
    const bool first = steps == 0;
    spmv_rows<G>(Q, r, [&](int i, T s, bool lead) {
      if (lead) {
        T qpi, pi;
        if (first) {  // p = r = r0: Q p is the product itself
          qpi = s;
          pi = p[i];
        } else {      // Q p = Q r + beta Q p_old, p = r + beta p_old
          qpi = add_rn(s, mul_rn(beta, q[i]));
          pi = add_rn(r[i], mul_rn(beta, p[i]));
          p[i] = pi;
        }
        q[i] = qpi;  // Q p itself; q = Q p + p/tau is re-formed from it below
        acc.add_prod(pi, qpi + pi * inv_tau);
      }
    });
    block_dot_store(acc, part_pq + blockIdx.x);
    if (!grid_sync_sum<A>(bar, st, tmo, never_release, gen, part_pq, [&](const double* t) {
          const double pq = t[0];
          const bool bad = !(pq > 0.0) || !isfinite(pq);
          s_flag = bad;
          s_coef = bad ? T(0) : ratio<T>(s_rr, pq);
        }))
      return;
    never_release = false;
    if (s_flag) {
      numerr = true;
      break;
    }
    const T alpha = s_coef;
    acc = A();
    mv[0] = A();
    mv[1] = A();
    // x += alpha p, r -= alpha q with a rounded product then a rounded sum,
    // exactly as the elementwise vector statements of textbook CG; qx follows
    // x through the stored Q p (recovering it as q - p/tau would cancel badly
    // in FP32 when 1/tau dominates Q).
    // FP32: 16-byte packs of the five vectors (every buffer is 256-byte
    // aligned), then the tail of n mod 4 entries; each entry's arithmetic is
    // the same either way.  (FP64 packs would not fit the register budget of
    // three 512-thread blocks per SM.)
    {
      using P = Pack16<T>;
      constexpr int N = P::N;
      const long long np = kSplit<T> ? n / N : 0;
      P* xp = reinterpret_cast<P*>(x);
      P* qxp = reinterpret_cast<P*>(qx);
      P* rp = reinterpret_cast<P*>(r);
      const P* pp = reinterpret_cast<const P*>(p);
      const P* qp = reinterpret_cast<const P*>(q);
      const P* xsp = reinterpret_cast<const P*>(ss.x_save);
      const P* qxsp = reinterpret_cast<const P*>(ss.qx_save);
      for (long long i = t0; i < np; i += nt) {
        const P pv = pp[i], qv = qp[i], xv = xp[i], qxv = qxp[i], rv = rp[i];
        P xo, qxo, ro;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T qi = qv.v[j] + pv.v[j] * inv_tau;
          xo.v[j] = add_rn(xv.v[j], mul_rn(alpha, pv.v[j]));
          qxo.v[j] = add_rn(qxv.v[j], mul_rn(alpha, qv.v[j]));
          ro.v[j] = sub_rn(rv.v[j], mul_rn(alpha, qi));
          acc.add_prod(ro.v[j], ro.v[j]);
        }
        xp[i] = xo;
        qxp[i] = qxo;
        rp[i] = ro;
        if (move_sums) {  // ||x+ - x||^2 and (x+ - x)'(Q x+ - Q x) from the attempt's start
          const P xs = xsp[i], qxs = qxsp[i];
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const T dx = xo.v[j] - xs.v[j];
            mv[0].add_prod(dx, dx);
            mv[1].add_prod(dx, qxo.v[j] - qxs.v[j]);
          }
        }
      }
      for (long long i = np * N + t0; i < n; i += nt) {
        const T pi = p[i], qpi = q[i];
        const T qi = qpi + pi * inv_tau;
        const T xn = add_rn(x[i], mul_rn(alpha, pi));
        const T qxn = add_rn(qx[i], mul_rn(alpha, qpi));
        x[i] = xn;
        qx[i] = qxn;
        const T ri = sub_rn(r[i], mul_rn(alpha, qi));
        r[i] = ri;
        acc.add_prod(ri, ri);
        if (move_sums) {
          const T dx = xn - ss.x_save[i];
          mv[0].add_prod(dx, dx);
          mv[1].add_prod(dx, qxn - ss.qx_save[i]);
        }
      }
    }
    A sums[3] = {acc, mv[0], mv[1]};
    block_pairs_store<3>(sums, part_rr + 3 * size_t(blockIdx.x));
    if (!grid_sync_sum<A, 3>(bar, st, tmo, false, gen, part_rr, [&](const double* t) {
          const double rr_new = t[0];
          s_mv[0] = t[1];
          s_mv[1] = t[2];
          const int done_steps = steps + 1;
          const bool stop = mode == kCgFixed
                                ? done_steps >= nfix
                                : (scaled_norm_le<T>(s_tau, rr_new, s_eps) ||
                                   done_steps >= cgmax);
          s_flag = stop || rr_new == 0.0;
          s_coef = ratio<T>(rr_new, s_rr);
          s_rr = rr_new;
        }))
      return;
    ++steps;
    if (s_flag) break;
    beta = s_coef;
  }
  // the totals of the last step's move sums are the attempt's primal move (a
  // launch with no step leaves x = x_save: both are zero)
  if (move_sums && !numerr && blockIdx.x == 0 && threadIdx.x == 0) {
    ss.part[0] = s_mv[0];
    ss.part[1] = s_mv[1];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (numerr) {
      st->done = kDoneNumerical;
      st->iter_active = 0;
    } else {
      st->iter_active = 1;
      st->attempts += 1;
      st->cg_total += steps;
      st->last_cg = steps;
      st->spmv_total += steps;
      if (adaptive_step) {
        st->eps_try = s_eps;  // kept if the attempt is accepted (step_decide)
      } else {
        st->eps = s_eps;
        st->k_total += 1;
        st->j += 1;
      }
    }
  }
}

// ------------------------------------- BB projected gradient (Section 4)
// With variable bounds lo <= x <= hi the primal subproblem
// min_{lo<=x<=hi} 1/2 x'(Q + I/tau)x - rhs'x is solved by the Barzilai-
// Borwein projected gradient from x^k.  The kernel that forms the CG start
// (k_atv, k_prepare) leaves r = p = -g0, the negated gradient at x^k, and
// g0'g0.  Phases:
//   [0] q = Q p: alpha0 = g0'M g0 / g0'g0 (M = Q + I/tau)
//   [A] x+ = min(max(x + r/alpha, lo), hi); s = x+ - x into p; x = x+; s's
//   [B] w = Q s + s/tau; r -= w (the gradient moves by w); qx += Q s; s'w
// then stop when ||s|| <= eps (adaptive, after at least one step), after
// cg_max steps, or after N steps (fixed), else alpha = s'w / s's.  One
// product with Q per step plus the first; the mixed path passes its
// displacement dx and the bounds shifted by the restart point.
template <int G, class T>
__global__ void __launch_bounds__(kCgBlock, kCgBlocksPerSm)
    k_bb(CsrT<T> Q, LongRows LQ, T* qseg, T* qlong, T* x, T* r, T* p, T* qx,
         const T* __restrict__ lo, const T* __restrict__ hi, const double* r0r0, double* part,
         DevState* st, GridBarrier* bar, int n, StepStart<T> sstart) {
  using A = typename Acc<T>::type;
  const bool active = running(st) && st->attempts < st->opt.max_iter;
  if (!active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iter_active = 0;
    return;
  }
  // Every read of st happens before the first barrier; block 0 writes the
  // counters only after the last one.  The FP64 scalars live in thread 0 of
  // each block, which shares 1/tau, 1/alpha and the flags through shared
  // memory (see grid_sync_sum).
  const int mode = st->opt.cg_mode, nfix = st->opt.cg_fixed_n, cgmax = st->opt.cg_max;
  const bool adaptive_step = st->opt.step_mode == kStepAdaptive;
  const int tmo = st->opt.barrier_timeout_ms;
  bool never_release = (st->opt.debug_flags & kDebugBarrierNeverReleases) != 0u;
  __shared__ double s_eps, s_rr, s_ss;  // thread 0's
  __shared__ T s_inv_tau, s_inv_alpha;
  __shared__ int s_flag;  // skip / numerical error / stop
  if (threadIdx.x == 0) {
    s_eps = mode == kCgAdaptive ? st->eps + st->opt.cg_eps_factor * st->relkkt_last : st->eps;
    s_rr = __ldcg(r0r0);
    s_inv_tau = T(1.0 / st->tau);
    s_flag = (mode == kCgFixed && nfix <= 0) || s_rr == 0.0;
  }
  __syncthreads();
  const T inv_tau = s_inv_tau;
  const bool skip = s_flag != 0;
  double* part_a = part;
  double* part_b = part + gridDim.x;
  const long long t0 = grid_tid(), nt = grid_threads();
  int steps = 0, products = 0;
  bool numerr = false, failed = false;
  unsigned int gen = grid_gen(bar);
  // Q p over every row (long rows first), f(i, (Q p)_i) for each row
  auto qprod = [&](auto&& f) {
    if (LQ.nlong > 0) {
      long_segments(Q, p, LQ, qseg);
      if (!grid_sync(bar, st, tmo, never_release, gen)) return false;
      never_release = false;
      long_finish(LQ, qseg, qlong);
      if (!grid_sync(bar, st, tmo, false, gen)) return false;
    }
    spmv_rows<G>(Q, p, [&](int i, T s, bool lead) {
      if (lead) f(i, s);
    });
    ++products;
    return true;
  };
  if (!skip) {
    {
      A acc;
      if (!qprod([&](int i, T s) {
            const T pi = p[i];
            acc.add_prod(pi, s + pi * inv_tau);
          }))
        return;
      block_dot_store(acc, part_a + blockIdx.x);
      if (!grid_sync_sum<A>(bar, st, tmo, never_release, gen, part_a, [&](const double* t) {
            const double gmg = t[0];
            s_flag = !(gmg > 0.0) || !isfinite(gmg);
            s_inv_alpha = inv_ratio<T>(gmg, s_rr);  // alpha = g'M g / g'g
          }))
        return;
      never_release = false;
      numerr = s_flag != 0;
    }
    while (!numerr && !failed) {
      const T inv_alpha = s_inv_alpha;
      A acc;
      for (long long i = t0; i < n; i += nt) {
        const T xi = x[i];
        const T xn = fmin(fmax(xi + r[i] * inv_alpha, lo[i]), hi[i]);
        const T si = xn - xi;
        p[i] = si;
        x[i] = xn;
        acc.add_prod(si, si);
      }
      block_dot_store(acc, part_a + blockIdx.x);
      if (!grid_sync_sum<A>(bar, st, tmo, false, gen, part_a, [&](const double* t) { s_ss = t[0]; }))
        return;
      A acc2;
      if (!qprod([&](int i, T s) {
            const T si = p[i];
            const T wi = s + si * inv_tau;
            r[i] = sub_rn(r[i], wi);
            qx[i] = add_rn(qx[i], s);
            acc2.add_prod(si, wi);
          }))
        return;
      block_dot_store(acc2, part_b + blockIdx.x);
      // flag: 0 continue, 1 stop, 2 numerical error
      if (!grid_sync_sum<A>(bar, st, tmo, false, gen, part_b, [&](const double* t) {
            const double sw = t[0];
            const int done_steps = steps + 1;
            const bool stop = mode == kCgFixed ? done_steps >= nfix
                                               : (scaled_norm_le<T>(1.0, s_ss, s_eps) ||
                                                  done_steps >= cgmax);
            if (stop || s_ss == 0.0) {
              s_flag = 1;
            } else if (!(sw > 0.0) || !isfinite(sw)) {
              s_flag = 2;
            } else {
              s_flag = 0;
              s_inv_alpha = inv_ratio<T>(sw, s_ss);  // alpha = s'w / s's
            }
          }))
        return;
      ++steps;
      if (s_flag == 1) break;
      if (s_flag == 2) {
        numerr = true;
        break;
      }
    }
  }
  if (sstart.part && !numerr) step_start_sums<T, A>(sstart, x, qx, n);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (numerr) {
      st->done = kDoneNumerical;
      st->iter_active = 0;
    } else {
      st->iter_active = 1;
      st->attempts += 1;
      st->cg_total += steps;
      st->last_cg = steps;
      st->spmv_total += products;
      if (adaptive_step) {
        st->eps_try = s_eps;
      } else {
        st->eps = s_eps;
        st->k_total += 1;
        st->j += 1;
      }
    }
  }
}

// Mixed path with variable bounds: the bounds of the displacement dx = x - x_a
// from the restart point, lo - x_a and hi - x_a, formed in FP64 from the FP64
// bounds and the compensated restart point, then rounded (+-inf stay).
__global__ void k_bound_shift(const double* __restrict__ lo, const double* __restrict__ hi,
                              const float* __restrict__ x_a, const float* __restrict__ x_a_lo,
                              float* lo_d, float* hi_d, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const double xa = (double)x_a[i] + (double)x_a_lo[i];
    lo_d[i] = float(lo[i] - xa);
    hi_d[i] = float(hi[i] - xa);
  }
}

// x <- min(max(x, lo), hi): a start point or a promoted iterate into the box.
template <class T>
__global__ void k_project_box(T* x, const T* __restrict__ lo, const T* __restrict__ hi, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) x[i] = fmin(fmax(x[i], lo[i]), hi[i]);
}

// ------------------------------------------- dual step (Algorithm 1, y-update)
// y+ = y + sigma (2 A x+ - A x - b), projected to >= 0 on rows >= m_eq; the
// A x cache and the running average of y are updated in the same pass.  The
// mixed path passes the displacement dx = x - x_a from the restart point x_a
// as x, b - A x_a as b and A dx as the cache: the same step, but every FP32
// quantity it gathers or subtracts is small near convergence.
//
// Adaptive step size (T.y_new != nullptr): the step is a trial.  y, its low
// word, the A x cache and the average stay as they are; the trial y+ (and its
// low word) and A x+ go to T.y_new, T.yn_lo, T.ax_new.  Each block stores the
// partial sums ||y+ - y||^2 and (y+ - y)'(A x+ - A x) at part_step[2 * block];
// the last block to finish combines them, and the x-step kernel's partials of
// ||x+ - x||^2 and (x+ - x)'(Q x+ - Q x) (StepStart: part_n, n_parts block
// partials, or the two totals when n_parts is 0),
// in a fixed order and takes the Section 4 step decision (step_decide).
// k_atv then commits or drops the trial.
template <class T>
struct StepTrial {
  T* y_new = nullptr;
  T* yn_lo = nullptr;
  T* ax_new = nullptr;
  double* part_step = nullptr;
  const double* part_n = nullptr;
  int n_parts = 0;
  const double* pow_table = nullptr;  // step_decide's (a+1)^-0.3, (a+1)^-0.6
  unsigned int* ticket = nullptr;
};

// The SpMV kernels hold 32 (FP32) or 40 (FP64) registers so that 8 or 6
// blocks of 256 threads stay resident per SM: their gathers need the warps.
// The FP64 dual step, with the adaptive step's four accumulators, gets 48.
template <class T>
constexpr int kSpmvBlocksPerSm = kSplit<T> ? 8 : 6;
template <class T>
constexpr int kDualBlocksPerSm = kSplit<T> ? 8 : 5;

template <int G, class T>
__global__ void __launch_bounds__(kBlock, kDualBlocksPerSm<T>)
    k_dual(CsrT<T> A, const T* __restrict__ x,
                                                 const T* __restrict__ b, T* y, T* y_lo, T* ax,
                                                 T* y_avg, T* ya_lo, DevState* st,
                                                 StepTrial<T> tr) {
  if (!st->iter_active) return;
  // FP64 scalars once per block (thread 0), not once per thread
  __shared__ T s_sigma, s_inv_j;
  if (threadIdx.x == 0) {
    s_sigma = T(st->sigma);
    s_inv_j = T(1.0 / (double)st->j);
  }
  __syncthreads();
  const T sigma = s_sigma;
  const T inv_j = s_inv_j;
  const bool first = st->j == 1;
  const int m_eq = st->opt.m_eq;
  if (tr.y_new) {
    typename Acc<T>::type am[2];
    spmv_rows<G>(A, x, [&](int i, T s, bool lead) {
      if (!lead) return;
      const T da = s - ax[i];
      T dy;
      if constexpr (kSplit<T>) {
        T hi = y[i], lo = y_lo[i];
        split_add(hi, lo, sigma * (T(2) * s - ax[i] - b[i]));
        if (i >= m_eq && hi < T(0)) hi = lo = T(0);
        dy = (hi - y[i]) + (lo - y_lo[i]);
        tr.y_new[i] = hi;
        tr.yn_lo[i] = lo;
      } else {
        T yn = y[i] + sigma * (T(2) * s - ax[i] - b[i]);
        if (i >= m_eq && yn < T(0)) yn = T(0);
        dy = yn - y[i];
        tr.y_new[i] = yn;
      }
      tr.ax_new[i] = s;
      am[0].add_prod(dy, dy);
      am[1].add_prod(dy, da);
    });
    block_pairs_store<2>(am, tr.part_step + 2 * size_t(blockIdx.x));
    __shared__ int s_last;
    if (threadIdx.x == 0) s_last = take_ticket(tr.ticket, gridDim.x);
    __syncthreads();
    if (s_last) {  // the whole last block (the branch is uniform)
      double t[2], u[2];
      block_pairs_total<2, typename Acc<T>::type>(tr.part_step, gridDim.x, t);
      if (tr.n_parts > 0) {  // per-block partials (the BB kernel)
        block_pairs_total<2, typename Acc<T>::type>(tr.part_n, tr.n_parts, u);
      } else {               // the CG kernel's totals
        u[0] = __ldcg(tr.part_n);
        u[1] = __ldcg(tr.part_n + 1);
      }
      if (threadIdx.x == 0) {
        if constexpr (kSplit<T>)  // FP32 arithmetic, as the values are applied in
          step_decide_f(st, float(u[0]), float(u[1]), float(t[0]), float(t[1]), tr.pow_table);
        else
          step_decide(st, u[0], u[1], t[0], t[1], tr.pow_table);
        *tr.ticket = 0u;  // for the next launch (ordered by the kernel boundary)
      }
    }
    return;
  }
  spmv_rows<G>(A, x, [&](int i, T s, bool lead) {
    if (lead) {
      if constexpr (kSplit<T>) {
        T hi = y[i], lo = y_lo[i];
        split_add(hi, lo, sigma * (T(2) * s - ax[i] - b[i]));
        if (i >= m_eq && hi < T(0)) hi = lo = T(0);
        y[i] = hi;
        y_lo[i] = lo;
        ax[i] = s;
        T ah = hi, al = lo;
        if (!first) {
          ah = y_avg[i];
          al = ya_lo[i];
          split_add(ah, al, ((hi - ah) + (lo - al)) * inv_j);
        }
        y_avg[i] = ah;
        ya_lo[i] = al;
      } else {
        T yn = y[i] + sigma * (T(2) * s - ax[i] - b[i]);
        if (i >= m_eq && yn < T(0)) yn = T(0);
        y[i] = yn;
        ax[i] = s;
        y_avg[i] += (yn - y_avg[i]) * inv_j;
      }
    }
  });
}

// Adaptive step size, after k_dual's decision: an accepted trial becomes y
// (with its low word) and the A x cache, and enters the running average of y
// with the step weight; a rejected one is dropped.  Run by the last `blocks`
// blocks of the k_atv launch (block b of them: index b).
template <class T>
struct Commit {
  T* y = nullptr;
  T* y_lo = nullptr;
  const T* y_new = nullptr;
  const T* yn_lo = nullptr;
  T* ax = nullptr;
  const T* ax_new = nullptr;
  T* y_avg = nullptr;
  T* ya_lo = nullptr;
  int m = 0;
  int blocks = 0;  // 0: no commit (fixed step)
};

template <class T>
__device__ __forceinline__ void commit_m(const Commit<T>& cm, const DevState* st, int b) {
  if (!st->accepted) return;
  __shared__ T s_w;  // the step weight, converted once per block
  if (threadIdx.x == 0) s_w = T(st->avg_w);
  __syncthreads();
  const T w = s_w;
  const bool first = st->j == 1;
  const long long nt = (long long)cm.blocks * blockDim.x;
  for (long long i = (long long)b * blockDim.x + threadIdx.x; i < cm.m; i += nt) {
    cm.ax[i] = cm.ax_new[i];
    if constexpr (kSplit<T>) {
      const T hi = cm.y_new[i], lo = cm.yn_lo[i];
      cm.y[i] = hi;
      cm.y_lo[i] = lo;
      T ah = hi, al = lo;
      if (!first) {
        ah = cm.y_avg[i];
        al = cm.ya_lo[i];
        split_add(ah, al, ((hi - ah) + (lo - al)) * w);
      }
      cm.y_avg[i] = ah;
      cm.ya_lo[i] = al;
    } else {
      const T yn = cm.y_new[i];
      cm.y[i] = yn;
      cm.y_avg[i] += (yn - cm.y_avg[i]) * w;
    }
  }
}

// A' y+ over the explicit transpose, fused with the running average of x and
// with the next CG's start: r0 = p0 = -(qx + c + A'y+) and r0'r0 partials.
// (The mixed path averages the displacement dx, see k_dual.)
//
// Adaptive step size (x_save != nullptr), after k_dual's decision: after an
// accepted step the product reads the trial y+ (y_trial), the average takes
// the step weight and (x, Q x) are saved as the start of the next attempt,
// while the launch's last cm.blocks blocks commit the trial into y, A x and
// the average of y (neither side reads what the other writes); after a
// rejected one x and Q x go back to the saved start and the CG start is
// formed from the unchanged A'y, with no product.
template <int G, class T>
__global__ void __launch_bounds__(kBlock, kSpmvBlocksPerSm<T>)
    k_atv(CsrT<T> At, const T* __restrict__ y, T* aty, T* x, T* x_avg, T* qx,
          const T* __restrict__ c, T* r, T* p, double* part_r0, unsigned int* ticket,
          const DevState* st, T* x_save, T* qx_save, const T* __restrict__ y_trial,
          Commit<T> cm, double* part_chunk, unsigned int* chunk_ctr) {
  if (!st->iter_active) return;
  const int nb = int(gridDim.x) - cm.blocks;  // the product's blocks
  if (int(blockIdx.x) >= nb) {
    commit_m(cm, st, int(blockIdx.x) - nb);
    return;
  }
  const bool adaptive = x_save != nullptr;
  typename Acc<T>::type acc;
  if (adaptive && !st->accepted) {
    const long long nt = (long long)nb * blockDim.x;
    for (long long i = grid_tid(); i < At.rows; i += nt) {
      const T xs = x_save[i], qs = qx_save[i];
      x[i] = xs;
      qx[i] = qs;
      const T ri = -(qs + c[i] + aty[i]);
      r[i] = ri;
      p[i] = ri;
      acc.add_prod(ri, ri);
    }
    store_and_finish_dot(acc, part_r0, ticket, nb);
    return;
  }
  __shared__ T s_w;  // the average's weight, once per block
  if (threadIdx.x == 0) s_w = adaptive ? T(st->avg_w) : T(1.0 / (double)st->j);
  __syncthreads();
  const T w = s_w;
  const T* yv = adaptive && y_trial != nullptr ? y_trial : y;
  auto row = [&](int i, T s, bool lead) {
    if (lead) {
      aty[i] = s;
      const T xi = x[i], qxi = qx[i];
      x_avg[i] += (xi - x_avg[i]) * w;
      const T ri = -(qxi + c[i] + s);
      r[i] = ri;
      p[i] = ri;
      acc.add_prod(ri, ri);
      if (adaptive) {
        x_save[i] = xi;
        qx_save[i] = qxi;
      }
    }
  };
  if constexpr ((G & kMedRows) != 0) {
    // rows of very uneven lengths (A' of a power-law A): chunks would make
    // the warps of a block wait for each other at every chunk (measured
    // slower), so the fixed shares of spmv_rows
    spmv_rows<G>(At, yv, row, nb);
    store_and_finish_dot(acc, part_r0, ticket, nb);
    return;
  }
  // short and long rows in chunks, r0'r0 partial per chunk; the last block
  // adds the chunks' partials in chunk order, then the blocks' (zero here)
  spmv_rows_chunked<G>(At, yv, chunk_ctr, row, [&](int ch) {
    block_dot_store(acc, part_chunk + ch);
    acc = typename Acc<T>::type();
  });
  __shared__ int s_last;
  block_dot_store(acc, part_r0 + blockIdx.x);
  if (threadIdx.x == 0) s_last = take_ticket(ticket, unsigned(nb));
  __syncthreads();
  if (s_last) {  // the whole last block (the branch is uniform)
    const int nchunks = (At.rows + kChunkRows - 1) / kChunkRows;
    using A = typename Acc<T>::type;
    const double t_chunks = block_total_dot<8>(part_chunk, nchunks, A());
    const double t_blocks = block_total_dot<8>(part_r0, nb, A());
    if (threadIdx.x == 0) {
      part_r0[nb] = t_chunks + t_blocks;
      *ticket = 0u;     // for the next launch (ordered by the kernel boundary)
      *chunk_ctr = 0u;
    }
  }
}

// r0 = p0 = -(qx + c + A'y) and r0'r0 partials, for the first CG after a
// set-up, an evaluation or a restart.  Launched with the grid of k_atv.
// With the adaptive step size (x_save != nullptr) it also saves (x, Q x) as
// the start of the next attempt.
template <class T>
__global__ void __launch_bounds__(kBlock) k_prepare(const T* __restrict__ qx,
                                                    const T* __restrict__ c,
                                                    const T* __restrict__ aty, T* r, T* p, int n,
                                                    double* part_r0, unsigned int* ticket,
                                                    const T* __restrict__ x, T* x_save,
                                                    T* qx_save) {
  typename Acc<T>::type acc;
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const T qxi = qx[i];
    const T ri = -(qxi + c[i] + aty[i]);
    r[i] = ri;
    p[i] = ri;
    acc.add_prod(ri, ri);
    if (x_save) {
      x_save[i] = x[i];
      qx_save[i] = qxi;
    }
  }
  store_and_finish_dot(acc, part_r0, ticket);
}

// Plain out = M v, optionally with per-block partial sums of out_i^2 (double).
template <int G, class T>
__global__ void __launch_bounds__(kBlock) k_spmv(CsrT<T> M, const T* __restrict__ v, T* out,
                                                 double* part_sq, unsigned int* ticket,
                                                 const double* inv_norm_sq) {
  // out = M v / ||v||_2 when inv_norm_sq points at ||v||_2^2 (the power
  // iteration's normalisation, applied to the product instead of to v)
  __shared__ T s_scale;  // 1/||v||_2, formed once per block (FP64 sqrt and division)
  if (threadIdx.x == 0) {
    const double l2 = inv_norm_sq ? __ldcg(inv_norm_sq) : 1.0;
    s_scale = l2 > 0.0 ? T(1.0 / sqrt(l2)) : T(0);
  }
  __syncthreads();
  const T scale = s_scale;
  typename Acc<T>::type acc;
  spmv_rows<G>(M, v, [&](int i, T s, bool lead) {
    if (lead) {
      const T o = s * scale;
      out[i] = o;
      acc.add_prod(o, o);
    }
  });
  // ||out||^2: block partials, and the total (part_sq[gridDim.x]) from the
  // last block to finish
  if (part_sq) store_and_finish_dot(acc, part_sq, ticket);
}

// ------------------------------------------------ relKKT terms (Section 4)
// Per block (stride kPartStride), over the n index space, from the products
// qx = Q x, qxa = Q x~ and A'y, A'y~ computed just before:
//  [0] max|Qx + A'y + c - lambda|  [1] max|Qx|  [2] max|A'y|  [3] sum x.Qx  [4] sum c.x
//  [5..9] the same for the average (x~, y~)            [10] max|c|
//  [11] lb of (x, y)  [12] lb of (x~, y~)
// With variable bounds (lo != nullptr; +-inf allowed) lambda are the reduced
// costs of g = Qx + A'y + c: g where both bounds are finite, max(g, 0) with
// only a lower one, min(g, 0) with only an upper one, 0 with none; and
// lb = lo'lambda^+ - hi'lambda^- over the finite bounds.  Without bounds
// lambda = 0 and lb = 0.
// With diagonal scaling (inv_d2 != nullptr) the iterate is the scaled x~ and
// the infinity norms are of the original quantities: row j of Qx, A'y, c and
// Qx + A'y + c is inv_d2[j] times the scaled one; the dot products, the
// reduced costs' signs and lb are invariant under the scaling.
template <class T>
__global__ void __launch_bounds__(kBlock) k_kkt_n(const T* __restrict__ x,
                                                  const T* __restrict__ x_avg,
                                                  const T* __restrict__ qx,
                                                  const T* __restrict__ qxa,
                                                  const T* __restrict__ aty,
                                                  const T* __restrict__ aty_avg,
                                                  const T* __restrict__ c,
                                                  const T* __restrict__ inv_d2,
                                                  const T* __restrict__ lo,
                                                  const T* __restrict__ hi, int n,
                                                  double* part) {
  using A = typename Acc<T>::type;
  T mx[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};  // maxima, see the map below
  A sm[6];  // x.Qx, c.x, x~.Qx~, c.x~, lb, lb~
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const T ci = c[i], q1 = qx[i], q2 = qxa[i];
    const T w = inv_d2 ? inv_d2[i] : T(1);
    const T g1 = q1 + aty[i] + ci, g2 = q2 + aty_avg[i] + ci;
    T l1 = T(0), l2 = T(0);
    if (lo) {
      const T li = lo[i], hi_ = hi[i];
      l1 = reduced_cost(g1, li, hi_);
      l2 = reduced_cost(g2, li, hi_);
      sm[4].add_prod(T(1), bound_term(l1, li, hi_));
      sm[5].add_prod(T(1), bound_term(l2, li, hi_));
    }
    mx[0] = fmax(mx[0], w * fabs(g1 - l1));
    mx[1] = fmax(mx[1], w * fabs(q1));
    mx[2] = fmax(mx[2], w * fabs(aty[i]));
    sm[0].add_prod(x[i], q1);
    sm[1].add_prod(ci, x[i]);
    mx[3] = fmax(mx[3], w * fabs(g2 - l2));
    mx[4] = fmax(mx[4], w * fabs(q2));
    mx[5] = fmax(mx[5], w * fabs(aty_avg[i]));
    sm[2].add_prod(x_avg[i], q2);
    sm[3].add_prod(ci, x_avg[i]);
    mx[6] = fmax(mx[6], w * fabs(ci));
  }
  // fmax drops NaN; a NaN iterate still reaches relKKT through the dot products.
  __shared__ double out[13];
  block_reduce_ms<7, 6>(mx, sm, out);
  if (threadIdx.x == 0) {
    double* o = part + size_t(blockIdx.x) * kPartStride;
    // maxima at 0,1,2,5,6,7,10 and sums at 3,4,8,9,11,12 (kKktNMaxMask)
    o[0] = out[0];
    o[1] = out[1];
    o[2] = out[2];
    o[3] = out[7];
    o[4] = out[8];
    o[5] = out[3];
    o[6] = out[4];
    o[7] = out[5];
    o[8] = out[9];
    o[9] = out[10];
    o[10] = out[6];
    o[11] = out[11];
    o[12] = out[12];
  }
}

// Over the m index space, from ax = A x (cached) and ax_avg = A x~:
//  [0] max viol(x)  [1] max|Ax|  [2] sum b.y  [3] max viol(x~)  [4] max|Ax~|
//  [5] sum b.y~  [6] max|b|;  viol = |Ax-b| on equality rows, [Ax-b]^+ else.
// With diagonal scaling (inv_d1 != nullptr) row i of Ax - b, Ax and b is
// inv_d1[i] times the scaled one.
template <class T>
__global__ void __launch_bounds__(kBlock) k_kkt_m(const T* __restrict__ ax,
                                                  const T* __restrict__ ax_avg,
                                                  const T* __restrict__ b,
                                                  const T* __restrict__ y,
                                                  const T* __restrict__ y_avg,
                                                  const T* __restrict__ inv_d1, int m, int m_eq,
                                                  double* part) {
  using A = typename Acc<T>::type;
  T mx[5] = {T(0), T(0), T(0), T(0), T(0)};  // viol, |Ax|, viol~, |Ax~|, |b|
  A sm[2];                                   // b.y, b.y~
  for (long long i = grid_tid(); i < m; i += grid_threads()) {
    const T bi = b[i], s = ax_avg[i];
    const T w = inv_d1 ? inv_d1[i] : T(1);
    const T d = ax[i] - bi, da = s - bi;
    const T vc = i < m_eq ? fabs(d) : (d > T(0) ? d : T(0));
    const T va = i < m_eq ? fabs(da) : (da > T(0) ? da : T(0));
    mx[0] = fmax(mx[0], w * vc);
    mx[1] = fmax(mx[1], w * fabs(ax[i]));
    sm[0].add_prod(bi, y[i]);
    mx[2] = fmax(mx[2], w * va);
    mx[3] = fmax(mx[3], w * fabs(s));
    sm[1].add_prod(bi, y_avg[i]);
    mx[4] = fmax(mx[4], w * fabs(bi));
  }
  __shared__ double out[7];
  block_reduce_ms<5, 2>(mx, sm, out);
  if (threadIdx.x == 0) {
    double* o = part + size_t(blockIdx.x) * kPartStride;
    o[0] = out[0];
    o[1] = out[1];
    o[2] = out[5];
    o[3] = out[2];
    o[4] = out[3];
    o[5] = out[6];
    o[6] = out[4];
  }
}



// One block: reduce the relKKT partials, then control_decide.
__global__ void __launch_bounds__(kBlock) k_control(const double* part_n, int gn,
                                                    const double* part_m, int gm, DevState* st,
                                                    int mode) {
  double rn[13], rm[7];
  block_reduce_rows<13>(part_n, gn, kPartStride, kKktNMaxMask, rn);
  block_reduce_rows<7>(part_m, gm, kPartStride, kKktMMaxMask, rm);
  if (threadIdx.x != 0) return;
  const KktTerms kc =
      kkt_from(rm[0], rm[1], rm[6], rn[0], rn[1], rn[2], rn[10], rn[3], rn[4], rm[2], rn[11]);
  const KktTerms ka =
      kkt_from(rm[3], rm[4], rm[6], rn[5], rn[6], rn[7], rn[10], rn[8], rn[9], rm[5], rn[12]);
  control_decide(st, kc, ka, mode);
}

// Restart to the candidate (Algorithm 1, restart step), n side: distance to
// the previous restart point for the primal weight, then anchor = x = cand.
template <class T>
__global__ void __launch_bounds__(kBlock) k_restart_n(T* x, const T* __restrict__ x_avg,
                                                      T* x_anchor, T* aty,
                                                      const T* __restrict__ aty_avg, T* qx,
                                                      const T* __restrict__ qx_avg,
                                                      const DevState* st, int n, double* part) {
  const int pending = st->restart_pending;
  if (pending == 0) return;
  typename Acc<T>::type acc;
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const T cand = pending == 2 ? x_avg[i] : x[i];
    const T d = cand - x_anchor[i];
    acc.add_prod(d, d);
    x_anchor[i] = cand;
    x[i] = cand;
    if (pending == 2) {
      aty[i] = aty_avg[i];
      qx[i] = qx_avg[i];
    }
  }
  block_sum_store(acc, part + blockIdx.x);
}

// Mixed path, n side: the candidate is the restart point plus dx (or plus the
// average of dx), so its distance to the restart point is that displacement;
// the restart point (x_a, x_a_lo) moves by it and dx and its average restart
// from zero.
__global__ void __launch_bounds__(kBlock) k_restart_n_delta(float* x_a, float* x_a_lo, float* dx,
                                                            float* dx_avg, float* aty,
                                                            const float* __restrict__ aty_avg,
                                                            float* qx,
                                                            const float* __restrict__ qx_avg,
                                                            const DevState* st, int n,
                                                            double* part) {
  const int pending = st->restart_pending;
  if (pending == 0) return;
  AccF acc;
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const float d = pending == 2 ? dx_avg[i] : dx[i];
    acc.add_prod(d, d);
    float hi = x_a[i], lo = x_a_lo[i];
    split_add(hi, lo, d);
    x_a[i] = hi;
    x_a_lo[i] = lo;
    dx[i] = 0.f;
    dx_avg[i] = 0.f;
    if (pending == 2) {
      aty[i] = aty_avg[i];
      qx[i] = qx_avg[i];
    }
  }
  block_sum_store(acc, part + blockIdx.x);
}

// The mixed path passes A dx as ax and also b - A x_a (b_shift) with b: the
// new restart point x_a' = x_a + dx (or + the average of dx, whose product
// A x~ is ax_avg) gives b - A x_a' and A dx' = 0.
template <class T>
__global__ void __launch_bounds__(kBlock) k_restart_m(T* y, T* y_lo, const T* __restrict__ y_avg,
                                                      const T* __restrict__ ya_lo,
                                                      T* y_anchor, T* ax,
                                                      const T* __restrict__ ax_avg, T* b_shift,
                                                      const T* __restrict__ b,
                                                      const DevState* st, int m, double* part) {
  const int pending = st->restart_pending;
  if (pending == 0) return;
  typename Acc<T>::type acc;
  for (long long i = grid_tid(); i < m; i += grid_threads()) {
    const T cand = pending == 2 ? y_avg[i] : y[i];
    const T d = cand - y_anchor[i];
    acc.add_prod(d, d);
    y_anchor[i] = cand;
    y[i] = cand;
    if constexpr (kSplit<T>) {
      if (pending == 2) {
        y_lo[i] = ya_lo[i];
        b_shift[i] = b[i] - ax_avg[i];
      } else {
        b_shift[i] -= ax[i];
      }
      ax[i] = T(0);
    } else {
      if (pending == 2) ax[i] = ax_avg[i];
    }
  }
  block_sum_store(acc, part + blockIdx.x);
}


__global__ void __launch_bounds__(kBlock) k_restart_finish(const double* part_n, int gn,
                                                           const double* part_m, int gm,
                                                           DevState* st) {
  if (st->restart_pending == 0) return;
  double dx2[1], dy2[1];
  block_reduce_rows<1>(part_n, gn, 1, 0u, dx2);
  block_reduce_rows<1>(part_m, gm, 1, 0u, dy2);
  if (threadIdx.x != 0) return;
  restart_finish_decide(st, dx2[0], dy2[0]);
}

// ---------------------------------------------------------- set-up kernels
// Start of a solve: cold start zeros everything; warm start copies (x0, y0).
// The mixed path's extra words (null for FP64) start at zero: the low word
// of the restart point, the displacement dx and its average, and the low
// words of y and of its average.
template <class T>
__global__ void k_init_vectors(T* x, T* x_avg, T* x_anchor, const T* __restrict__ x0, int n, T* y,
                               T* y_avg, T* y_anchor, const T* __restrict__ y0, int m, T* x_a_lo,
                               T* dx, T* dx_avg, T* y_lo, T* ya_lo) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const T v = x0 ? x0[i] : T(0);
    x[i] = v;
    x_anchor[i] = v;
    x_avg[i] = T(0);
    if (x_a_lo) {
      x_a_lo[i] = T(0);
      dx[i] = T(0);
      dx_avg[i] = T(0);
    }
  }
  for (long long i = grid_tid(); i < m; i += grid_threads()) {
    const T v = y0 ? y0[i] : T(0);
    y[i] = v;
    y_anchor[i] = v;
    y_avg[i] = T(0);
    if (y_lo) {
      y_lo[i] = T(0);
      ya_lo[i] = T(0);
    }
  }
}

// v = 1/sqrt(n) (power-iteration start) and per-block partials of ||c||^2, ||b||^2.
template <class T>
__global__ void k_pow_start(T* v, int n, const T* __restrict__ c, const T* __restrict__ b, int m,
                            double* part2) {
  __shared__ T s_v0;  // 1/sqrt(n), once per block
  if (threadIdx.x == 0) s_v0 = T(1.0 / sqrt((double)n));
  __syncthreads();
  const T v0 = s_v0;
  typename Acc<T>::type a[2];
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    v[i] = v0;
    a[0].add_prod(c[i], c[i]);
  }
  for (long long i = grid_tid(); i < m; i += grid_threads()) a[1].add_prod(b[i], b[i]);
  block_reduce_ms<0, 2, T>(nullptr, a, part2 + size_t(blockIdx.x) * 2);
}

// step_decide's table: t[2 a] = (a+1)^-0.3, t[2 a + 1] = (a+1)^-0.6.
__global__ void k_step_pow(double* t, int count) {
  for (long long a = grid_tid(); a < count; a += grid_threads()) step_pow_entry(t, a);
}

// Element-wise type conversion (FP64 <-> FP32 copies of a vector).
template <class Ti, class To>
__global__ void k_convert(const Ti* __restrict__ in, To* out, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) out[i] = To(in[i]);
}

// Conversion of a vector that may carry a compensation word on either side:
// v = in + in_lo (in_lo may be null), out = round(v), out_lo = the rounding
// error of out when out_lo is not null.
template <class Ti, class To>
__global__ void k_convert_split(const Ti* __restrict__ in, const Ti* __restrict__ in_lo, To* out,
                                To* out_lo, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const double v = in_lo ? (double)in[i] + (double)in_lo[i] : (double)in[i];
    const To o = To(v);
    out[i] = o;
    if (out_lo) out_lo[i] = To(v - (double)o);
  }
}

// Mixed-path x in FP64: out = x_a + x_a_lo + d (d may be null).
__global__ void k_delta_join(const float* __restrict__ x_a, const float* __restrict__ x_a_lo,
                             const float* __restrict__ d, double* out, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads())
    out[i] = ((double)x_a[i] + (double)x_a_lo[i]) + (d ? (double)d[i] : 0.0);
}

// Displacement of an FP64 iterate from the FP64 restart point, in FP32.
__global__ void k_delta_split(const double* __restrict__ v, const double* __restrict__ v_a,
                              float* d, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) d[i] = float(v[i] - v_a[i]);
}

// Mixed path, before an evaluation or a cache refresh: the full x~ = x_a + dx
// and its average (rounded to FP32) for the products and relKKT terms, and,
// when b is given, A x~ = (b - b_shift) + A dx.
__global__ void k_materialize(const float* __restrict__ x_a, const float* __restrict__ x_a_lo,
                              const float* __restrict__ dx, const float* __restrict__ dx_avg,
                              float* x, float* x_avg, int n, const float* __restrict__ b,
                              const float* __restrict__ b_shift, const float* __restrict__ ax_d,
                              float* ax, int m) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const double a = (double)x_a[i] + (double)x_a_lo[i];
    x[i] = float(a + (double)dx[i]);
    x_avg[i] = float(a + (double)dx_avg[i]);
  }
  if (b)
    for (long long i = grid_tid(); i < m; i += grid_threads()) ax[i] = (b[i] - b_shift[i]) + ax_d[i];
}

// b_shift = b - A x_a with A x_a already in ax (cache refresh of the mixed path).
__global__ void k_shift_rhs(const float* __restrict__ b, const float* __restrict__ ax,
                            float* b_shift, int m) {
  for (long long i = grid_tid(); i < m; i += grid_threads()) b_shift[i] = b[i] - ax[i];
}


__global__ void __launch_bounds__(kBlock) k_setup_finish(const double* part2, int g2,
                                                         const double* w_norm_sq, DevState* st,
                                                         int reset) {
  double s[2];
  block_reduce_rows<2>(part2, g2, 2, 0u, s);
  if (threadIdx.x != 0) return;
  st->lam = sqrt(__ldcg(w_norm_sq));  // ||A'A v|| of the last power step
  setup_finish_decide(st, s[0], s[1], reset);
}

}  // namespace pdhcg
