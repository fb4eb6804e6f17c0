// Device side of the B300 restarted-PDHCG solver (arXiv 2405.16160).
//
// One PDHCG iteration (Algorithm 1 loop body) is three launches:
//   k_cg    cooperative, persistent: the whole inexact CG solve of
//           (Q + I/tau) x = x/tau - c - A'y (Section 2), grid barriers between
//           the SpMV and the vector phases, deterministic FP64 reductions;
//   k_dual  A x+ fused with the projected dual step, the A x cache and the
//           running average of y (Algorithm 1, y-update and averages);
//   k_atv   A' y+ (explicit transpose) fused with the running average of x.
// Every eval_freq iterations: k_spmv (A' y~), k_kkt_n, k_kkt_m (relKKT terms
// of Section 4 for the current iterate and the average), k_control (one warp:
// termination and the restart tests), k_restart_n / k_restart_m /
// k_restart_finish (restart to the candidate and the primal-weight update).
//
// Reductions never use floating-point atomics: each block writes partials,
// and every consumer reduces them in one fixed order, so results do not
// depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <math_constants.h>
#include <stdint.h>

namespace pdhcg {

constexpr int kBlock = 256;
constexpr int kCgBlock = 512;  // persistent CG kernel: fewer, larger blocks
constexpr int kPartStride = 16;  // doubles per block in the multi-value partial buffers
constexpr int kCgAdaptive = 0;
constexpr int kCgFixed = 1;
constexpr int kRestartAdaptive = 0;

// done codes: 0 running, otherwise 1 + qp_termination
constexpr int kDoneSolved = 1;
constexpr int kDoneIterLimit = 2;
constexpr int kDoneNumerical = 4;

constexpr int kErrBarrierTimeout = 1;
constexpr unsigned kDebugBarrierNeverReleases = 1u;

// Which entries of the relKKT partial buffers are maxima (bit set) or sums.
constexpr unsigned kKktNMaxMask = 0b10011100111u;  // 11 entries, see k_kkt_n
constexpr unsigned kKktMMaxMask = 0b1011011u;      // 7 entries, see k_kkt_m

struct DevCsr {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  int32_t rows;
};

struct DevOptions {
  double tol;
  long long max_iter;
  int cg_mode, cg_fixed_n, cg_max, restart_mode;
  double cg_eps_factor, beta_suff, beta_nec, beta_art, theta_pw, eps_zero;
  double omega0, eta_override;
  int pw_update, m_eq;
  unsigned debug_flags;
  int barrier_timeout_ms;
};

struct DevState {
  DevOptions opt;
  double eta, omega, tau, sigma;
  double eps;            // adaptive CG precision eps_k
  double relkkt_last;    // latest evaluated relKKT of the current iterate
  double kkt_anchor;     // relKKT of the epoch's restart point
  double kkt_prev_cand;  // candidate relKKT at the previous evaluation
  double kkt_cand;       // candidate relKKT of a pending restart
  double norm_A, lam;
  double kkt_cur[6], kkt_avg[6];  // r_primal, r_dual, r_gap, relKKT, pobj, dobj
  double kkt_ret[6];              // terms of the iterate a stop now would return
  long long j, k_total, n_restarts, cg_total, last_cg, n_evals, spmv_total;
  int done, returned_avg, iter_active, restart_pending, last_restart, err;
};

struct alignas(128) GridBarrier {
  unsigned int count;
  unsigned int pad0[31];
  unsigned int gen;
  unsigned int pad1[31];
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool running(const DevState* st) { return st->done == 0 && st->err == 0; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of K per-thread values; bit k of max_mask selects max
// (of non-negative values) instead of sum.  Thread 0 writes out[0..K).
template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], unsigned max_mask, double* out) {
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double x = ((max_mask >> k) & 1u) ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < nwarps ? sh[k][lane] : 0.0;
      x = ((max_mask >> k) & 1u) ? warp_max(x) : warp_sum(x);
      if (lane == 0) out[k] = x;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void block_sum_store(double v, double* out) {
  double a[1] = {v};
  block_reduce_store<1>(a, 0u, out);
}

// Fixed-order reduction of n block partials (stride apart) by one warp; every
// lane returns the same value, and so does every block that calls it.
__device__ __forceinline__ double warp_reduce_partials(const double* p, int n, int stride,
                                                       bool is_max) {
  const int lane = threadIdx.x & 31;
  double x = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double v = __ldcg(p + size_t(i) * stride);
    x = is_max ? fmax(x, v) : x + v;
  }
  return is_max ? warp_max(x) : warp_sum(x);
}

// The same value broadcast to every thread of the block.
__device__ __forceinline__ double block_all_reduce_partials(const double* p, int n) {
  __shared__ double s_val;
  if (threadIdx.x < 32) {
    const double v = warp_reduce_partials(p, n, 1, false);
    if (threadIdx.x == 0) s_val = v;
  }
  __syncthreads();
  const double v = s_val;
  __syncthreads();
  return v;
}

// Sense-free generation barrier over all blocks of a co-resident grid.  Every
// wait is bounded: after opt.barrier_timeout_ms (globaltimer) or 2^27 polls the
// block records kErrBarrierTimeout and the kernel winds down; a block that
// sees the error flag stops waiting too.  Returns false on error.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, DevState* st, int timeout_ms,
                                          bool never_release) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(bar->gen);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar->count);
    cuda::atomic_ref<int, cuda::thread_scope_device> err(st->err);
    int ok = 1;
    const unsigned int g = gen.load(cuda::memory_order_acquire);
    __threadfence();
    const unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    if (arrived == gridDim.x - 1 && !never_release) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.fetch_add(1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = global_ns();
      const unsigned long long limit = (unsigned long long)timeout_ms * 1000000ull;
      unsigned int polls = 0;
      while (gen.load(cuda::memory_order_acquire) == g) {
        if (err.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
        if ((++polls & 255u) == 0u) {
          if (global_ns() - t0 > limit || polls > (1u << 27)) {
            err.fetch_or(kErrBarrierTimeout, cuda::memory_order_relaxed);
            ok = 0;
            break;
          }
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Row-group CSR SpMV: G lanes share a row (G in {1,2,4,8,16,32}), all 32 lanes
// of a warp walk the same number of row blocks so the group shuffles never
// diverge.  Each lane accumulates its strided share of the row in FP64 and
// the group reduces with xor shuffles, so a row's sum does not depend on the
// launch configuration.  f(i, sum, leader) is called by every lane of the
// group; `leader` is lane 0 of the group.
template <int G, class F>
__device__ __forceinline__ void spmv_rows(const DevCsr& M, const double* v, F&& f) {
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = gw * kRowsPerWarp; base < M.rows; base += nw * kRowsPerWarp) {
    const int i = int(base) + lane / G;
    double s = 0.0;
    if (i < M.rows) {
      const int e = __ldg(M.rowptr + i + 1);
      for (int k = __ldg(M.rowptr + i) + sub; k < e; k += G)
        s = fma(__ldg(M.val + k), v[__ldg(M.col + k)], s);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i < M.rows) f(i, s, sub == 0);
  }
}

// Same walk, two vectors through one pass over the matrix row.
template <int G, class F>
__device__ __forceinline__ void spmv2_rows(const DevCsr& M, const double* v1, const double* v2,
                                           F&& f) {
  constexpr int kRowsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = gw * kRowsPerWarp; base < M.rows; base += nw * kRowsPerWarp) {
    const int i = int(base) + lane / G;
    double s1 = 0.0, s2 = 0.0;
    if (i < M.rows) {
      const int e = __ldg(M.rowptr + i + 1);
      for (int k = __ldg(M.rowptr + i) + sub; k < e; k += G) {
        const double a = __ldg(M.val + k);
        const int cj = __ldg(M.col + k);
        s1 = fma(a, v1[cj], s1);
        s2 = fma(a, v2[cj], s2);
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (i < M.rows) f(i, s1, s2, sub == 0);
  }
}

__device__ __forceinline__ long long grid_tid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long grid_threads() { return (long long)gridDim.x * blockDim.x; }

// ------------------------------------------------------------- CG (Section 2)
// Inexact CG on (Q + I/tau) x = x^k/tau - c - A'y^k warm-started at x^k.  The
// initial residual simplifies to r0 = -(Q x^k + c + A'y^k).  Phases per CG
// step: [A] q = Qp + p/tau, p'q  | [B] x += a p, r -= a q, r'r  | [C] p = r + b p.
// part holds 2 * gridDim.x doubles.
template <int G>
__global__ void __launch_bounds__(kCgBlock, 3) k_cg(DevCsr Q, const double* __restrict__ c,
                                               const double* __restrict__ aty, double* x,
                                               double* r, double* p, double* q, double* part,
                                               DevState* st, GridBarrier* bar, int n) {
  const bool active = running(st) && st->k_total < st->opt.max_iter;
  if (!active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iter_active = 0;
    return;
  }
  // Every read of st happens before the first barrier; block 0 writes the
  // counters only after the last one.
  const double tau = st->tau;
  const double inv_tau = 1.0 / tau;
  const int mode = st->opt.cg_mode, nfix = st->opt.cg_fixed_n, cgmax = st->opt.cg_max;
  const int tmo = st->opt.barrier_timeout_ms;
  const bool never_release = (st->opt.debug_flags & kDebugBarrierNeverReleases) != 0u;
  const double eps =
      mode == kCgAdaptive ? st->eps + st->opt.cg_eps_factor * st->relkkt_last : st->eps;
  double* part_rr = part;
  double* part_pq = part + gridDim.x;
  const long long t0 = grid_tid(), nt = grid_threads();

  double acc = 0.0;
  spmv_rows<G>(Q, x, [&](int i, double s, bool lead) {
    if (lead) {
      const double ri = -(s + c[i] + aty[i]);
      r[i] = ri;
      p[i] = ri;
      acc = fma(ri, ri, acc);
    }
  });
  block_sum_store(acc, part_rr + blockIdx.x);
  if (!grid_sync(bar, st, tmo, never_release)) return;
  double rr = block_all_reduce_partials(part_rr, gridDim.x);

  int steps = 0;
  bool numerr = false;
  const bool skip = (mode == kCgFixed && nfix <= 0) || rr == 0.0;
  while (!skip) {
    acc = 0.0;
    spmv_rows<G>(Q, p, [&](int i, double s, bool lead) {
      if (lead) {
        const double pi = p[i];
        const double qi = s + pi * inv_tau;
        q[i] = qi;
        acc = fma(pi, qi, acc);
      }
    });
    block_sum_store(acc, part_pq + blockIdx.x);
    if (!grid_sync(bar, st, tmo, false)) return;
    const double pq = block_all_reduce_partials(part_pq, gridDim.x);
    if (!(pq > 0.0) || !isfinite(pq)) {
      numerr = true;
      break;
    }
    const double alpha = rr / pq;
    acc = 0.0;
    // x += alpha p, r -= alpha q with a rounded product then a rounded sum,
    // exactly as the elementwise vector statements of textbook CG.
    for (long long i = t0; i < n; i += nt) {
      x[i] = __dadd_rn(x[i], __dmul_rn(alpha, p[i]));
      const double ri = __dsub_rn(r[i], __dmul_rn(alpha, q[i]));
      r[i] = ri;
      acc = fma(ri, ri, acc);
    }
    block_sum_store(acc, part_rr + blockIdx.x);
    if (!grid_sync(bar, st, tmo, false)) return;
    const double rr_new = block_all_reduce_partials(part_rr, gridDim.x);
    ++steps;
    const bool stop = mode == kCgFixed ? steps >= nfix : (tau * sqrt(rr_new) <= eps || steps >= cgmax);
    if (stop || rr_new == 0.0) break;
    const double beta = rr_new / rr;
    rr = rr_new;
    for (long long i = t0; i < n; i += nt) p[i] = __dadd_rn(r[i], __dmul_rn(beta, p[i]));
    if (!grid_sync(bar, st, tmo, false)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (numerr) {
      st->done = kDoneNumerical;
      st->iter_active = 0;
    } else {
      st->iter_active = 1;
      st->eps = eps;
      st->cg_total += steps;
      st->last_cg = steps;
      st->spmv_total += steps + 1;
      st->k_total += 1;
      st->j += 1;
    }
  }
}

// ------------------------------------------- dual step (Algorithm 1, y-update)
// y+ = y + sigma (2 A x+ - A x - b), projected to >= 0 on rows >= m_eq; the
// A x cache and the running average of y are updated in the same pass.
template <int G>
__global__ void __launch_bounds__(kBlock) k_dual(DevCsr A, const double* __restrict__ x,
                                                 const double* __restrict__ b, double* y,
                                                 double* ax, double* y_avg, const DevState* st) {
  if (!st->iter_active) return;
  const double sigma = st->sigma;
  const double inv_j = 1.0 / (double)st->j;
  const int m_eq = st->opt.m_eq;
  spmv_rows<G>(A, x, [&](int i, double s, bool lead) {
    if (lead) {
      double yn = y[i] + sigma * (2.0 * s - ax[i] - b[i]);
      if (i >= m_eq && yn < 0.0) yn = 0.0;
      y[i] = yn;
      ax[i] = s;
      y_avg[i] += (yn - y_avg[i]) * inv_j;
    }
  });
}

// A' y+ over the explicit transpose, fused with the running average of x.
template <int G>
__global__ void __launch_bounds__(kBlock) k_atv(DevCsr At, const double* __restrict__ y,
                                                double* aty, const double* __restrict__ x,
                                                double* x_avg, const DevState* st) {
  if (!st->iter_active) return;
  const double inv_j = 1.0 / (double)st->j;
  spmv_rows<G>(At, y, [&](int i, double s, bool lead) {
    if (lead) {
      aty[i] = s;
      x_avg[i] += (x[i] - x_avg[i]) * inv_j;
    }
  });
}

// Plain out = M v, optionally with per-block partial sums of out_i^2.
template <int G>
__global__ void __launch_bounds__(kBlock) k_spmv(DevCsr M, const double* __restrict__ v,
                                                 double* out, double* part_sq) {
  double acc = 0.0;
  spmv_rows<G>(M, v, [&](int i, double s, bool lead) {
    if (lead) {
      out[i] = s;
      acc = fma(s, s, acc);
    }
  });
  if (part_sq) block_sum_store(acc, part_sq + blockIdx.x);
}

// ------------------------------------------------ relKKT terms (Section 4)
// Per block (stride kPartStride), over the n index space:
//  [0] max|Qx + A'y + c|  [1] max|Qx|  [2] max|A'y|  [3] sum x.Qx  [4] sum c.x
//  [5..9] the same for the average (x~, y~)            [10] max|c|
template <int G>
__global__ void __launch_bounds__(kBlock) k_kkt_n(DevCsr Q, const double* __restrict__ x,
                                                  const double* __restrict__ x_avg,
                                                  const double* __restrict__ aty,
                                                  const double* __restrict__ aty_avg,
                                                  const double* __restrict__ c, double* part) {
  double v[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) v[k] = 0.0;
  spmv2_rows<G>(Q, x, x_avg, [&](int i, double qx, double qxa, bool lead) {
    if (lead) {
      const double ci = c[i];
      v[0] = fmax(v[0], fabs(qx + aty[i] + ci));
      v[1] = fmax(v[1], fabs(qx));
      v[2] = fmax(v[2], fabs(aty[i]));
      v[3] = fma(x[i], qx, v[3]);
      v[4] = fma(ci, x[i], v[4]);
      v[5] = fmax(v[5], fabs(qxa + aty_avg[i] + ci));
      v[6] = fmax(v[6], fabs(qxa));
      v[7] = fmax(v[7], fabs(aty_avg[i]));
      v[8] = fma(x_avg[i], qxa, v[8]);
      v[9] = fma(ci, x_avg[i], v[9]);
      v[10] = fmax(v[10], fabs(ci));
    }
  });
  // fmax drops NaN; a NaN iterate still reaches relKKT through the dot products.
  block_reduce_store<11>(v, kKktNMaxMask, part + size_t(blockIdx.x) * kPartStride);
}

// Over the m index space (A x~ is computed here and stored for a restart):
//  [0] max viol(x)  [1] max|Ax|  [2] sum b.y  [3] max viol(x~)  [4] max|Ax~|
//  [5] sum b.y~  [6] max|b|;  viol = |Ax-b| on equality rows, [Ax-b]^+ else.
template <int G>
__global__ void __launch_bounds__(kBlock) k_kkt_m(DevCsr A, const double* __restrict__ x_avg,
                                                  const double* __restrict__ ax, double* ax_avg,
                                                  const double* __restrict__ b,
                                                  const double* __restrict__ y,
                                                  const double* __restrict__ y_avg, int m_eq,
                                                  double* part) {
  double v[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) v[k] = 0.0;
  spmv_rows<G>(A, x_avg, [&](int i, double s, bool lead) {
    if (lead) {
      ax_avg[i] = s;
      const double bi = b[i];
      const double d = ax[i] - bi, da = s - bi;
      const double vc = i < m_eq ? fabs(d) : (d > 0.0 ? d : 0.0);
      const double va = i < m_eq ? fabs(da) : (da > 0.0 ? da : 0.0);
      v[0] = fmax(v[0], vc);
      v[1] = fmax(v[1], fabs(ax[i]));
      v[2] = fma(bi, y[i], v[2]);
      v[3] = fmax(v[3], va);
      v[4] = fmax(v[4], fabs(s));
      v[5] = fma(bi, y_avg[i], v[5]);
      v[6] = fmax(v[6], fabs(bi));
    }
  });
  block_reduce_store<7>(v, kKktMMaxMask, part + size_t(blockIdx.x) * kPartStride);
}

struct KktTerms {
  double t[6];
};

__device__ __forceinline__ KktTerms kkt_from(double maxviol, double maxAx, double maxb,
                                             double maxdres, double maxQx, double maxAty,
                                             double maxc, double xQx, double cx, double by) {
  KktTerms k;
  k.t[0] = maxviol / (1.0 + fmax(maxAx, maxb));
  k.t[1] = maxdres / (1.0 + fmax(maxQx, fmax(maxAty, maxc)));
  const double pobj = 0.5 * xQx + cx;
  k.t[2] = fabs(xQx + cx + by) / (1.0 + fmax(fabs(pobj), fabs(0.5 * xQx + by)));
  // relKKT = max of the three; a NaN anywhere must stay visible.
  double m = fmax(k.t[0], fmax(k.t[1], k.t[2]));
  if (isnan(k.t[0]) || isnan(k.t[1]) || isnan(k.t[2])) m = CUDART_NAN;
  k.t[3] = m;
  k.t[4] = pobj;
  k.t[5] = -0.5 * xQx - by;
  return k;
}

// One warp.  mode 0: evaluation at the starting point; 1: regular evaluation
// with termination and restart decisions; 2: evaluate only (no decisions).
__global__ void k_control(const double* part_n, int gn, const double* part_m, int gm, DevState* st,
                          int mode) {
  double rn[11], rm[7];
#pragma unroll
  for (int k = 0; k < 11; ++k)
    rn[k] = warp_reduce_partials(part_n + k, gn, kPartStride, (kKktNMaxMask >> k) & 1u);
#pragma unroll
  for (int k = 0; k < 7; ++k)
    rm[k] = warp_reduce_partials(part_m + k, gm, kPartStride, (kKktMMaxMask >> k) & 1u);
  if (threadIdx.x != 0) return;
  const KktTerms kc = kkt_from(rm[0], rm[1], rm[6], rn[0], rn[1], rn[2], rn[10], rn[3], rn[4], rm[2]);
  const KktTerms ka = kkt_from(rm[3], rm[4], rm[6], rn[5], rn[6], rn[7], rn[10], rn[8], rn[9], rm[5]);
  for (int k = 0; k < 6; ++k) {
    st->kkt_cur[k] = kc.t[k];
    st->kkt_avg[k] = ka.t[k];
  }
  if (mode == 2 || !running(st)) return;
  st->n_evals += 1;
  st->last_restart = 0;
  if (mode == 0) {
    st->relkkt_last = kc.t[3];
    st->kkt_anchor = kc.t[3];
    st->kkt_prev_cand = CUDART_INF;
    st->returned_avg = 0;
    for (int k = 0; k < 6; ++k) st->kkt_ret[k] = kc.t[k];
    if (!isfinite(kc.t[3])) st->done = kDoneNumerical;
    else if (kc.t[3] <= st->opt.tol) st->done = kDoneSolved;
    return;
  }
  // Candidate: the lower relKKT of the current iterate and the average.
  const bool has_avg = st->j > 0;
  const bool best_avg = has_avg && ka.t[3] <= kc.t[3];
  const KktTerms& best = best_avg ? ka : kc;
  for (int k = 0; k < 6; ++k) st->kkt_ret[k] = best.t[k];
  st->returned_avg = best_avg ? 1 : 0;
  if (!isfinite(best.t[3])) {
    st->done = kDoneNumerical;
    return;
  }
  if (best.t[3] <= st->opt.tol) {
    st->done = kDoneSolved;
    return;
  }
  st->relkkt_last = kc.t[3];
  if (st->opt.restart_mode == kRestartAdaptive && has_avg) {
    const double anchor = st->kkt_anchor, b = best.t[3];
    const bool restart = b <= st->opt.beta_suff * anchor ||
                         (b <= st->opt.beta_nec * anchor && b > st->kkt_prev_cand) ||
                         (double)st->j >= st->opt.beta_art * (double)st->k_total;
    if (restart) {
      st->restart_pending = best_avg ? 2 : 1;
      st->last_restart = st->restart_pending;
      st->kkt_cand = b;
      st->returned_avg = 0;  // the restart copies the candidate into (x, y)
    } else {
      st->kkt_prev_cand = b;
    }
  }
  if (st->k_total >= st->opt.max_iter) st->done = kDoneIterLimit;
}

// Restart to the candidate (Algorithm 1, restart step), n side: distance to
// the previous restart point for the primal weight, then anchor = x = cand.
__global__ void __launch_bounds__(kBlock) k_restart_n(double* x, const double* __restrict__ x_avg,
                                                      double* x_anchor, double* aty,
                                                      const double* __restrict__ aty_avg,
                                                      const DevState* st, int n, double* part) {
  const int pending = st->restart_pending;
  if (pending == 0) return;
  double acc = 0.0;
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const double cand = pending == 2 ? x_avg[i] : x[i];
    const double d = cand - x_anchor[i];
    acc = fma(d, d, acc);
    x_anchor[i] = cand;
    x[i] = cand;
    if (pending == 2) aty[i] = aty_avg[i];
  }
  block_sum_store(acc, part + blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) k_restart_m(double* y, const double* __restrict__ y_avg,
                                                      double* y_anchor, double* ax,
                                                      const double* __restrict__ ax_avg,
                                                      const DevState* st, int m, double* part) {
  const int pending = st->restart_pending;
  if (pending == 0) return;
  double acc = 0.0;
  for (long long i = grid_tid(); i < m; i += grid_threads()) {
    const double cand = pending == 2 ? y_avg[i] : y[i];
    const double d = cand - y_anchor[i];
    acc = fma(d, d, acc);
    y_anchor[i] = cand;
    y[i] = cand;
    if (pending == 2) ax[i] = ax_avg[i];
  }
  block_sum_store(acc, part + blockIdx.x);
}

// Primal weight (Section 4): omega <- exp(theta log(dy/dx) + (1-theta) log omega).
__global__ void k_restart_finish(const double* part_n, int gn, const double* part_m, int gm,
                                 DevState* st) {
  if (st->restart_pending == 0) return;
  const double dx2 = warp_reduce_partials(part_n, gn, 1, false);
  const double dy2 = warp_reduce_partials(part_m, gm, 1, false);
  if (threadIdx.x != 0) return;
  const double dx = sqrt(dx2), dy = sqrt(dy2);
  if (st->opt.pw_update && dx > st->opt.eps_zero && dy > st->opt.eps_zero) {
    const double th = st->opt.theta_pw;
    st->omega = exp(th * log(dy / dx) + (1.0 - th) * log(st->omega));
  }
  st->tau = st->eta / st->omega;
  st->sigma = st->eta * st->omega;
  st->j = 0;
  st->eps = 0.0;
  st->kkt_anchor = st->kkt_cand;
  st->kkt_prev_cand = CUDART_INF;
  st->relkkt_last = st->kkt_cand;
  st->n_restarts += 1;
  st->restart_pending = 0;
}

// ---------------------------------------------------------- set-up kernels
// Start of a solve: cold start zeros everything; warm start copies (x0, y0).
__global__ void k_init_vectors(double* x, double* x_avg, double* x_anchor,
                               const double* __restrict__ x0, int n, double* y, double* y_avg,
                               double* y_anchor, const double* __restrict__ y0, int m) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    const double v = x0 ? x0[i] : 0.0;
    x[i] = v;
    x_anchor[i] = v;
    x_avg[i] = 0.0;
  }
  for (long long i = grid_tid(); i < m; i += grid_threads()) {
    const double v = y0 ? y0[i] : 0.0;
    y[i] = v;
    y_anchor[i] = v;
    y_avg[i] = 0.0;
  }
}

// v = 1/sqrt(n) (power-iteration start) and per-block partials of ||c||^2, ||b||^2.
__global__ void k_pow_start(double* v, int n, const double* __restrict__ c,
                            const double* __restrict__ b, int m, double* part2) {
  const double v0 = 1.0 / sqrt((double)n);
  double a[2] = {0.0, 0.0};
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    v[i] = v0;
    a[0] = fma(c[i], c[i], a[0]);
  }
  for (long long i = grid_tid(); i < m; i += grid_threads()) a[1] = fma(b[i], b[i], a[1]);
  block_reduce_store<2>(a, 0u, part2 + size_t(blockIdx.x) * 2);
}

// v = w / lambda with lambda = ||w||_2 from the partials of the A' u pass.
__global__ void k_pow_scale(const double* __restrict__ w, double* v, int n, const double* part,
                            int gp, DevState* st) {
  const double lam = sqrt(block_all_reduce_partials(part, gp));
  const double inv_lam = lam > 0.0 ? 1.0 / lam : 0.0;
  for (long long i = grid_tid(); i < n; i += grid_threads()) v[i] = w[i] * inv_lam;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->lam = lam;
}

// eta = 1/(2||A||_2) (Section 3.2), omega0 = ||c||/||b|| (1 if either is ~0),
// tau = eta/omega, sigma = eta*omega.  reset != 0 also clears the counters.
__global__ void k_setup_finish(const double* part2, int g2, DevState* st, int reset) {
  double s0 = 0.0, s1 = 0.0;
  {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < g2; i += 32) {
      s0 += part2[2 * i];
      s1 += part2[2 * i + 1];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
  }
  if (threadIdx.x != 0) return;
  const DevOptions& o = st->opt;
  st->norm_A = sqrt(st->lam);
  st->eta = o.eta_override > 0.0 ? o.eta_override : 1.0 / (2.0 * fmax(st->norm_A, o.eps_zero));
  const double nc = sqrt(s0), nb = sqrt(s1);
  st->omega = o.omega0 > 0.0 ? o.omega0 : ((nc > o.eps_zero && nb > o.eps_zero) ? nc / nb : 1.0);
  st->tau = st->eta / st->omega;
  st->sigma = st->eta * st->omega;
  if (reset) {
    st->eps = 0.0;
    st->relkkt_last = CUDART_INF;
    st->kkt_anchor = CUDART_INF;
    st->kkt_prev_cand = CUDART_INF;
    st->kkt_cand = CUDART_INF;
    st->j = 0;
    st->k_total = 0;
    st->n_restarts = 0;
    st->cg_total = 0;
    st->last_cg = 0;
    st->n_evals = 0;
    st->spmv_total = 0;
    st->returned_avg = 0;
    st->iter_active = 0;
    st->restart_pending = 0;
    st->last_restart = 0;
  }
  st->done = 0;
  st->err = 0;
}

}  // namespace pdhcg
