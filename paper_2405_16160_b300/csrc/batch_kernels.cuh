// Device side of the batched solver: many small QPs, each solved to the end
// by one thread block in one persistent launch.
//
// An instance is min 1/2 x'Qx + c'x s.t. Ax <= b (first m_eq rows
// equalities) with Q = F F' + diag(qd), F n x k: the low-rank-plus-diagonal
// form of the paper's portfolio experiments, whose Q products cost 2nk
// (the P'P acceleration of Section 5.2).  Every step is the single-QP
// method: Algorithm 1 with the Section 4 heuristics (adaptive CG, restarts
// every eval_freq iterations, primal weight), the same readings and the same
// decision code (control_decide, restart_finish_decide,
// setup_finish_decide).
//
// Per block: a work queue hands out instance ids (an integer atomic; an
// instance's result does not depend on which block solves it).  The host
// groups instances of similar size into bins, each its own launch (on its
// own stream) with shared memory and block size fitted to the bin.  All vectors
// of the instance live in shared memory in FP64; the matrices stay in global
// memory (read through L1); an instance too large for shared memory keeps
// its vectors in a per-block slice of global memory instead.  The value type V of the data and of the Q, A,
// A' products is FP64 (the plain path) or FP32 (mixed); reductions, vector
// updates and every scalar are FP64 on both, and the relKKT of every
// evaluation is computed with the FP64 data, so termination is decided on
// the problem as given.
#pragma once

#include <type_traits>

#include "state.cuh"

namespace pdhcg {

// Rows with more entries than this are summed by a whole warp.
constexpr int kBatchLongRow = 32;

struct BatchDesc {
  int32_t n, m, m_eq, k;
  int64_t off_n, off_m;      // packed n- and m-vectors
  int64_t off_F;             // F, column-major (k x n: F[l * n + j])
  int64_t off_Arp, off_Ann;  // A: row pointers (instance-local), entries
  int64_t off_Trp, off_Tnn;  // A'
  int32_t off_Along, n_Along, off_Tlong, n_Tlong;  // rows with > kBatchLongRow entries
};

struct BatchResult {
  int32_t termination, returned_avg;
  long long iterations, cg_steps, restarts;
  double kkt[6];  // r_primal, r_dual, r_gap, relKKT, primal_obj, dual_obj
  double eta, omega, norm_A;
  long long attempts;
};

template <class V>
struct BatchData {
  const BatchDesc* desc;
  const int32_t* order;  // instance ids of this launch
  int count;
  const V* F;
  const V* qd;
  const double* F64;
  const double* qd64;
  const double* c;
  const double* b;
  const float* c32;  // FP32 copies of c and b (mixed precision)
  const float* b32;
  const int32_t* Arp;
  const int32_t* Acol;
  const V* Aval;
  const double* Aval64;
  const int32_t* Trp;
  const int32_t* Tcol;
  const V* Tval;
  const double* Tval64;
  const int32_t* Along;
  const int32_t* Tlong;
  const double* x0;
  const double* y0;
  int warm;
  // variable bounds, packed like x (+-inf where absent), or null: with them
  // every x-step is the Section 4 BB projected gradient
  const double* lo;
  const double* hi;
  const float* lo32;  // their FP32 copies (mixed precision)
  const float* hi32;
  double* x_out;
  double* y_out;
  BatchResult* res;
  int* next;
  DevOptions opt;
  int power_iters, eval_freq;
  int max_n, max_m, max_k;
  double* ws;          // per-block vector space in global memory, or null for shared memory
  long long ws_stride;  // doubles per block in ws
  int adaptive;         // Section 4 adaptive step size (its vectors are in the layout)
  const double* pow_table;  // step_decide's powers (kStepPowTable pairs)
};

// Vector space of one block, in doubles: shared memory when it fits, else
// a slice of a global workspace (same layout, reached through L1).  FP64
// vectors, plus (shadow) copies in the value type when that is FP32; the
// adaptive step size adds the start of the attempt (x, Q x) and the trial
// (y, A x).
inline size_t batch_block_doubles(int max_n, int max_m, int max_k, bool shadow,
                                  bool adaptive) {
  const size_t a = adaptive ? 2 * size_t(max_n) + 2 * size_t(max_m) : 0;
  const size_t d = 9 * size_t(max_n) + 6 * size_t(max_m) + size_t(max_k) + 16 + a;
  const size_t f = shadow ? 2 * size_t(max_n) + 2 * size_t(max_m) + size_t(max_k) + 8 : 0;
  return d + (f + 1) / 2;
}

template <class V>
struct LocalCsr {
  const int32_t* rp;
  const int32_t* col;
  const V* val;
  int rows;
  const int32_t* longr;
  int nlong;
};

template <class V>
__device__ __forceinline__ V warp_sum_v(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// out = M v: a thread per short row (entries in order), a warp per long row.
// The caller synchronises before reading out.
template <class V, int NT, class O = double>
__device__ void cta_spmv(const LocalCsr<V>& M, const V* v, O* out) {
  for (int i = threadIdx.x; i < M.rows; i += NT) {
    const int b = M.rp[i], e = M.rp[i + 1];
    if (e - b > kBatchLongRow) continue;
    V s = V(0);
    for (int k = b; k < e; ++k) s = fma(M.val[k], v[M.col[k]], s);
    out[i] = O(s);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = w; t < M.nlong; t += NT / 32) {
    const int i = M.longr[t];
    V s = V(0);
    for (int k = M.rp[i] + lane; k < M.rp[i + 1]; k += 32) s = fma(M.val[k], v[M.col[k]], s);
    s = warp_sum_v(s);
    if (lane == 0) out[i] = O(s);
  }
}

// The dual step fused into A x+ (Algorithm 1 y-update): whoever forms row i
// of A x+ also updates y_i = proj(y_i + sigma(2 (A x+)_i - (A x)_i - b_i)),
// its value-type copy, the A x cache and the running average.  With the
// adaptive step size (yn != nullptr) the step is a trial: y+ and A x+ go to
// yn and axn and nothing else changes.
template <class V, int NT>
__device__ void cta_dual(const LocalCsr<V>& A, const V* xv, const double* b, int m_eq,
                         double sigma, double inv_j, double* y, V* yv, double* ax, double* ya,
                         double* yn_out = nullptr, double* axn = nullptr) {
  auto row = [&](int i, double s) {
    double yn = y[i] + sigma * (2.0 * s - ax[i] - b[i]);
    if (i >= m_eq && yn < 0.0) yn = 0.0;
    if (yn_out) {
      yn_out[i] = yn;
      axn[i] = s;
      return;
    }
    y[i] = yn;
    yv[i] = V(yn);
    ax[i] = s;
    ya[i] += (yn - ya[i]) * inv_j;
  };
  for (int i = threadIdx.x; i < A.rows; i += NT) {
    const int b0 = A.rp[i], e = A.rp[i + 1];
    if (e - b0 > kBatchLongRow) continue;
    V s = V(0);
    for (int k = b0; k < e; ++k) s = fma(A.val[k], xv[A.col[k]], s);
    row(i, double(s));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = w; t < A.nlong; t += NT / 32) {
    const int i = A.longr[t];
    V s = V(0);
    for (int k = A.rp[i] + lane; k < A.rp[i + 1]; k += 32) s = fma(A.val[k], xv[A.col[k]], s);
    s = warp_sum_v(s);
    if (lane == 0) row(i, double(s));
  }
}

// out = (F F' + diag(qd)) p with F column-major: t = F'p by a warp per
// column, then a thread per row (row j by thread j mod NT).  p and t are in
// the value type.  Two barriers, out ready for every thread on return; with
// kSyncOut = false one barrier, and out[j] is ready for thread j mod NT only
// (the CG and BB steps read it that way, and a block reduction separates it
// from the next product's writes of t).
template <class V, int NT, bool kSyncOut = true, class O = double>
__device__ void cta_qprod(const V* F, const V* qd, int n, int k, const V* p, V* t, O* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = w; l < k; l += NT / 32) {
    const V* Fl = F + size_t(l) * n;
    V s = V(0);
    for (int j = lane; j < n; j += 32) s = fma(Fl[j], p[j], s);
    s = warp_sum_v(s);
    if (lane == 0) t[l] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) {
    V s = qd[j] * p[j];
    for (int l = 0; l < k; ++l) s = fma(F[size_t(l) * n + j], t[l], s);
    out[j] = O(s);
  }
  if constexpr (kSyncOut) __syncthreads();
}

// q = (F F' + diag(qd)) p as cta_qprod<V, NT, false> (q[j] ready for thread
// j mod NT), returning p'(Q + I/tau)p to every thread without a block
// reduction of its own: p'Q p = ||F'p||^2 + sum qd_j p_j^2, so the warps that
// form t = F'p also form one more "column", d = sum (qd_j + 1/tau) p_j^2
// (over the FP64 p), and after the product's one barrier every warp forms
// ||t||^2 + d with the same lanes and the same shuffle tree.  Used by the BB
// step, which needs two such products per step; the CG step keeps its block
// reduction of p'q (measured faster there: the FP64 column lengthens the
// product's critical path more than the barrier it saves).
template <class V, int NT>
__device__ double cta_qprod_pmp(const V* F, const V* qd, int n, int k, const V* p,
                                const double* p64, double inv_tau, V* t, double* td,
                                double* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = w; l <= k; l += NT / 32) {
    if (l < k) {
      const V* Fl = F + size_t(l) * n;
      V s = V(0);
      for (int j = lane; j < n; j += 32) s = fma(Fl[j], p[j], s);
      s = warp_sum_v(s);
      if (lane == 0) {
        t[l] = s;
        td[l] = double(s);
      }
    } else {
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s = fma((double(qd[j]) + inv_tau) * p64[j], p64[j], s);
      s = warp_sum(s);
      if (lane == 0) td[k] = s;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) {
    V s = qd[j] * p[j];
    for (int l = 0; l < k; ++l) s = fma(F[size_t(l) * n + j], t[l], s);
    out[j] = double(s);
  }
  // ||t||^2 by every warp alike: lane partials, then the xor tree
  double tt = 0.0;
  for (int l = lane; l < k; l += 32) tt = fma(td[l], td[l], tt);
  return td[k] + warp_sum(tt);
}

// Block-wide sums (S values) and maxima (M values) in one pass; every thread
// gets the results.  Warp partials are combined in warp order.
template <int NT, int S, int M>
__device__ void cta_reduce(double (&sum)[S > 0 ? S : 1], double (&mx)[M > 0 ? M : 1],
                           double* red) {
  constexpr int NW = NT / 32, K = S + M;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const double v = warp_sum(sum[s]);
    if (lane == 0) red[w * K + s] = v;
  }
#pragma unroll
  for (int s = 0; s < M; ++s) {
    double v = mx[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_xor(v, o));
    if (lane == 0) red[w * K + S + s] = v;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    double a = 0.0;
    for (int i = 0; i < NW; ++i) a += red[i * K + s];
    sum[s] = a;
  }
#pragma unroll
  for (int s = 0; s < M; ++s) {
    double a = 0.0;
    for (int i = 0; i < NW; ++i) a = fmax(a, red[i * K + S + s]);
    mx[s] = a;
  }
  __syncthreads();
}

// A block-wide sum whose total only thread 0 forms (the warp partials added
// in warp order, exactly as cta_reduce does) and hands to f(total) before the
// closing barrier; f writes what the block needs into shared memory.  The
// method's FP64 scalars (alpha, beta, the stop test) are then derived once
// per block instead of once per thread: B300's FP64 pipe runs at 1/58 of
// FP32, and a division or square root is dozens of its instructions.
template <int NT, class F>
__device__ __forceinline__ void cta_sum_t0(double v, double* red, F&& f) {
  constexpr int NW = NT / 32;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < NW; ++i) a += red[i];
    f(a);
  }
  __syncthreads();
}

// FP32 forms of the block sums, for the mixed solve: warp partials by xor
// shuffles, combined in warp order.  cta_sum_f gives every thread the S
// totals; cta_sum_t0f hands thread 0's total to f before the closing
// barrier, like cta_sum_t0.
template <int NT, int S>
__device__ __forceinline__ void cta_sum_f(float (&v)[S], float* red) {
  constexpr int NW = NT / 32;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float x = warp_sum_v(v[s]);
    if (lane == 0) red[w * S + s] = x;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    float a = 0.f;
    for (int i = 0; i < NW; ++i) a += red[i * S + s];
    v[s] = a;
  }
  __syncthreads();
}

template <int NT, class F>
__device__ __forceinline__ void cta_sum_t0f(float v, float* red, F&& f) {
  constexpr int NW = NT / 32;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum_v(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int i = 0; i < NW; ++i) a += red[i];
    f(a);
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double cta_sum1(double v, double* red) {
  double s[1] = {v}, m[1] = {0.0};
  cta_reduce<NT, 1, 0>(s, m, red);
  return s[0];
}

template <int NT>
__device__ __forceinline__ double cta_sum2(double v0, double v1, double* red, double* second) {
  double s[2] = {v0, v1}, m[1] = {0.0};
  cta_reduce<NT, 2, 0>(s, m, red);
  *second = s[1];
  return s[0];
}

// FP64 products of the data with (x, y) and with the averages (x~, y~),
// and F'x: the evaluation's scratch (4n + 2m + k doubles).
struct EvalScratch {
  double *Qx, *Qxa, *Aty, *Atya, *Ax, *Axa, *t;
};

// relKKT of (x, y) and of (x~, y~) with the FP64 data (Section 4), then the
// termination / restart decision (control_decide); every thread returns
// after it.
template <int NT>
__device__ void batch_evaluate(const double* F64, const double* qd64, const LocalCsr<double>& A64,
                               const LocalCsr<double>& At64, const double* c, const double* b,
                               const double* lo, const double* hi, const BatchDesc& d,
                               const double* x, const double* xa, const double* y,
                               const double* ya, const EvalScratch& e, DevState& st, double* red,
                               int mode) {
  const int n = d.n, m = d.m, k = d.k, tid = threadIdx.x;
  cta_qprod<double, NT>(F64, qd64, n, k, x, e.t, e.Qx);    // Q x
  cta_qprod<double, NT>(F64, qd64, n, k, xa, e.t, e.Qxa);  // Q x~
  cta_spmv<double, NT>(At64, y, e.Aty);                    // A'y
  cta_spmv<double, NT>(At64, ya, e.Atya);                  // A'y~
  cta_spmv<double, NT>(A64, x, e.Ax);                      // A x
  cta_spmv<double, NT>(A64, xa, e.Axa);                    // A x~
  __syncthreads();
  double s4[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, m7[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int j = tid; j < n; j += NT) {
    const double cj = c[j], q1 = e.Qx[j], q2 = e.Qxa[j];
    const double g1 = q1 + e.Aty[j] + cj, g2 = q2 + e.Atya[j] + cj;
    double l1 = 0.0, l2 = 0.0;
    if (lo) {  // reduced costs of the bounds
      l1 = reduced_cost(g1, lo[j], hi[j]);
      l2 = reduced_cost(g2, lo[j], hi[j]);
      s4[4] += bound_term(l1, lo[j], hi[j]);
      s4[5] += bound_term(l2, lo[j], hi[j]);
    }
    m7[0] = fmax(m7[0], fabs(g1 - l1));
    m7[1] = fmax(m7[1], fabs(q1));
    m7[2] = fmax(m7[2], fabs(e.Aty[j]));
    s4[0] = fma(x[j], q1, s4[0]);
    s4[1] = fma(cj, x[j], s4[1]);
    m7[3] = fmax(m7[3], fabs(g2 - l2));
    m7[4] = fmax(m7[4], fabs(q2));
    m7[5] = fmax(m7[5], fabs(e.Atya[j]));
    s4[2] = fma(xa[j], q2, s4[2]);
    s4[3] = fma(cj, xa[j], s4[3]);
    m7[6] = fmax(m7[6], fabs(cj));
  }
  cta_reduce<NT, 6, 7>(s4, m7, red);
  double s2[2] = {0.0, 0.0}, m5[5] = {0, 0, 0, 0, 0};
  for (int i = tid; i < m; i += NT) {
    const double bi = b[i], dd = e.Ax[i] - bi, da = e.Axa[i] - bi;
    const double vc = i < d.m_eq ? fabs(dd) : (dd > 0.0 ? dd : 0.0);
    const double va = i < d.m_eq ? fabs(da) : (da > 0.0 ? da : 0.0);
    m5[0] = fmax(m5[0], vc);
    m5[1] = fmax(m5[1], fabs(e.Ax[i]));
    s2[0] = fma(bi, y[i], s2[0]);
    m5[2] = fmax(m5[2], va);
    m5[3] = fmax(m5[3], fabs(e.Axa[i]));
    s2[1] = fma(bi, ya[i], s2[1]);
    m5[4] = fmax(m5[4], fabs(bi));
  }
  cta_reduce<NT, 2, 5>(s2, m5, red);
  if (tid == 0) {
    const KktTerms kc = kkt_from(m5[0], m5[1], m5[4], m7[0], m7[1], m7[2], m7[6], s4[0], s4[1],
                                 s2[0], s4[4]);
    const KktTerms ka = kkt_from(m5[2], m5[3], m5[4], m7[3], m7[4], m7[5], m7[6], s4[2], s4[3],
                                 s2[1], s4[5]);
    control_decide(&st, kc, ka, mode);
  }
  __syncthreads();
}

// One instance, solved by the whole block in FP64 (data, products, vectors
// and scalars).
template <int NT>
__device__ void batch_solve_fp64(const BatchData<double>& B, int id, double* sm, DevState& st,
                                 double* red) {
  using V = double;
  const BatchDesc d = B.desc[id];
  const int n = d.n, m = d.m, k = d.k, tid = threadIdx.x;
  // the FP64 scalars of the method, derived by thread 0 and read by all
  // (cta_sum_t0); s_flag: 0 go on, 1 stop, 2 numerical error
  __shared__ double s_sc[6];  // tau, 1/tau, eps, r'r (or s's), alpha or 1/alpha, beta
  __shared__ int s_flag;
  // FP64 vectors
  double* x = sm;
  double* xa = x + B.max_n;   // average
  double* x0 = xa + B.max_n;  // restart point
  double* r = x0 + B.max_n;
  double* p = r + B.max_n;
  double* q = p + B.max_n;
  double* qx = q + B.max_n;
  double* aty = qx + B.max_n;
  double* wv = aty + B.max_n;
  double* y = wv + B.max_n;
  double* ya = y + B.max_m;
  double* y0 = ya + B.max_m;
  double* ax = y0 + B.max_m;
  double* axe = ax + B.max_m;
  double* axa = axe + B.max_m;
  // adaptive step size: the attempt's start (x, Q x) and trial (y, A x)
  double* xs = axa + B.max_m;
  double* qxs = B.adaptive ? xs + B.max_n : xs;
  double* yn = B.adaptive ? qxs + B.max_n : xs;
  double* axn = B.adaptive ? yn + B.max_m : xs;
  double* t = B.adaptive ? axn + B.max_m : xs;
  // the vectors the products read
  V* pv = p;
  V* xv = x;
  V* yv = y;
  V* uv = axa;
  V* tv = t;
  // instance data
  const double* c = B.c + d.off_n;
  const double* b = B.b + d.off_m;
  const V* F = B.F + d.off_F;
  const V* qd = B.qd + d.off_n;
  const double* F64 = B.F64 + d.off_F;
  const double* qd64 = B.qd64 + d.off_n;
  const LocalCsr<V> A{B.Arp + d.off_Arp, B.Acol + d.off_Ann, B.Aval + d.off_Ann, m,
                      B.Along + d.off_Along, d.n_Along};
  const LocalCsr<V> At{B.Trp + d.off_Trp, B.Tcol + d.off_Tnn, B.Tval + d.off_Tnn, n,
                       B.Tlong + d.off_Tlong, d.n_Tlong};
  const LocalCsr<double> A64{A.rp, A.col, B.Aval64 + d.off_Ann, m, A.longr, A.nlong};
  const LocalCsr<double> At64{At.rp, At.col, B.Tval64 + d.off_Tnn, n, At.longr, At.nlong};

  // bounds count for this instance when one of them is finite (as for one
  // problem: all absent means CG x-steps)
  const double* lo = nullptr;
  const double* hi = nullptr;
  if (B.lo) {
    bool fin = false;
    for (int j = tid; j < n; j += NT)
      fin = fin || isfinite(B.lo[d.off_n + j]) || isfinite(B.hi[d.off_n + j]);
    if (__syncthreads_or(fin)) {
      lo = B.lo + d.off_n;
      hi = B.hi + d.off_n;
    }
  }
  // ---- start: x = x0 (warm) or 0 (projected into the box), empty averages
  for (int j = tid; j < n; j += NT) {
    double v = B.warm ? B.x0[d.off_n + j] : 0.0;
    if (lo) v = fmin(fmax(v, lo[j]), hi[j]);
    x[j] = v;
    x0[j] = v;
    xa[j] = 0.0;
  }
  for (int i = tid; i < m; i += NT) {
    const double v = B.warm ? B.y0[d.off_m + i] : 0.0;
    y[i] = v;
    y0[i] = v;
    ya[i] = 0.0;
  }
  if (tid == 0) {
    st.opt = B.opt;
    st.opt.m_eq = d.m_eq;
    st.lam = 0.0;
  }
  __syncthreads();
  // caches A x, A'y, Q x
  cta_spmv<V, NT>(A, xv, ax);
  cta_spmv<V, NT>(At, yv, aty);
  __syncthreads();
  cta_qprod<V, NT>(F, qd, n, k, xv, tv, qx);

  // ---- ||A||_2 by power iteration on A'A from ones/sqrt(n) (Section 3.2)
  {
    const double v0 = 1.0 / sqrt((double)n);
    double cc = 0.0, bb = 0.0;
    for (int j = tid; j < n; j += NT) {
      pv[j] = V(v0);
      cc = fma(c[j], c[j], cc);
    }
    for (int i = tid; i < m; i += NT) bb = fma(b[i], b[i], bb);
    double nb2;
    const double nc2 = cta_sum2<NT>(cc, bb, red, &nb2);
    double lam = 0.0;
    for (int it = 0; it < B.power_iters; ++it) {
      cta_spmv<V, NT>(A, pv, axa);  // u = A v
      __syncthreads();
      cta_spmv<V, NT>(At, uv, q);  // w = A'u
      __syncthreads();
      double ww = 0.0;
      for (int j = tid; j < n; j += NT) ww = fma(q[j], q[j], ww);
      cta_sum_t0<NT>(ww, red, [&](double t) {
        s_sc[0] = sqrt(t);
        s_sc[1] = s_sc[0] > 0.0 ? 1.0 / s_sc[0] : 0.0;
      });
      const double inv = s_sc[1];
      for (int j = tid; j < n; j += NT) pv[j] = V(q[j] * inv);
      __syncthreads();
    }
    if (tid == 0) {
      lam = s_sc[0];
      st.lam = lam;
      setup_finish_decide(&st, nc2, nb2, 1);
    }
    __syncthreads();
  }

  // ---- relKKT of (x, y) and (x~, y~) with the FP64 data (Section 4)
  const EvalScratch es{r, p, q, wv, axe, axa, t};
  auto evaluate = [&](int mode) {
    batch_evaluate<NT>(F64, qd64, A64, At64, c, b, lo, hi, d, x, xa, y, ya, es, st, red, mode);
  };
  // r0 = p0 = -(Qx + c + A'y): the CG start of the next iteration
  auto prepare = [&]() -> double {
    double rr = 0.0;
    for (int j = tid; j < n; j += NT) {
      const double v = -(qx[j] + c[j] + aty[j]);
      r[j] = v;
      p[j] = v;
      rr = fma(v, v, rr);
    }
    return cta_sum1<NT>(rr, red);
  };

  // adaptive step size: (x, Q x) at the start of the next attempt
  auto save_start = [&]() {
    if (!B.adaptive) return;
    for (int j = tid; j < n; j += NT) {
      xs[j] = x[j];
      qxs[j] = qx[j];
    }
  };

  evaluate(0);
  double rr0 = prepare();
  save_start();
  const int efreq = B.eval_freq;
  while (running(&st)) {
    for (int it = 0; it < efreq && running(&st) && st.attempts < st.opt.max_iter; ++it) {
      // ---- x-step: inexact CG on (Q + I/tau) x = x/tau - c - A'y (Section 2)
      const int mode = st.opt.cg_mode, nfix = st.opt.cg_fixed_n, cgmax = st.opt.cg_max;
      if (tid == 0) {
        s_sc[0] = st.tau;
        s_sc[1] = 1.0 / st.tau;
        s_sc[2] = mode == kCgAdaptive ? st.eps + st.opt.cg_eps_factor * st.relkkt_last : st.eps;
        s_sc[3] = rr0;
        s_flag = (mode == kCgFixed && nfix <= 0) || rr0 == 0.0;
      }
      __syncthreads();
      const double inv_tau = s_sc[1];
      int steps = 0;
      bool numerr = false;
      const bool skip = s_flag != 0;
      if (lo && !skip) {
        // ---- BB projected gradient (Section 4) from x, with r = p = -g:
        // alpha0 = g'Mg / g'g, then x+ = min(max(x + r/alpha, lo), hi), s = x+ - x,
        // r -= M s, Q x += Q s, alpha = s'Ms / s's (M = Q + I/tau)
        const double gmg = cta_qprod_pmp<V, NT>(F, qd, n, k, pv, p, inv_tau, tv, t, q);
        if (tid == 0) {
          s_flag = !(gmg > 0.0) || !isfinite(gmg) ? 2 : 0;
          s_sc[4] = 1.0 / (gmg / s_sc[3]);  // 1/alpha, alpha = g'Mg / g'g
        }
        __syncthreads();
        numerr = s_flag == 2;
        while (!numerr) {
          const double inv_alpha = s_sc[4];
          double ss = 0.0;
          for (int j = tid; j < n; j += NT) {
            const double xj = x[j];
            const double xn = fmin(fmax(xj + r[j] * inv_alpha, lo[j]), hi[j]);
            const double sj = xn - xj;
            p[j] = sj;
            x[j] = xn;
            ss = fma(sj, sj, ss);
          }
          cta_sum_t0<NT>(ss, red, [&](double t) { s_sc[3] = t; });
          // q = Q s and s'(Q + I/tau)s
          const double sw = cta_qprod_pmp<V, NT>(F, qd, n, k, pv, p, inv_tau, tv, t, q);
          for (int j = tid; j < n; j += NT) {
            const double sj = p[j], qj = q[j];
            r[j] -= qj + sj * inv_tau;
            qx[j] += qj;
          }
          if (tid == 0) {
            const double ssv = s_sc[3];
            const bool stop = mode == kCgFixed ? steps + 1 >= nfix
                                               : (sqrt(ssv) <= s_sc[2] || steps + 1 >= cgmax);
            if (stop || ssv == 0.0) {
              s_flag = 1;
            } else if (!(sw > 0.0) || !isfinite(sw)) {
              s_flag = 2;
            } else {
              s_flag = 0;
              s_sc[4] = 1.0 / (sw / ssv);  // 1/alpha, alpha = s'w / s's
            }
          }
          __syncthreads();
          ++steps;
          if (s_flag == 1) break;
          if (s_flag == 2) {
            numerr = true;
            break;
          }
        }
      }
      while (!skip && !lo) {
        cta_qprod<V, NT, false>(F, qd, n, k, pv, tv, q);  // q = Q p
        double pq = 0.0;
        for (int j = tid; j < n; j += NT) pq = fma(p[j], q[j] + p[j] * inv_tau, pq);
        cta_sum_t0<NT>(pq, red, [&](double t) {
          s_flag = !(t > 0.0) || !isfinite(t) ? 2 : 0;
          s_sc[4] = s_sc[3] / t;  // alpha = r'r / p'q
        });
        if (s_flag == 2) {
          numerr = true;
          break;
        }
        const double alpha = s_sc[4];
        double rn = 0.0;
        for (int j = tid; j < n; j += NT) {
          const double pj = p[j], qpj = q[j];
          const double xn = __dadd_rn(x[j], __dmul_rn(alpha, pj));
          x[j] = xn;
          qx[j] = __dadd_rn(qx[j], __dmul_rn(alpha, qpj));
          const double rj = __dsub_rn(r[j], __dmul_rn(alpha, qpj + pj * inv_tau));
          r[j] = rj;
          rn = fma(rj, rj, rn);
        }
        cta_sum_t0<NT>(rn, red, [&](double rr_new) {
          const bool stop = mode == kCgFixed
                                ? steps + 1 >= nfix
                                : (s_sc[0] * sqrt(rr_new) <= s_sc[2] || steps + 1 >= cgmax);
          s_flag = stop || rr_new == 0.0;
          s_sc[5] = rr_new / s_sc[3];  // beta
          s_sc[3] = rr_new;
        });
        ++steps;
        if (s_flag) break;
        const double beta = s_sc[5];
        for (int j = tid; j < n; j += NT) {
          const double pn = __dadd_rn(r[j], __dmul_rn(beta, p[j]));
          p[j] = pn;
        }
        __syncthreads();
      }
      if (numerr) {
        if (tid == 0) {
          st.done = kDoneNumerical;
          st.iter_active = 0;
        }
        __syncthreads();
        break;
      }
      if (tid == 0) {
        st.attempts += 1;
        st.cg_total += steps;
        st.last_cg = steps;
        if (B.adaptive) {
          st.eps_try = s_sc[2];
        } else {
          st.eps = s_sc[2];
          st.k_total += 1;
          st.j += 1;
        }
      }
      __syncthreads();
      if (B.adaptive) {
        // ---- trial y-step, the Section 4 step test, then commit or restore
        cta_dual<V, NT>(A, xv, b, d.m_eq, st.sigma, 0.0, y, yv, ax, ya, yn, axn);
        __syncthreads();
        double a4[4] = {0.0, 0.0, 0.0, 0.0}, m1[1] = {0.0};
        for (int j = tid; j < n; j += NT) {
          const double dx = x[j] - xs[j];
          a4[0] = fma(dx, dx, a4[0]);
          a4[1] = fma(dx, qx[j] - qxs[j], a4[1]);
        }
        for (int i = tid; i < m; i += NT) {
          const double dy = yn[i] - y[i];
          a4[2] = fma(dy, dy, a4[2]);
          a4[3] = fma(dy, axn[i] - ax[i], a4[3]);
        }
        cta_reduce<NT, 4, 0>(a4, m1, red);
        if (tid == 0) step_decide(&st, a4[0], a4[1], a4[2], a4[3], B.pow_table);
        __syncthreads();
        if (st.accepted) {
          const double w = st.avg_w;
          for (int i = tid; i < m; i += NT) {
            const double v = yn[i];
            y[i] = v;
            yv[i] = V(v);
            ax[i] = axn[i];
            ya[i] += (v - ya[i]) * w;
          }
          __syncthreads();
          cta_spmv<V, NT>(At, yv, aty);
          for (int j = tid; j < n; j += NT) xa[j] += (x[j] - xa[j]) * w;
        } else {
          for (int j = tid; j < n; j += NT) {
            x[j] = xs[j];
            qx[j] = qxs[j];
          }
        }
        __syncthreads();
        rr0 = prepare();
        save_start();
        __syncthreads();
        continue;
      }
      // ---- y-step fused into A x+, then A'y+, x~ and the next CG start
      if (tid == 0) s_sc[5] = 1.0 / (double)st.j;
      __syncthreads();
      const double inv_j = s_sc[5];
      cta_dual<V, NT>(A, xv, b, d.m_eq, st.sigma, inv_j, y, yv, ax, ya);
      __syncthreads();
      cta_spmv<V, NT>(At, yv, aty);
      for (int j = tid; j < n; j += NT) xa[j] += (x[j] - xa[j]) * inv_j;
      __syncthreads();
      rr0 = prepare();
    }
    // ---- evaluation, termination, restart (Section 4)
    evaluate(1);
    const int pending = st.restart_pending;
    if (pending != 0) {
      double dx = 0.0, dy = 0.0;
      for (int j = tid; j < n; j += NT) {
        const double cand = pending == 2 ? xa[j] : x[j];
        const double e = cand - x0[j];
        dx = fma(e, e, dx);
        x0[j] = cand;
        x[j] = cand;
      }
      for (int i = tid; i < m; i += NT) {
        const double cand = pending == 2 ? ya[i] : y[i];
        const double e = cand - y0[i];
        dy = fma(e, e, dy);
        y0[i] = cand;
        y[i] = cand;
      }
      double dy2;
      const double dx2 = cta_sum2<NT>(dx, dy, red, &dy2);
      if (tid == 0) restart_finish_decide(&st, dx2, dy2);
      __syncthreads();
      cta_spmv<V, NT>(A, xv, ax);
      cta_spmv<V, NT>(At, yv, aty);
      __syncthreads();
    }
    // exact Q x for the tracked cache, then the next CG start
    cta_qprod<V, NT>(F, qd, n, k, xv, tv, qx);
    rr0 = prepare();
    save_start();
    __syncthreads();
  }

  // ---- the returned iterate and its statistics
  const bool avg = st.returned_avg != 0;
  for (int j = tid; j < n; j += NT) B.x_out[d.off_n + j] = avg ? xa[j] : x[j];
  for (int i = tid; i < m; i += NT) B.y_out[d.off_m + i] = avg ? ya[i] : y[i];
  if (tid == 0) {
    BatchResult& o = B.res[id];
    o.termination = st.done > 0 ? st.done - 1 : 1;
    o.returned_avg = st.returned_avg;
    o.iterations = st.k_total;
    o.cg_steps = st.cg_total;
    o.restarts = st.n_restarts;
    for (int s = 0; s < 6; ++s) o.kkt[s] = st.kkt_ret[s];
    o.eta = st.eta;
    o.omega = st.omega;
    o.norm_A = st.norm_A;
    o.attempts = st.attempts;
  }
  __syncthreads();
}

// ------------------------------------------------------------ mixed mode
// Vector space of one block of the mixed-precision solve, in doubles.  The
// restart points x0, y0 in FP64 (n + m).  The iterates x and y and their
// running averages as FP32 pairs hi + lo (split_add; 2n + 2m).  The rest is
// one region used two ways.  During the attempts it holds F'p's FP64 copy
// (k + 16) and the FP32 working vectors: the trial x the products read, r,
// p, q, the tracked Q x, A'y, the attempt's moves dx of x and dq of Q x (8n);
// the A x cache, the trial A x and the trial y pair (4m); F'p (k + 16).
// During an evaluation it holds the FP64 products of (x, y) and of the
// averages (4n + 2m), F'x (k + 16) and the FP64 values of x, y and the
// averages (2n + 2m); the FP32 vectors are formed again after it.
inline size_t batch_block_doubles_mixed(int max_n, int max_m, int max_k) {
  const size_t n = size_t(max_n), m = size_t(max_m), k = size_t(max_k) + 16;
  const size_t iter = k + (8 * n + 4 * m + k + 1) / 2;
  const size_t eval = 6 * n + 4 * m + k;
  return 3 * n + 3 * m + (iter > eval ? iter : eval);
}

// q = (F F' + diag(qd)) p in FP32 as cta_qprod<float, NT, false, float>,
// returning p'(Q + I/tau)p = ||F'p||^2 + sum (qd_j + 1/tau) p_j^2 to every
// thread: the warps that form t = F'p form the diagonal sum as one more
// column, and after the product's one barrier every warp adds the squares of
// t (FP64) with the same lanes and shuffle tree.  The mixed BB step's product.
template <int NT>
__device__ double cta_qprod_pmp_f(const float* F, const float* qd, int n, int k, const float* p,
                                  float inv_tau, float* t, double* td, float* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = w; l <= k; l += NT / 32) {
    float s = 0.f;
    if (l < k) {
      const float* Fl = F + size_t(l) * n;
      for (int j = lane; j < n; j += 32) s = fmaf(Fl[j], p[j], s);
    } else {
      for (int j = lane; j < n; j += 32) s = fmaf((qd[j] + inv_tau) * p[j], p[j], s);
    }
    s = warp_sum_v(s);
    if (lane == 0) {
      if (l < k) t[l] = s;
      td[l] = double(s);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) {
    float s = qd[j] * p[j];
    for (int l = 0; l < k; ++l) s = fmaf(F[size_t(l) * n + j], t[l], s);
    out[j] = s;
  }
  double tt = 0.0;
  for (int l = lane; l < k; l += 32) tt = fma(td[l], td[l], tt);
  return td[k] + warp_sum(tt);
}

// A pair's value, and a value as a pair (hi the nearest float).
__device__ __forceinline__ double pair_value(float hi, float lo) {
  return double(hi) + double(lo);
}
__device__ __forceinline__ void pair_set(double v, float& hi, float& lo) {
  hi = float(v);
  lo = float(v - double(hi));
}
// The running average (ah, al) += ((h, l) - (ah, al)) w; weight 1 (the first
// point after a start or restart) copies the pair exactly.
__device__ __forceinline__ void pair_average(float& ah, float& al, float h, float l, float w) {
  if (w == 1.f) {
    ah = h;
    al = l;
  } else {
    float a = ah, b = al;
    split_add(a, b, ((h - a) + (l - b)) * w);
    ah = a;
    al = b;
  }
}

// The mixed dual step fused into A x+: the move sigma (2 (A x+)_i - (A x)_i -
// b_i), added to the pair y_i and projected, all in FP32.  With the adaptive
// step size (ynh != nullptr) the result is a trial: y+ and A x+ go to
// (ynh, ynl) and axn.  Otherwise y, the A x cache and the running average of
// y (weight w) are updated.
template <int NT>
__device__ void cta_dual_mixed(const LocalCsr<float>& A, const float* xv, const float* b,
                               int m_eq, float sigma, float w, float* yh, float* yl, float* ax,
                               float* yah, float* yal, float* ynh = nullptr,
                               float* ynl = nullptr, float* axn = nullptr) {
  auto row = [&](int i, float s) {
    float h = yh[i], l = yl[i];
    split_add(h, l, sigma * (2.f * s - ax[i] - b[i]));
    if (i >= m_eq && h < 0.f) h = l = 0.f;
    if (ynh) {
      ynh[i] = h;
      ynl[i] = l;
      axn[i] = s;
      return;
    }
    yh[i] = h;
    yl[i] = l;
    ax[i] = s;
    pair_average(yah[i], yal[i], h, l, w);
  };
  for (int i = threadIdx.x; i < A.rows; i += NT) {
    const int b0 = A.rp[i], e = A.rp[i + 1];
    if (e - b0 > kBatchLongRow) continue;
    float s = 0.f;
    for (int k = b0; k < e; ++k) s = fmaf(A.val[k], xv[A.col[k]], s);
    row(i, s);
  }
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = wp; t < A.nlong; t += NT / 32) {
    const int i = A.longr[t];
    float s = 0.f;
    for (int k = A.rp[i] + lane; k < A.rp[i + 1]; k += 32) s = fmaf(A.val[k], xv[A.col[k]], s);
    s = warp_sum_v(s);
    if (lane == 0) row(i, s);
  }
}

// One instance in mixed precision, solved by the whole block.  The data of
// the iterations (F, qd, A, A', c, b and the bounds) and every vector of an
// attempt are FP32, with per-thread FP32 partial sums whose block totals
// and the method's scalars are FP64.  The iterates x and y and their running
// averages are FP32 pairs (split_add), whose high words the products read:
// an attempt adds up its move dx of x and leaves x alone, a kept attempt adds
// dx to x once, a rejected one is dropped with nothing to restore.  So every
// per-element operation of an attempt runs on the FP32 pipe (B300's FP64
// pipe is 1/58 of it).  Each evaluation forms x, y and the averages in FP64
// and uses the FP64 data (batch_evaluate), as the FP64 solve does, so
// termination is decided on the problem as given; the restart points are
// FP64.  The method and its decisions are those of batch_solve_fp64.
template <int NT>
__device__ void batch_solve_mixed(const BatchData<float>& B, int id, double* sm, DevState& st,
                                  double* red) {
  const BatchDesc d = B.desc[id];
  const int n = d.n, m = d.m, k = d.k, tid = threadIdx.x;
  const int Nn = B.max_n, Mm = B.max_m, Kk = B.max_k + 16;
  // The scalars of an attempt, derived by thread 0 from the FP32 block
  // sums (cta_sum_t0f) in FP32, the precision they are applied in (FP64
  // divisions and square roots on one thread would hold up the block for
  // microseconds on B300's narrow FP64 pipe); s_flag: 0 go on, 1 stop,
  // 2 numerical error
  __shared__ double s_sc[1];  // ||A|| of the power iteration
  // 1/tau, alpha or 1/alpha, beta, sigma, average weight, tau, eps, r'r (or s's)
  __shared__ float s_f[8];
  __shared__ int s_flag;
  double* x0 = sm;  // restart points
  double* y0 = x0 + Nn;
  float* xh = reinterpret_cast<float*>(y0 + Mm);  // x = xh + xl
  float* xl = xh + Nn;
  float* xah = xl + Nn;  // its running average
  float* xal = xah + Nn;
  float* yh = xal + Nn;  // y = yh + yl
  float* yl = yh + Mm;
  float* yah = yl + Mm;
  float* yal = yah + Mm;
  double* U = y0 + Mm + 2 * Nn + 2 * Mm;
  // the attempts' view of U
  double* td = U;  // F'p in FP64 (BB step)
  float* xv = reinterpret_cast<float*>(td + Kk);  // x as the products read it (trial x)
  float* r = xv + Nn;
  float* p = r + Nn;
  float* q = p + Nn;
  float* qx = q + Nn;  // tracked Q x
  float* aty = qx + Nn;
  float* dx = aty + Nn;  // the attempt's move of x
  float* dq = dx + Nn;   // and of Q x
  float* ax = dq + Nn;   // A x cache
  float* axn = ax + Mm;  // trial A x
  float* ynh = axn + Mm;  // trial y
  float* ynl = ynh + Mm;
  float* t = ynl + Mm;  // F'p
  // the evaluation's view of U
  const EvalScratch es{U, U + Nn, U + 2 * Nn, U + 3 * Nn, U + 4 * Nn, U + 4 * Nn + Mm,
                       U + 4 * Nn + 2 * Mm};
  double* x64 = U + 4 * Nn + 2 * Mm + Kk;
  double* xa64 = x64 + Nn;
  double* y64 = xa64 + Nn;
  double* ya64 = y64 + Mm;
  // instance data
  const double* c = B.c + d.off_n;
  const double* b = B.b + d.off_m;
  const float* c32 = B.c32 + d.off_n;
  const float* b32 = B.b32 + d.off_m;
  const float* F = B.F + d.off_F;
  const float* qd = B.qd + d.off_n;
  const double* F64 = B.F64 + d.off_F;
  const double* qd64 = B.qd64 + d.off_n;
  const LocalCsr<float> A{B.Arp + d.off_Arp, B.Acol + d.off_Ann, B.Aval + d.off_Ann, m,
                          B.Along + d.off_Along, d.n_Along};
  const LocalCsr<float> At{B.Trp + d.off_Trp, B.Tcol + d.off_Tnn, B.Tval + d.off_Tnn, n,
                           B.Tlong + d.off_Tlong, d.n_Tlong};
  const LocalCsr<double> A64{A.rp, A.col, B.Aval64 + d.off_Ann, m, A.longr, A.nlong};
  const LocalCsr<double> At64{At.rp, At.col, B.Tval64 + d.off_Tnn, n, At.longr, At.nlong};

  const double* lo = nullptr;
  const double* hi = nullptr;
  const float* lo32 = nullptr;
  const float* hi32 = nullptr;
  if (B.lo) {
    bool fin = false;
    for (int j = tid; j < n; j += NT)
      fin = fin || isfinite(B.lo[d.off_n + j]) || isfinite(B.hi[d.off_n + j]);
    if (__syncthreads_or(fin)) {
      lo = B.lo + d.off_n;
      hi = B.hi + d.off_n;
      lo32 = B.lo32 + d.off_n;
      hi32 = B.hi32 + d.off_n;
    }
  }
  // ---- start: x = x0 (warm) or 0 (projected into the box), empty averages
  for (int j = tid; j < n; j += NT) {
    double v = B.warm ? B.x0[d.off_n + j] : 0.0;
    if (lo) v = fmin(fmax(v, lo[j]), hi[j]);
    x0[j] = v;
    pair_set(v, xh[j], xl[j]);
    xah[j] = 0.f;
    xal[j] = 0.f;
  }
  for (int i = tid; i < m; i += NT) {
    const double v = B.warm ? B.y0[d.off_m + i] : 0.0;
    y0[i] = v;
    pair_set(v, yh[i], yl[i]);
    yah[i] = 0.f;
    yal[i] = 0.f;
  }
  if (tid == 0) {
    st.opt = B.opt;
    st.opt.m_eq = d.m_eq;
    st.lam = 0.0;
  }
  __syncthreads();

  // ---- ||A||_2 by power iteration on A'A from ones/sqrt(n) (Section 3.2)
  {
    const float v0 = float(1.0 / sqrt((double)n));
    double cc = 0.0, bb = 0.0;
    for (int j = tid; j < n; j += NT) {
      p[j] = v0;
      cc = fma(c[j], c[j], cc);
    }
    for (int i = tid; i < m; i += NT) bb = fma(b[i], b[i], bb);
    double nb2;
    const double nc2 = cta_sum2<NT>(cc, bb, red, &nb2);
    for (int it = 0; it < B.power_iters; ++it) {
      cta_spmv<float, NT, float>(A, p, ax);  // u = A v
      __syncthreads();
      cta_spmv<float, NT, float>(At, ax, q);  // w = A'u
      __syncthreads();
      float ww = 0.f;
      for (int j = tid; j < n; j += NT) ww = fmaf(q[j], q[j], ww);
      cta_sum_t0<NT>(double(ww), red, [&](double tt) {
        s_sc[0] = sqrt(tt);
        s_f[0] = s_sc[0] > 0.0 ? float(1.0 / s_sc[0]) : 0.f;
      });
      const float inv = s_f[0];
      for (int j = tid; j < n; j += NT) p[j] = q[j] * inv;
      __syncthreads();
    }
    if (tid == 0) {
      st.lam = s_sc[0];
      setup_finish_decide(&st, nc2, nb2, 1);
    }
    __syncthreads();
  }

  // relKKT of the FP64 values of the pairs, with the FP64 data
  auto evaluate = [&](int mode) {
    for (int j = tid; j < n; j += NT) {
      x64[j] = pair_value(xh[j], xl[j]);
      xa64[j] = pair_value(xah[j], xal[j]);
    }
    for (int i = tid; i < m; i += NT) {
      y64[i] = pair_value(yh[i], yl[i]);
      ya64[i] = pair_value(yah[i], yal[i]);
    }
    __syncthreads();
    batch_evaluate<NT>(F64, qd64, A64, At64, c, b, lo, hi, d, x64, xa64, y64, ya64, es, st, red,
                       mode);
  };
  // the FP32 vectors from the iterates: x for the products, the A x, A'y and
  // Q x caches
  auto refresh = [&]() {
    for (int j = tid; j < n; j += NT) xv[j] = xh[j];
    __syncthreads();
    cta_spmv<float, NT, float>(A, xv, ax);
    cta_spmv<float, NT, float>(At, yh, aty);
    __syncthreads();
    cta_qprod<float, NT, true, float>(F, qd, n, k, xv, t, qx);
  };
  float* redf = reinterpret_cast<float*>(red);
  // r0 = p0 = -(Qx + c + A'y), the next attempt's CG start, and empty moves
  auto prepare = [&]() -> float {
    float rr = 0.f;
    for (int j = tid; j < n; j += NT) {
      const float v = -(qx[j] + c32[j] + aty[j]);
      r[j] = v;
      p[j] = v;
      dx[j] = 0.f;
      dq[j] = 0.f;
      rr = fmaf(v, v, rr);
    }
    float t1[1] = {rr};
    cta_sum_f<NT, 1>(t1, redf);
    return t1[0];
  };
  // an attempt is kept: x += dx (projected into the box when there is one),
  // Q x += dq, and the running average of x with weight w
  auto commit_x = [&](float w) {
    for (int j = tid; j < n; j += NT) {
      float h = xh[j], l = xl[j];
      split_add(h, l, dx[j]);
      if (lo && (h <= lo32[j] || h >= hi32[j])) {  // at or past a bound: project in FP64
        const double v = pair_value(h, l);
        if (v < lo[j] || v > hi[j]) pair_set(fmin(fmax(v, lo[j]), hi[j]), h, l);
      }
      xh[j] = h;
      xl[j] = l;
      xv[j] = h;
      qx[j] += dq[j];
      pair_average(xah[j], xal[j], h, l, w);
    }
  };

  evaluate(0);
  refresh();
  float rr0 = prepare();
  const int efreq = B.eval_freq;
  while (running(&st)) {
    for (int it = 0; it < efreq && running(&st) && st.attempts < st.opt.max_iter; ++it) {
      // ---- x-step: inexact CG on (Q + I/tau) x = x/tau - c - A'y (Section 2)
      const int mode = st.opt.cg_mode, nfix = st.opt.cg_fixed_n, cgmax = st.opt.cg_max;
      if (tid == 0) {
        const double eps =
            mode == kCgAdaptive ? st.eps + st.opt.cg_eps_factor * st.relkkt_last : st.eps;
        if (B.adaptive)
          st.eps_try = eps;
        else
          st.eps = eps;
        s_f[5] = float(st.tau);
        s_f[0] = 1.f / s_f[5];
        s_f[3] = float(st.sigma);
        s_f[6] = float(eps);
        s_f[7] = rr0;
        s_flag = (mode == kCgFixed && nfix <= 0) || rr0 == 0.f;
      }
      __syncthreads();
      const float inv_tau = s_f[0];
      int steps = 0;
      bool numerr = false;
      const bool skip = s_flag != 0;
      if (lo && !skip) {
        // ---- BB projected gradient (Section 4) from x, with r = p = -g, on
        // the FP32 x the products read (xv), whose moves add up in dx
        const double gmg = cta_qprod_pmp_f<NT>(F, qd, n, k, p, inv_tau, t, td, q);
        if (tid == 0) {
          s_flag = !(gmg > 0.0) || !isfinite(gmg) ? 2 : 0;
          s_f[1] = s_f[7] / float(gmg);  // 1/alpha, alpha = g'Mg / g'g
        }
        __syncthreads();
        numerr = s_flag == 2;
        while (!numerr) {
          const float inv_alpha = s_f[1];
          float ss = 0.f;
          for (int j = tid; j < n; j += NT) {
            const float xj = xv[j];
            const float xn = fminf(fmaxf(fmaf(r[j], inv_alpha, xj), lo32[j]), hi32[j]);
            const float sj = xn - xj;
            p[j] = sj;
            xv[j] = xn;
            dx[j] += sj;
            ss = fmaf(sj, sj, ss);
          }
          cta_sum_t0f<NT>(ss, redf, [&](float tt) { s_f[7] = tt; });
          // q = Q s and s'(Q + I/tau)s
          const double sw = cta_qprod_pmp_f<NT>(F, qd, n, k, p, inv_tau, t, td, q);
          for (int j = tid; j < n; j += NT) {
            const float sj = p[j], qj = q[j];
            r[j] -= fmaf(sj, inv_tau, qj);
            dq[j] += qj;
          }
          if (tid == 0) {
            const float ssv = s_f[7];
            const bool stop = mode == kCgFixed ? steps + 1 >= nfix
                                               : (sqrtf(ssv) <= s_f[6] || steps + 1 >= cgmax);
            if (stop || ssv == 0.f) {
              s_flag = 1;
            } else if (!(sw > 0.0) || !isfinite(sw)) {
              s_flag = 2;
            } else {
              s_flag = 0;
              s_f[1] = ssv / float(sw);  // 1/alpha, alpha = s'w / s's
            }
          }
          __syncthreads();
          ++steps;
          if (s_flag == 1) break;
          if (s_flag == 2) {
            numerr = true;
            break;
          }
        }
      }
      // CG with one barrier per product: the warps that form t = F'p (with
      // p = r + beta p, i.e. t = F'r + beta t) also form the diagonal part
      // sum (qd_j + 1/tau) p_j^2 as one more column; after the barrier every
      // warp forms p'(Q + I/tau)p = ||t||^2 + that sum with the same lanes and
      // shuffle tree, so alpha needs no block reduction; one pass over the
      // rows then forms p, q = Q p and the updates, and r'r is the step's one
      // block sum.
      if (!skip && !lo) {
        const int wp = tid >> 5, lane = tid & 31;
        float beta = 0.f;  // the first step: p = r
        for (;;) {
          for (int l = wp; l <= k; l += NT / 32) {
            float sa = 0.f;
            if (l < k) {
              const float* Fl = F + size_t(l) * n;
              for (int j = lane; j < n; j += 32) sa = fmaf(Fl[j], r[j], sa);
            } else {
              for (int j = lane; j < n; j += 32) {
                const float pj = fmaf(beta, p[j], r[j]);
                sa = fmaf((qd[j] + inv_tau) * pj, pj, sa);
              }
            }
            sa = warp_sum_v(sa);
            if (lane == 0) t[l] = (l < k && beta != 0.f) ? fmaf(beta, t[l], sa) : sa;
          }
          __syncthreads();
          float tt = 0.f;
          for (int l = lane; l < k; l += 32) tt = fmaf(t[l], t[l], tt);
          const float pq = warp_sum_v(tt) + t[k];
          if (!(pq > 0.f) || !isfinite(pq)) {  // the same value in every thread
            numerr = true;
            break;
          }
          const float alpha = s_f[7] / pq;  // alpha = r'r / p'(Q + I/tau)p
          float rn = 0.f;
          for (int j = tid; j < n; j += NT) {
            const float pj = fmaf(beta, p[j], r[j]);
            float qj = qd[j] * pj;
            for (int l = 0; l < k; ++l) qj = fmaf(F[size_t(l) * n + j], t[l], qj);
            p[j] = pj;
            dx[j] = fmaf(alpha, pj, dx[j]);
            dq[j] = fmaf(alpha, qj, dq[j]);
            const float rj = fmaf(-alpha, fmaf(pj, inv_tau, qj), r[j]);
            r[j] = rj;
            rn = fmaf(rj, rj, rn);
          }
          cta_sum_t0f<NT>(rn, redf, [&](float rr_new) {
            const bool stop = mode == kCgFixed
                                  ? steps + 1 >= nfix
                                  : (s_f[5] * sqrtf(rr_new) <= s_f[6] || steps + 1 >= cgmax);
            s_flag = stop || rr_new == 0.f;
            s_f[2] = rr_new / s_f[7];  // beta
            s_f[7] = rr_new;
          });
          ++steps;
          if (s_flag) break;
          beta = s_f[2];
        }
      }
      if (numerr) {
        if (tid == 0) {
          st.done = kDoneNumerical;
          st.iter_active = 0;
        }
        __syncthreads();
        break;
      }
      if (tid == 0) {
        st.attempts += 1;
        st.cg_total += steps;
        st.last_cg = steps;
        if (!B.adaptive) {
          st.k_total += 1;
          st.j += 1;
          s_f[4] = 1.f / float(st.j);
        }
      }
      __syncthreads();
      const float sigma = s_f[3];
      if (B.adaptive) {
        // ---- trial y-step at x + dx, the Section 4 step test on the moves,
        // then keep or drop the attempt
        float f4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = tid; j < n; j += NT) {
          const float mj = dx[j];
          if (!lo) xv[j] += mj;  // the BB step already moved xv
          f4[0] = fmaf(mj, mj, f4[0]);
          f4[1] = fmaf(mj, dq[j], f4[1]);
        }
        __syncthreads();
        cta_dual_mixed<NT>(A, xv, b32, d.m_eq, sigma, 0.f, yh, yl, ax, yah, yal, ynh, ynl, axn);
        __syncthreads();
        for (int i = tid; i < m; i += NT) {
          const float dy = (ynh[i] - yh[i]) + (ynl[i] - yl[i]);
          f4[2] = fmaf(dy, dy, f4[2]);
          f4[3] = fmaf(dy, axn[i] - ax[i], f4[3]);
        }
        cta_sum_f<NT, 4>(f4, redf);
        if (tid == 0) {
          step_decide_f(&st, f4[0], f4[1], f4[2], f4[3], B.pow_table);
          s_f[4] = float(st.avg_w);
        }
        __syncthreads();
        if (st.accepted) {
          const float w = s_f[4];
          for (int i = tid; i < m; i += NT) {
            const float h = ynh[i], l = ynl[i];
            yh[i] = h;
            yl[i] = l;
            ax[i] = axn[i];
            pair_average(yah[i], yal[i], h, l, w);
          }
          commit_x(w);
          __syncthreads();
          cta_spmv<float, NT, float>(At, yh, aty);
        } else {
          for (int j = tid; j < n; j += NT) xv[j] = xh[j];
        }
        __syncthreads();
        rr0 = prepare();
        continue;
      }
      // ---- keep the x-step, then the y-step fused into A x+, A'y+ and the
      // next CG start
      const float inv_j = s_f[4];
      commit_x(inv_j);
      __syncthreads();
      cta_dual_mixed<NT>(A, xv, b32, d.m_eq, sigma, inv_j, yh, yl, ax, yah, yal);
      __syncthreads();
      cta_spmv<float, NT, float>(At, yh, aty);
      __syncthreads();
      rr0 = prepare();
    }
    // ---- evaluation, termination, restart (Section 4)
    evaluate(1);
    const int pending = st.restart_pending;
    if (pending != 0) {
      double ex = 0.0, ey = 0.0;
      for (int j = tid; j < n; j += NT) {
        const double cand = pending == 2 ? xa64[j] : x64[j];
        const double e = cand - x0[j];
        ex = fma(e, e, ex);
        x0[j] = cand;
        if (pending == 2) {
          xh[j] = xah[j];
          xl[j] = xal[j];
        }
      }
      for (int i = tid; i < m; i += NT) {
        const double cand = pending == 2 ? ya64[i] : y64[i];
        const double e = cand - y0[i];
        ey = fma(e, e, ey);
        y0[i] = cand;
        if (pending == 2) {
          yh[i] = yah[i];
          yl[i] = yal[i];
        }
      }
      double dy2;
      const double dx2 = cta_sum2<NT>(ex, ey, red, &dy2);
      if (tid == 0) restart_finish_decide(&st, dx2, dy2);
      __syncthreads();
    }
    refresh();
    rr0 = prepare();
    __syncthreads();
  }

  // ---- the returned iterate and its statistics
  const bool avg = st.returned_avg != 0;
  for (int j = tid; j < n; j += NT)
    B.x_out[d.off_n + j] = avg ? pair_value(xah[j], xal[j]) : pair_value(xh[j], xl[j]);
  for (int i = tid; i < m; i += NT)
    B.y_out[d.off_m + i] = avg ? pair_value(yah[i], yal[i]) : pair_value(yh[i], yl[i]);
  if (tid == 0) {
    BatchResult& o = B.res[id];
    o.termination = st.done > 0 ? st.done - 1 : 1;
    o.returned_avg = st.returned_avg;
    o.iterations = st.k_total;
    o.cg_steps = st.cg_total;
    o.restarts = st.n_restarts;
    for (int s = 0; s < 6; ++s) o.kkt[s] = st.kkt_ret[s];
    o.eta = st.eta;
    o.omega = st.omega;
    o.norm_A = st.norm_A;
    o.attempts = st.attempts;
  }
  __syncthreads();
}

// Blocks per SM the register budget is sized for (launch bounds): 128
// registers per thread at every block size.
template <class V, int NT>
constexpr int batch_min_blocks() {
  return NT == 64 ? 8 : (NT == 128 ? 4 : (NT == 256 ? 2 : 1));
}

// The work queue of one block: instances until the queue is empty, each
// solved with its vectors at sm.
template <class V, int NT>
__device__ __forceinline__ void batch_queue(const BatchData<V>& B, double* sm, DevState& st,
                                            double* red, int& id_s) {
  for (;;) {
    if (threadIdx.x == 0) id_s = atomicAdd(B.next, 1);
    __syncthreads();
    const int idx = id_s;
    __syncthreads();
    if (idx >= B.count) break;
    if constexpr (std::is_same<V, float>::value)
      batch_solve_mixed<NT>(B, B.order[idx], sm, st, red);
    else
      batch_solve_fp64<NT>(B, B.order[idx], sm, st, red);
  }
}

// Two call sites, so that in the shared-memory one (the common case) every
// vector pointer is known to address shared memory: 32-bit shared loads and
// stores, and half the registers per pointer.
template <class V, int NT>
__global__ void __launch_bounds__(NT, batch_min_blocks<V, NT>()) k_batch(BatchData<V> B) {
  extern __shared__ double sm_dyn[];
  __shared__ DevState st;
  __shared__ double red[(NT / 32) * 13];
  __shared__ int id_s;
  if (B.ws)
    batch_queue<V, NT>(B, B.ws + (long long)blockIdx.x * B.ws_stride, st, red, id_s);
  else
    batch_queue<V, NT>(B, sm_dyn, st, red, id_s);
}

// Host entry points of k_batch<V, NT>.  batch_inst.cu defines them and is
// compiled once per (V, NT), so that the eight instantiations of the solver
// compile in parallel; the host code (batch.cu) only calls these.
template <class V, int NT>
struct BatchLaunch {
  // allow smem bytes of dynamic shared memory; *occupancy = resident blocks per SM
  static cudaError_t prepare(size_t smem, int* occupancy);
  static cudaError_t launch(int grid, size_t smem, cudaStream_t stream, const BatchData<V>& B);
};

}  // namespace pdhcg
