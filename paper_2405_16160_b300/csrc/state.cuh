// Scalar state of a restarted-PDHCG solve and the decisions taken on it:
// the options, the step sizes and counters, the relKKT terms (Section 4
// progress metric), termination, the three restart tests, the primal-weight
// update and the step-size set-up (Section 3.2, Section 4).  Device-only
// inline code shared by the single-QP kernels and the batched solver, so
// both take exactly the same decisions.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace pdhcg {

constexpr int kCgAdaptive = 0;
constexpr int kCgFixed = 1;
constexpr int kRestartAdaptive = 0;

// done codes: 0 running, otherwise 1 + qp_termination
constexpr int kDoneSolved = 1;
constexpr int kDoneIterLimit = 2;
constexpr int kDoneNumerical = 4;

constexpr int kErrBarrierTimeout = 1;
constexpr unsigned kDebugBarrierNeverReleases = 1u;

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

__device__ __forceinline__ bool running(const DevState* st) { return st->done == 0 && st->err == 0; }

template <class T>
__device__ __forceinline__ T shfl_xor(T v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
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

// The scalar side of an evaluation (Section 4): record the relKKT terms of
// the current iterate (kc) and of the average (ka), then decide.  mode 0:
// evaluation at the starting point; 1: regular evaluation with termination
// and restart decisions; 2: evaluate only (no decisions).  Shared by the
// single-QP control kernel and the batched solver.
__device__ inline void control_decide(DevState* st, const KktTerms& kc, const KktTerms& ka,
                                      int mode) {
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

// Primal weight (Section 4): omega <- exp(theta log(dy/dx) + (1-theta) log omega),
// from the squared distances of the new restart point to the previous one;
// a new epoch starts.  Shared by the single-QP kernel below and the batched
// solver.
__device__ inline void restart_finish_decide(DevState* st, double dx2, double dy2) {
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

// eta = 1/(2||A||_2) (Section 3.2) with ||A||_2 = sqrt(st->lam) from the
// power iteration, omega0 = ||c||/||b|| (1 if either is ~0) from the squared
// norms s0 = ||c||^2, s1 = ||b||^2 (Section 4), tau = eta/omega, sigma =
// eta*omega.  reset != 0 also clears the counters.  Shared with the batched
// solver.
__device__ inline void setup_finish_decide(DevState* st, double s0, double s1, int reset) {
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
