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

// Compensated FP32 storage on the mixed paths (the iterates, their running
// averages and restart points): the value is hi + lo, the products read hi,
// and lo keeps the rounding error of every update (two-sum, then the pair
// renormalised so that |lo| <= ulp(hi)/2).  Without it a step below half an
// ulp of hi is lost.  Every operation runs on the FP32 pipe.
__device__ __forceinline__ void split_add(float& hi, float& lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float t = __fadd_rn(lo, e);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

constexpr int kCgAdaptive = 0;
constexpr int kCgFixed = 1;
constexpr int kRestartAdaptive = 0;
constexpr int kStepFixed = 0;
constexpr int kStepAdaptive = 1;
// Exponents of PDLP's step update, which the Section 4 adaptive step rule
// builds on: the next eta is min((1 - (a+1)^-0.3) L, (1 + (a+1)^-0.6) eta).
constexpr double kStepReductionExp = 0.3;
constexpr double kStepGrowthExp = 0.6;

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
  int step_mode;
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
  // adaptive step size: attempts so far (= k_total with the fixed step), the
  // sum of the epoch's accepted etas, the averaging weight eta/sum of the
  // step just accepted, the CG precision of the pending attempt, and whether
  // the last attempt was accepted
  long long attempts;
  double weight_sum, avg_w, eps_try;
  int accepted;
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

// Variable bounds (+-inf where absent): the reduced cost of gradient entry g
// (g with both bounds finite, max(g, 0) with only a lower one, min(g, 0) with
// only an upper one, 0 with none) and its term lo lambda^+ - hi lambda^- of
// the dual objective.
template <class T>
__device__ __forceinline__ T reduced_cost(T g, T lo, T hi) {
  const bool lf = lo > -CUDART_INF_F, hf = hi < CUDART_INF_F;
  return lf ? (hf ? g : (g > T(0) ? g : T(0))) : (hf ? (g < T(0) ? g : T(0)) : T(0));
}

template <class T>
__device__ __forceinline__ T bound_term(T lam, T lo, T hi) {
  return lam > T(0) ? lam * lo : (lam < T(0) ? -lam * -hi : T(0));
}

// lb = lo'lambda^+ - hi'lambda^-, the variable bounds' share of the dual
// objective (0 without bounds): dual objective -1/2 x'Qx - b'y + lb.
__device__ __forceinline__ KktTerms kkt_from(double maxviol, double maxAx, double maxb,
                                             double maxdres, double maxQx, double maxAty,
                                             double maxc, double xQx, double cx, double by,
                                             double lb = 0.0) {
  KktTerms k;
  k.t[0] = maxviol / (1.0 + fmax(maxAx, maxb));
  k.t[1] = maxdres / (1.0 + fmax(maxQx, fmax(maxAty, maxc)));
  const double pobj = 0.5 * xQx + cx;
  const double dobj = -0.5 * xQx - by + lb;
  k.t[2] = fabs(xQx + cx + by - lb) / (1.0 + fmax(fabs(pobj), fabs(dobj)));
  // relKKT = max of the three; a NaN anywhere must stay visible.
  double m = fmax(k.t[0], fmax(k.t[1], k.t[2]));
  if (isnan(k.t[0]) || isnan(k.t[1]) || isnan(k.t[2])) m = CUDART_NAN;
  k.t[3] = m;
  k.t[4] = pobj;
  k.t[5] = dobj;
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
  if (st->attempts >= st->opt.max_iter) st->done = kDoneIterLimit;
}

// Adaptive step size (Section 4), after an attempt with step eta from z to
// the trial z': dx2 = ||dx||^2, dxqdx = dx'Q dx, dy2 = ||dy||^2 and cross =
// dy'A dx.  L = (omega dx2 + dy2/omega) / (2|cross| + dxqdx) (infinite when
// the denominator is 0); the attempt is accepted when eta <= L; the next eta
// is min((1 - (a+1)^-0.3) L, (1 + (a+1)^-0.6) eta) with a = st->attempts (this
// attempt included).  On acceptance the iteration counters advance, the CG
// precision of the attempt is kept and the averaging weight eta / (sum of
// the epoch's accepted etas) is set.  Shared by the single-QP step kernel
// and the batched solver.
//
// pow_table (may be null): pow_table[2 a] = (a+1)^-0.3 and pow_table[2 a + 1]
// = (a+1)^-0.6 for a < kStepPowTable, filled with step_pow_entry (the same
// pow calls), so that the thread deciding (alone on its SM, on B300's narrow
// FP64 pipe) reads them instead of evaluating two FP64 powers.
constexpr int kStepPowTable = 1 << 17;

// Entry a of the table (the same pow calls step_decide makes without it).
__device__ __forceinline__ void step_pow_entry(double* t, long long a) {
  const double a1 = (double)(a + 1);
  t[2 * a] = pow(a1, -kStepReductionExp);
  t[2 * a + 1] = pow(a1, -kStepGrowthExp);
}

__device__ inline void step_decide(DevState* st, double dx2, double dxqdx, double dy2,
                                   double cross, const double* pow_table = nullptr) {
  const double eta = st->eta, om = st->omega;
  const double movement = om * dx2 + dy2 / om;
  const double interaction = 2.0 * fabs(cross) + dxqdx;
  const double lim = interaction > 0.0 ? movement / interaction : CUDART_INF;
  const long long a = st->attempts;
  const double a1 = (double)(a + 1);
  const bool tab = pow_table != nullptr && a >= 0 && a < kStepPowTable;
  const double pr = tab ? pow_table[2 * a] : pow(a1, -kStepReductionExp);
  const double pg = tab ? pow_table[2 * a + 1] : pow(a1, -kStepGrowthExp);
  const double next = fmin((1.0 - pr) * lim, (1.0 + pg) * eta);
  const bool acc = eta <= lim;
  st->accepted = acc ? 1 : 0;
  st->eta = next;
  st->tau = next / om;
  st->sigma = next * om;
  if (acc) {
    st->eps = st->eps_try;
    st->j += 1;
    st->k_total += 1;
    st->weight_sum += eta;
    st->avg_w = eta / st->weight_sum;
  }
}

// step_decide with FP32 arithmetic, for the mixed batched solve, whose
// deciding thread would otherwise spend microseconds per attempt in FP64
// divisions on B300's narrow FP64 pipe while its block waits: the same rule
// and the same state updates, the sums and the limit in FP32, the epoch's
// weight sum kept in FP64.
__device__ inline void step_decide_f(DevState* st, float dx2, float dxqdx, float dy2, float cross,
                                     const double* pow_table) {
  const float eta = float(st->eta), om = float(st->omega);
  const float movement = om * dx2 + dy2 / om;
  const float interaction = 2.f * fabsf(cross) + dxqdx;
  const float lim = interaction > 0.f ? movement / interaction : CUDART_INF_F;
  const long long a = st->attempts;
  float pr, pg;
  if (pow_table != nullptr && a >= 0 && a < kStepPowTable) {
    pr = float(pow_table[2 * a]);
    pg = float(pow_table[2 * a + 1]);
  } else {
    pr = powf(float(a + 1), -float(kStepReductionExp));
    pg = powf(float(a + 1), -float(kStepGrowthExp));
  }
  const float next = fminf((1.f - pr) * lim, (1.f + pg) * eta);
  const bool acc = eta <= lim;
  st->accepted = acc ? 1 : 0;
  st->eta = next;
  st->tau = next / om;
  st->sigma = next * om;
  if (acc) {
    st->eps = st->eps_try;
    st->j += 1;
    st->k_total += 1;
    st->weight_sum += eta;
    st->avg_w = eta / float(st->weight_sum);
  }
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
  st->weight_sum = 0.0;
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
    st->attempts = 0;
    st->weight_sum = 0.0;
    st->avg_w = 1.0;
    st->eps_try = 0.0;
    st->accepted = 1;
  }
  st->done = 0;
  st->err = 0;
}

}  // namespace pdhcg
