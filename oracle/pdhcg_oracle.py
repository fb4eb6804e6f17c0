"""Plain FP64 CPU oracle of restarted PDHCG (Huang et al., arXiv 2405.16160).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
statement of what the CUDA solver computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA library: it receives plain numpy arrays and follows the paper's
steps in the paper's order, using numpy / scipy.sparse primitives
(CSR mat-vec, dot, norms) as the only building blocks.

Problem (paper Eq. (1)):   min 1/2 x'Qx + c'x   s.t.  Ax <= b,  Q PSD.
Saddle form (paper Eq. (2)): L(x, y) = 1/2 x'Qx + c'x + y'Ax - b'y, y >= 0.
The first ``m_eq`` rows are equalities G x = q (Section 4, augmented-penalty
paragraph) whose multipliers are free.

Readings of the paper taken here (each is a documented choice; the CUDA
path implements the same one):

* Dual step sign (Algorithm 1, y-update).  Eq. (2) and the KKT measure of
  Section 4 fix the convention Ax <= b, y >= 0, so the projected ascent step
  is y+ = proj(y + sigma (A(2x+ - x) - b)); the primal subproblem of
  Algorithm 1 is (Q + I/tau) x = x^k/tau - c - A'y^k.
* Averages (Algorithm 1 with beta_k = k, Lemma A.1(2)): uniform mean of the
  iterates x^{n,1..k}, y^{n,1..k} of the current epoch.
* Adaptive CG stop (Section 4, BB/CG paragraph): epsilon_0 = 0 and
  epsilon_{k+1} = epsilon_k + 0.05 relKKT(z^{n,k}), with relKKT(z^{n,k}) the
  most recent evaluated relKKT of the current iterate; CG (at least one step)
  stops when tau ||r_l||_2 <= epsilon, which implies the Section 2 criterion
  ||x_l - x_*|| <= epsilon because lambda_min(Q + I/tau) >= 1/tau; or at
  ``cg_max`` steps.  Fixed-N mode (PDHCG-fixed, Section 2) runs exactly N.
* Restart (Section 4 "Adaptive restart", the three tests of the cited
  rAPDHG Section 6 with beta_suff=0.2, beta_nec=0.8, beta_art=0.2): every
  ``eval_freq`` iterations the candidate is whichever of the current iterate
  and the average has the lower relKKT; restart to it if
  (i) relKKT(cand) <= beta_suff relKKT(z^{n,0}), or
  (ii) relKKT(cand) <= beta_nec relKKT(z^{n,0}) and relKKT(cand) exceeds the
       candidate's relKKT at the previous evaluation of the epoch, or
  (iii) the epoch length is >= beta_art times the total iteration count.
* Primal weight (Section 4): omega <- exp(theta log(dy/dx) + (1-theta) log
  omega) when both distances exceed eps_zero (the printed formula lacks the
  log on omega); tau = eta/omega, sigma = eta*omega.
* Step size (Section 3.2): eta = 1/(2 ||A||_2), ||A||_2 from 30 power
  iterations on A'A from the normalised all-ones vector.  If ||A||_2 is not
  above eps_zero (no coupling), ||A||_2 is replaced by eps_zero.
* omega_0 = ||c||_2 / ||b||_2 when both exceed eps_zero, else 1; x0 = y0 = 0.
* Adaptive step size (Section 4, optional ``step_mode = STEP_ADAPTIVE``).  The
  paper prints only the bound eta <= ||dz||_w^2 / (2 dx'A'dy + dx'Q dx) and
  says the rule follows PDLP.  Reading: one *attempt* runs the whole
  iteration (CG x-step, dual step) with the current eta into a trial point
  z' = (x', y'); with dz = z' - z and the primal-weighted norm
  ||dz||_w^2 = omega ||dx||^2 + ||dy||^2 / omega (the weighting that tau =
  eta/omega, sigma = eta*omega imply), the limit is
  L = ||dz||_w^2 / (2 |dy'A dx| + dx'Q dx) (infinite when the denominator is
  0; the absolute value makes it a bound for either sign of the coupling).
  The attempt is accepted when eta <= L; either way the next eta is PDLP's
  min((1 - (a+1)^-0.3) L, (1 + (a+1)^-0.6) eta), a = attempts so far.  A
  rejected attempt leaves z unchanged.  The averages of the epoch are then
  step-weighted, sum eta_k z_k / sum eta_k (they are the uniform mean when
  eta is fixed); the CG precision epsilon advances once per accepted
  iteration; eval_freq and max_iter count attempts (they equal iterations
  with the fixed step).
* Theoretical CG precision (Section 3, eq. stop-criteria; ``cg_mode =
  CG_THEORY``, an option beside the practical Section 4 rule).  The appendix
  proofs update y first and pair z^k = (x^k, y^{k+1}), which in Algorithm 1's
  order (x first) is the iterate (x^k, y^k) itself.  So, per epoch:
  epsilon^1 = zeta ||y^ - y^{n,0}|| / (1 + tau ||Q||_2), with y^ the dual step
  from the restart point taken with x_bar = x^{n,0} (the proofs' y^1, which
  Algorithm 1's order only forms after the first x-step), and
  epsilon^k = epsilon^{k-1} + zeta ||z^{n,k-1} - z^{n,k-2}|| / (1 + tau ||Q||_2)
  for k >= 2.  zeta defaults to ||A||_2 / (4 K^2), the largest value the
  bound 2 zeta <= min{(1 - sqrt(sigma tau)||A||)/(2 sqrt(sigma tau) K^2),
  (1 - sqrt(sigma tau)||A||)/(2 tau K^2)} allows when sigma = tau =
  1/(2||A||_2), with K = eval_freq (restarts are decided every eval_freq
  iterations).  CG stops as in the adaptive rule: tau ||r||_2 <= epsilon^k
  after at least one step, or at cg_max.
* Variable bounds lo <= x <= hi (optional ``OracleProblem.lo/hi``, +-inf
  allowed).  Section 4 switches the primal subproblem to a Barzilai-Borwein
  projected gradient when box constraints are present: x_{l+1} =
  P(x_l - g_l/alpha_l) with alpha_l = s'w / s's (s the last step, w its
  gradient change), alpha_0 the exact steepest-descent step g'Mg / g'g,
  M = Q + I/tau, from the warm start x^{n,k}.  It stops when the step length
  ||x_{l+1} - x_l|| is at most the adaptive precision epsilon_k (the
  criterion the paper states for this switch), after at least one step, or
  at cg_max (FIXED: exactly N steps).  The iterates stay in the box (x^0 is
  the projection of 0).  The paper's relKKT has no bound terms; PDLP's
  reduced costs give them: with g = Qx + A'y + c, lambda_j = g_j where both
  bounds are finite, max(g_j, 0) with only a lower one, min(g_j, 0) with only
  an upper one, 0 with none; r_dual measures g - lambda, and the dual
  objective gains lo'lambda^+ - hi'lambda^- (without bounds both reduce to
  the definitions above).
* Augmented penalty (Section 4, optional ``penalty``).  With G x = q the
  equality rows, the objective gains rho/2 ||G x - q||^2, i.e. the iteration
  runs on Q + rho G'G and c - rho G'q (the constant is dropped), with
  rho = 0.1 ||Q||_2 / ||G'G||_2; both norms by 30 power iterations from the
  normalised all-ones vector (||G'G||_2 = ||G||_2^2).  No equality rows, or
  ||G'G||_2 <= eps_zero, gives rho = 0.  The penalty and its gradient vanish
  where G x = q, so the penalised problem has the same KKT points, and every
  relKKT (termination, restarts, the CG precision) is taken on the problem
  as given.  With ``scale`` the scaling is computed on the penalised K.
* Preprocessing (Section 4, optional ``scale``): D1 (constraints) and D2
  (variables) from 10 Ruiz equilibration steps and one Pock-Chambolle step
  (alpha = 1) on the symmetric K = [[Q, A'], [A, 0]]; the iteration runs on
  D2 Q D2, D1 A D2, D2 c, D1 b, and every relKKT (termination, restarts, the
  CG precision) is evaluated on the original problem at x = D2 x~, y = D1 y~.

Every function is pinned: tests/test_oracle_pins.py, and for the restart
decisions (``restart_test``, ``evaluate``), the primal-weight update inside
``restart_to`` and the omega_0 rule of ``initial_state``,
tests/test_oracle_restart_pins.py (a decision table and an evaluation
sequence worked by hand against the printed beta_sufficient = 0.2,
beta_necessary = 0.8, beta_artificial = 0.2, and hand-computed PWeight
updates with theta = 0.2 and eps_zero = 1e-10).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

CG_ADAPTIVE = 0
CG_FIXED = 1
CG_THEORY = 2  # the CG precision sequence of Section 3 (eq. stop-criteria)

RESTART_ADAPTIVE = 0
RESTART_FIXED = 1  # restart to the average every K iterations (Algorithm 1)
RESTART_NONE = 2

STEP_FIXED = 0
STEP_ADAPTIVE = 1

SOLVED = 0
ITER_LIMIT = 1
TIME_LIMIT = 2
NUMERICAL_ERROR = 3


class NumericalError(RuntimeError):
    pass


@dataclass
class OracleProblem:
    Q: sp.csr_matrix
    A: sp.csr_matrix
    c: np.ndarray
    b: np.ndarray
    m_eq: int = 0
    lo: np.ndarray | None = None  # variable bounds (+-inf allowed); None: unbounded
    hi: np.ndarray | None = None

    @property
    def has_bounds(self) -> bool:
        return self.lo is not None and (bool(np.any(np.isfinite(self.lo)))
                                        or bool(np.any(np.isfinite(self.hi))))

    @property
    def n(self) -> int:
        return self.Q.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[0]


def problem_from_csr(n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b):
    """Build the oracle's problem from raw CSR arrays (duplicates are summed)."""
    Q = sp.csr_matrix((np.asarray(Q_val, np.float64), np.asarray(Q_col), np.asarray(Q_rowptr)),
                      shape=(n, n))
    A = sp.csr_matrix((np.asarray(A_val, np.float64), np.asarray(A_col), np.asarray(A_rowptr)),
                      shape=(m, n))
    Q.sum_duplicates()
    A.sum_duplicates()
    return OracleProblem(Q, A, np.asarray(c, np.float64).copy(),
                         np.asarray(b, np.float64).copy(), int(m_eq))


def problem_from_instance(inst) -> OracleProblem:
    P = problem_from_csr(inst.n, inst.m, inst.m_eq, inst.Q_rowptr, inst.Q_col, inst.Q_val,
                         inst.A_rowptr, inst.A_col, inst.A_val, inst.c, inst.b)
    lo, hi = getattr(inst, "lo", None), getattr(inst, "hi", None)
    if lo is not None or hi is not None:
        P.lo = np.asarray(lo, np.float64).copy() if lo is not None else np.full(P.n, -np.inf)
        P.hi = np.asarray(hi, np.float64).copy() if hi is not None else np.full(P.n, np.inf)
    return P


def reduced_costs(P: OracleProblem, g: np.ndarray) -> np.ndarray:
    """Bound multipliers lambda for the gradient g = Qx + A'y + c (PDLP's reduced costs):
    g where both bounds are finite, max(g, 0) with only a lower bound, min(g, 0) with
    only an upper bound, 0 without bounds."""
    if not P.has_bounds:
        return np.zeros_like(g)
    lf, hf = np.isfinite(P.lo), np.isfinite(P.hi)
    lam = np.zeros_like(g)
    lam[lf & hf] = g[lf & hf]
    lam[lf & ~hf] = np.maximum(g[lf & ~hf], 0.0)
    lam[~lf & hf] = np.minimum(g[~lf & hf], 0.0)
    return lam


# --------------------------------------------------------------------------
# Progress metric: relative KKT error (Section 4, "Progress metric").
# --------------------------------------------------------------------------
@dataclass
class KKT:
    r_primal: float
    r_dual: float
    r_gap: float
    relkkt: float
    primal_obj: float
    dual_obj: float


def _inf_norm(v: np.ndarray) -> float:
    return float(np.max(np.abs(v))) if v.size else 0.0


def relkkt(P: OracleProblem, x: np.ndarray, y: np.ndarray) -> KKT:
    """r_primal, r_dual, r_gap and their maximum as defined in Section 4.

    r_primal = ||[Ax - b]^+||_inf / (1 + max(||Ax||_inf, ||b||_inf))
               (|Ax - b| on the equality rows)
    r_dual   = ||Qx + A'y + c||_inf / (1 + max(||Qx||_inf, ||A'y||_inf, ||c||_inf))
    r_gap    = |x'Qx + c'x + b'y| / (1 + max(|1/2 x'Qx + c'x|, |1/2 x'Qx + b'y|))

    With variable bounds, r_dual measures Qx + A'y + c - lambda (reduced_costs)
    and the dual objective gains lo'lambda^+ - hi'lambda^-.
    """
    Qx = P.Q @ x
    Ax = P.A @ x
    Aty = P.A.T @ y
    if P.has_bounds:
        g = Qx + Aty + P.c
        lam = reduced_costs(P, g)
        lp, lm = np.maximum(lam, 0.0), np.maximum(-lam, 0.0)
        lb = float(np.sum(P.lo[lp > 0] * lp[lp > 0]) - np.sum(P.hi[lm > 0] * lm[lm > 0]))
        viol = Ax - P.b
        viol[P.m_eq:] = np.maximum(viol[P.m_eq:], 0.0)
        viol[:P.m_eq] = np.abs(viol[:P.m_eq])
        r_primal = _inf_norm(viol) / (1.0 + max(_inf_norm(Ax), _inf_norm(P.b)))
        r_dual = _inf_norm(g - lam) / (1.0 + max(_inf_norm(Qx), _inf_norm(Aty), _inf_norm(P.c)))
        xQx = float(x @ Qx)
        pobj = 0.5 * xQx + float(P.c @ x)
        dobj = -0.5 * xQx - float(P.b @ y) + lb
        r_gap = abs(pobj - dobj) / (1.0 + max(abs(pobj), abs(dobj)))
        return KKT(r_primal, r_dual, r_gap, max(r_primal, r_dual, r_gap), pobj, dobj)
    viol = Ax - P.b
    viol[P.m_eq:] = np.maximum(viol[P.m_eq:], 0.0)
    viol[:P.m_eq] = np.abs(viol[:P.m_eq])
    r_primal = _inf_norm(viol) / (1.0 + max(_inf_norm(Ax), _inf_norm(P.b)))
    r_dual = _inf_norm(Qx + Aty + P.c) / (
        1.0 + max(_inf_norm(Qx), _inf_norm(Aty), _inf_norm(P.c)))
    xQx = float(x @ Qx)
    cx = float(P.c @ x)
    by = float(P.b @ y)
    pobj = 0.5 * xQx + cx
    dobj = -0.5 * xQx - by
    r_gap = abs(xQx + cx + by) / (1.0 + max(abs(0.5 * xQx + cx), abs(0.5 * xQx + by)))
    return KKT(r_primal, r_dual, r_gap, max(r_primal, r_dual, r_gap), pobj, dobj)


# --------------------------------------------------------------------------
# Preprocessing (Section 4): diagonal scaling of K = [[Q, A'], [A, 0]].
# --------------------------------------------------------------------------
def _row_norms_K(P: OracleProblem, d1: np.ndarray, d2: np.ndarray, ord_inf: bool):
    """Row norms (inf or 1) of D K D, D = diag(d2, d1): variable rows then constraint rows."""
    Qs = sp.diags(d2) @ abs(P.Q) @ sp.diags(d2)
    As = sp.diags(d1) @ abs(P.A) @ sp.diags(d2)
    if ord_inf:
        rq = np.asarray(Qs.max(axis=1).todense()).ravel() if P.n else np.zeros(0)
        ra_col = np.asarray(As.max(axis=0).todense()).ravel() if P.m else np.zeros(P.n)
        ra_row = np.asarray(As.max(axis=1).todense()).ravel() if P.m else np.zeros(0)
        return np.maximum(rq, ra_col), ra_row
    rq = np.asarray(Qs.sum(axis=1)).ravel()
    ra_col = np.asarray(As.sum(axis=0)).ravel() if P.m else np.zeros(P.n)
    ra_row = np.asarray(As.sum(axis=1)).ravel() if P.m else np.zeros(0)
    return rq + ra_col, ra_row


def diagonal_scaling(P: OracleProblem, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """D1 (m), D2 (n): `ruiz_iters` Ruiz steps, then one Pock-Chambolle step.

    Ruiz step: every row k of the current D K D is divided, on both sides,
    by sqrt(||row_k||_inf).  Pock-Chambolle (alpha = 1): the same with the
    1-norm.  Rows that are entirely zero keep their scale.
    """
    d1, d2 = np.ones(P.m), np.ones(P.n)
    for it in range(ruiz_iters + (1 if pock_chambolle else 0)):
        rn, rm = _row_norms_K(P, d1, d2, ord_inf=it < ruiz_iters)
        d2 = d2 / np.sqrt(np.where(rn > 0.0, rn, 1.0))
        d1 = d1 / np.sqrt(np.where(rm > 0.0, rm, 1.0))
    return d1, d2


def scale_problem(P: OracleProblem, d1: np.ndarray, d2: np.ndarray) -> OracleProblem:
    Q = (sp.diags(d2) @ P.Q @ sp.diags(d2)).tocsr()
    A = (sp.diags(d1) @ P.A @ sp.diags(d2)).tocsr()
    lo = P.lo / d2 if P.lo is not None else None  # x~ = x / d2
    hi = P.hi / d2 if P.hi is not None else None
    return OracleProblem(Q, A, d2 * P.c, d1 * P.b, P.m_eq, lo, hi)


# --------------------------------------------------------------------------
# Setup: spectral norm and step size (Section 3.2: sigma = tau = 1/(2||A||)).
# --------------------------------------------------------------------------
def spectral_norm(A: sp.csr_matrix, iters: int = 30) -> float:
    """||A||_2 by power iteration on A'A, started at ones/sqrt(n).

    lambda_t = ||A'A v_{t-1}||_2, v_t = A'A v_{t-1} / lambda_t; returns sqrt(lambda_iters).
    """
    n = A.shape[1]
    if n == 0 or A.shape[0] == 0:
        return 0.0
    v = np.ones(n) / math.sqrt(n)
    lam = 0.0
    for _ in range(iters):
        w = A.T @ (A @ v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return math.sqrt(lam)


def symmetric_norm(Q: sp.csr_matrix, iters: int = 30) -> float:
    """||Q||_2 of a symmetric PSD Q by power iteration on Q, started at ones/sqrt(n):
    lambda_t = ||Q v_{t-1}||_2, v_t = Q v_{t-1} / lambda_t; returns lambda_iters."""
    n = Q.shape[0]
    if n == 0:
        return 0.0
    v = np.ones(n) / math.sqrt(n)
    lam = 0.0
    for _ in range(iters):
        w = Q @ v
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


# --------------------------------------------------------------------------
# Augmented penalty (Section 4): rho/2 ||G x - q||^2 on the equality rows.
# --------------------------------------------------------------------------
def penalty_rho(P: OracleProblem, iters: int = 30, eps_zero: float = 1e-10) -> float:
    """rho = 0.1 ||Q||_2 / ||G'G||_2 with G the equality rows (0 without them)."""
    if P.m_eq == 0:
        return 0.0
    g2 = spectral_norm(P.A[:P.m_eq], iters) ** 2
    return 0.1 * symmetric_norm(P.Q, iters) / g2 if g2 > eps_zero else 0.0


def penalize(P: OracleProblem, rho: float) -> OracleProblem:
    """The problem with rho/2 ||G x - q||^2 added: Q + rho G'G, c - rho G'q."""
    if rho == 0.0 or P.m_eq == 0:
        return P
    G = P.A[:P.m_eq]
    Qp = (P.Q + rho * (G.T @ G)).tocsr()
    Qp.sum_duplicates()
    return OracleProblem(Qp, P.A, P.c - rho * (G.T @ P.b[:P.m_eq]), P.b, P.m_eq, P.lo, P.hi)


# --------------------------------------------------------------------------
# Inexact primal solve: CG on (Q + I/tau) x = rhs (Section 2).
# --------------------------------------------------------------------------
def cg(Q: sp.csr_matrix, tau: float, rhs: np.ndarray, x0: np.ndarray, mode: int,
       n_fixed: int = 0, eps: float = 0.0, cg_max: int = 100, history: list | None = None):
    """Textbook conjugate gradients on the SPD system (Q + I/tau) x = rhs, from x0.

    FIXED: exactly ``n_fixed`` steps.  ADAPTIVE: at least one step, stop when
    tau*||r||_2 <= eps or after cg_max steps.  Either mode stops early when the
    residual is exactly zero.  Returns (x, steps).
    """
    x = x0.copy()
    if mode == CG_FIXED and n_fixed <= 0:
        return x, 0
    r = rhs - (Q @ x + x / tau)
    rr = float(r @ r)
    if history is not None:
        history.append(x.copy())
    if rr == 0.0:
        return x, 0
    p = r.copy()
    steps = 0
    while True:
        q = Q @ p + p / tau
        pq = float(p @ q)
        if not pq > 0.0:
            raise NumericalError("p'(Q + I/tau)p <= 0: Q is not PSD or the data is not finite")
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        steps += 1
        if history is not None:
            history.append(x.copy())
        if mode == CG_FIXED:
            stop = steps >= n_fixed
        else:  # CG_ADAPTIVE and CG_THEORY: the precision epsilon of the caller
            stop = tau * math.sqrt(rr_new) <= eps or steps >= cg_max
        if stop or rr_new == 0.0:
            return x, steps
        p = r + (rr_new / rr) * p
        rr = rr_new


def bb(Q: sp.csr_matrix, tau: float, rhs: np.ndarray, x0: np.ndarray, lo: np.ndarray,
       hi: np.ndarray, mode: int, n_fixed: int = 0, eps: float = 0.0, bb_max: int = 100):
    """Projected Barzilai-Borwein gradient method (Section 4) on
    min_{lo <= x <= hi} 1/2 x'(Q + I/tau)x - rhs'x from x0 (in the box).

    g = M x - rhs, alpha_0 = g'Mg / g'g; then x+ = P(x - g/alpha), s = x+ - x,
    g += M s, alpha = s'Ms / s's.  FIXED: exactly n_fixed steps; otherwise at
    least one step and stop when ||s|| <= eps or after bb_max steps (or when s
    is exactly zero).  Returns (x, steps).
    """
    M = lambda v: Q @ v + v / tau
    x = x0.copy()
    if mode == CG_FIXED and n_fixed <= 0:
        return x, 0
    g = M(x) - rhs
    gg = float(g @ g)
    if gg == 0.0:
        return x, 0
    gmg = float(g @ M(g))
    if not gmg > 0.0:
        raise NumericalError("g'(Q + I/tau)g <= 0: Q is not PSD or the data is not finite")
    alpha = gmg / gg
    steps = 0
    while True:
        xn = np.minimum(np.maximum(x - g / alpha, lo), hi)
        s = xn - x
        ss = float(s @ s)
        w = M(s)
        x = xn
        steps += 1
        if mode == CG_FIXED:
            stop = steps >= n_fixed
        else:
            stop = math.sqrt(ss) <= eps or steps >= bb_max
        if stop or ss == 0.0:
            return x, steps
        sw = float(s @ w)
        if not sw > 0.0:
            raise NumericalError("s'(Q + I/tau)s <= 0: Q is not PSD or the data is not finite")
        g = g + w
        alpha = sw / ss


# --------------------------------------------------------------------------
# Solver state and one inner iteration (Algorithm 1 loop body).
# --------------------------------------------------------------------------
@dataclass
class OracleOptions:
    tol: float = 1e-4
    max_iter: int = 100_000
    time_limit: float = math.inf
    eval_freq: int = 64
    cg_mode: int = CG_ADAPTIVE
    cg_fixed_n: int = 5
    cg_max: int = 100
    cg_eps_factor: float = 0.05
    restart_mode: int = RESTART_ADAPTIVE
    restart_k: int = 64  # restart frequency K for RESTART_FIXED
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.2
    theta_pw: float = 0.2
    eps_zero: float = 1e-10
    primal_weight_update: bool = True
    power_iters: int = 30
    omega0: float = 0.0  # <= 0: ||c||/||b|| rule
    eta: float = 0.0  # <= 0: 1/(2||A||)
    scale: bool = False  # Section 4 preprocessing (Ruiz x10 + Pock-Chambolle)
    step_mode: int = STEP_FIXED  # STEP_ADAPTIVE: the Section 4 adaptive step size
    cg_zeta: float = 0.0  # CG_THEORY: zeta (<= 0: ||A||_2 / (4 eval_freq^2))
    penalty: bool = False  # Section 4 augmented penalty rho/2 ||Gx - q||^2 on the equality rows
    step_reduction_exp: float = 0.3
    step_growth_exp: float = 0.6


@dataclass
class OracleState:
    x: np.ndarray
    y: np.ndarray
    x_avg: np.ndarray
    y_avg: np.ndarray
    x_anchor: np.ndarray
    y_anchor: np.ndarray
    eta: float
    omega: float
    eps: float = 0.0  # adaptive CG precision epsilon_k
    j: int = 0  # iterates averaged in this epoch
    k_total: int = 0
    relkkt_last: float = math.inf  # latest evaluated relKKT of the current iterate
    kkt_anchor: float = math.inf  # relKKT of the epoch's restart point
    kkt_prev_cand: float = math.inf  # candidate relKKT at the previous evaluation
    n_restarts: int = 0
    cg_total: int = 0
    last_cg_steps: int = 0
    attempts: int = 0  # steps tried (= k_total with the fixed step)
    weight_sum: float = 0.0  # sum of the accepted steps' eta in this epoch
    last_accepted: bool = True
    # CG_THEORY: zeta, ||Q||_2 and the iterate before the last accepted step
    zeta: float = 0.0
    norm_Q: float = 0.0
    x_prev: np.ndarray | None = None
    y_prev: np.ndarray | None = None

    @property
    def tau(self) -> float:
        return self.eta / self.omega

    @property
    def sigma(self) -> float:
        return self.eta * self.omega

    def copy(self) -> "OracleState":
        return OracleState(**{k: (v.copy() if isinstance(v, np.ndarray) else v)
                              for k, v in self.__dict__.items()})


def initial_state(P: OracleProblem, o: OracleOptions) -> OracleState:
    """x0 = y0 = 0, eta = 1/(2||A||_2), omega0 = ||c||/||b||."""
    normA = spectral_norm(P.A, o.power_iters)
    eta = o.eta if o.eta > 0 else 1.0 / (2.0 * max(normA, o.eps_zero))
    if o.omega0 > 0:
        omega = o.omega0
    else:
        nc, nb = float(np.linalg.norm(P.c)), float(np.linalg.norm(P.b))
        omega = nc / nb if (nc > o.eps_zero and nb > o.eps_zero) else 1.0
    z = lambda k: np.zeros(k)
    st = OracleState(z(P.n), z(P.m), z(P.n), z(P.m), z(P.n), z(P.m), eta, omega)
    if P.has_bounds:  # x0: the projection of 0 onto the box
        st.x = np.minimum(np.maximum(st.x, P.lo), P.hi)
        st.x_anchor = st.x.copy()
    if o.cg_mode == CG_THEORY:
        st.zeta = o.cg_zeta if o.cg_zeta > 0 else normA / (4.0 * o.eval_freq ** 2)
        st.norm_Q = symmetric_norm(P.Q, o.power_iters)
    return st


def theory_precision(P: OracleProblem, st: OracleState) -> float:
    """epsilon^k of Section 3 (eq. stop-criteria) for the next iteration of the epoch."""
    scale = st.zeta / (1.0 + st.tau * st.norm_Q)
    if st.j == 0:
        # the proofs' y^1: the dual step from the restart point with x_bar = x^{n,0}
        y_hat = st.y + st.sigma * (P.A @ st.x - P.b)
        y_hat[P.m_eq:] = np.maximum(y_hat[P.m_eq:], 0.0)
        return scale * float(np.linalg.norm(y_hat - st.y))
    d2 = float(np.sum((st.x - st.x_prev) ** 2) + np.sum((st.y - st.y_prev) ** 2))
    return st.eps + scale * math.sqrt(d2)


def step_limit(P: OracleProblem, x: np.ndarray, y: np.ndarray, x_new: np.ndarray,
               y_new: np.ndarray, omega: float) -> float:
    """Section 4 adaptive step-size bound for the trial step z -> z':

    ||dz||_w^2 / (2 |dy' A dx| + dx' Q dx), ||dz||_w^2 = omega ||dx||^2 + ||dy||^2 / omega;
    infinite when the denominator is zero.
    """
    dx, dy = x_new - x, y_new - y
    movement = omega * float(dx @ dx) + float(dy @ dy) / omega
    interaction = 2.0 * abs(float(dy @ (P.A @ dx))) + float(dx @ (P.Q @ dx))
    return movement / interaction if interaction > 0.0 else math.inf


def next_step_size(eta: float, limit: float, attempts: int, o: OracleOptions) -> float:
    """PDLP's step update after an attempt: min((1-(a+1)^-0.3) L, (1+(a+1)^-0.6) eta)."""
    a1 = float(attempts + 1)
    return min((1.0 - a1 ** -o.step_reduction_exp) * limit, (1.0 + a1 ** -o.step_growth_exp) * eta)


def pdhcg_step(P: OracleProblem, st: OracleState, o: OracleOptions, eps: float):
    """The Algorithm 1 loop body from z = (x, y) with the current eta: returns (x', y', CG steps)."""
    tau, sigma = st.tau, st.sigma
    # x^{k+1} ~ argmin_x L(x, y^k) + ||x - x^k||^2/(2 tau):  (Q + I/tau) x = x^k/tau - c - A'y^k
    rhs = st.x / tau - P.c - P.A.T @ st.y
    if P.has_bounds:  # Section 4: BB projected gradient when box constraints are present
        x_new, steps = bb(P.Q, tau, rhs, st.x, P.lo, P.hi, o.cg_mode, o.cg_fixed_n, eps, o.cg_max)
    else:
        x_new, steps = cg(P.Q, tau, rhs, st.x, o.cg_mode, o.cg_fixed_n, eps, o.cg_max)
    # y^{k+1} = proj(y^k + sigma (A(2x^{k+1} - x^k) - b)); equality rows unprojected
    y_new = st.y + sigma * (P.A @ (2.0 * x_new - st.x) - P.b)
    y_new[P.m_eq:] = np.maximum(y_new[P.m_eq:], 0.0)
    return x_new, y_new, steps


def inner_step(P: OracleProblem, st: OracleState, o: OracleOptions) -> None:
    """One attempt of a PDHCG iteration z^{n,k} -> z^{n,k+1} (Algorithm 1 loop body), in place.

    Fixed step: always accepted.  Adaptive step (Section 4): accepted when
    eta <= step_limit, and eta moves to next_step_size either way.
    """
    # epsilon_{k+1} = epsilon_k + 0.05 relKKT(z^{n,k})   (Section 4), or Section 3's sequence
    if o.cg_mode == CG_ADAPTIVE:
        eps = st.eps + o.cg_eps_factor * st.relkkt_last
    elif o.cg_mode == CG_THEORY:
        eps = theory_precision(P, st)
    else:
        eps = st.eps
    x_new, y_new, steps = pdhcg_step(P, st, o, eps)
    st.attempts += 1
    st.cg_total += steps
    st.last_cg_steps = steps
    eta = st.eta
    if o.step_mode == STEP_ADAPTIVE:
        limit = step_limit(P, st.x, st.y, x_new, y_new, st.omega)
        st.eta = next_step_size(eta, limit, st.attempts, o)
        st.last_accepted = eta <= limit
        if not st.last_accepted:
            return
    st.eps = eps
    st.j += 1
    if o.step_mode == STEP_ADAPTIVE:
        # step-weighted averages: sum eta_k z_k / sum eta_k over the epoch
        st.weight_sum += eta
        w = eta / st.weight_sum
        st.x_avg = st.x_avg + w * (x_new - st.x_avg)
        st.y_avg = st.y_avg + w * (y_new - st.y_avg)
    else:
        # running averages with beta = j (uniform mean of the epoch's iterates)
        st.x_avg = st.x_avg + (x_new - st.x_avg) / st.j
        st.y_avg = st.y_avg + (y_new - st.y_avg) / st.j
    st.x_prev, st.y_prev = st.x, st.y
    st.x, st.y = x_new, y_new
    st.k_total += 1


def restart_to(P: OracleProblem, st: OracleState, o: OracleOptions, use_avg: bool,
               kkt_cand: float) -> None:
    """Start a new epoch at the candidate; update the primal weight (Section 4)."""
    xc = st.x_avg.copy() if use_avg else st.x.copy()
    yc = st.y_avg.copy() if use_avg else st.y.copy()
    if o.primal_weight_update:
        dx = float(np.linalg.norm(xc - st.x_anchor))
        dy = float(np.linalg.norm(yc - st.y_anchor))
        if dx > o.eps_zero and dy > o.eps_zero:
            st.omega = math.exp(o.theta_pw * math.log(dy / dx)
                                + (1.0 - o.theta_pw) * math.log(st.omega))
    st.x, st.y = xc, yc
    st.x_anchor, st.y_anchor = xc.copy(), yc.copy()
    st.j = 0
    st.weight_sum = 0.0
    st.eps = 0.0
    st.kkt_anchor = kkt_cand
    st.kkt_prev_cand = math.inf
    st.relkkt_last = kkt_cand
    st.n_restarts += 1


def restart_test(kkt_cand: float, st: OracleState, o: OracleOptions) -> bool:
    """The three restart conditions (sufficient, necessary+stall, artificial)."""
    if kkt_cand <= o.beta_suff * st.kkt_anchor:
        return True
    if kkt_cand <= o.beta_nec * st.kkt_anchor and kkt_cand > st.kkt_prev_cand:
        return True
    return st.j >= o.beta_art * st.k_total


@dataclass
class OracleResult:
    x: np.ndarray
    y: np.ndarray
    termination: int
    kkt: KKT
    iterations: int
    cg_steps: int
    restarts: int
    returned_avg: bool
    state: OracleState
    trace: list = field(default_factory=list)
    seconds: float = 0.0


def evaluate(P: OracleProblem, st: OracleState, o: OracleOptions, record: list,
             kkt=None) -> tuple:
    """relKKT of the current iterate and of the average, then the restart logic.

    ``kkt(x, y)`` scores an iterate (default: relkkt on P).  Returns
    (done, kkt, use_avg) where done is True when relKKT <= tol.
    """
    kkt = kkt or (lambda x, y: relkkt(P, x, y))
    kc = kkt(st.x, st.y)
    ka = kkt(st.x_avg, st.y_avg) if st.j > 0 else None
    rec = {"k": st.k_total, "kkt_cur": kc.relkkt, "kkt_avg": ka.relkkt if ka else None,
           "restart": False, "cand_avg": False, "omega": st.omega}
    record.append(rec)
    best_avg = ka is not None and ka.relkkt <= kc.relkkt
    best = ka if best_avg else kc
    if best.relkkt <= o.tol:
        return True, best, best_avg
    st.relkkt_last = kc.relkkt
    if o.restart_mode == RESTART_ADAPTIVE and ka is not None:
        if restart_test(best.relkkt, st, o):
            restart_to(P, st, o, best_avg, best.relkkt)
            rec["restart"], rec["cand_avg"] = True, best_avg
        else:
            st.kkt_prev_cand = best.relkkt
    return False, best, best_avg


def solve(P: OracleProblem, o: OracleOptions | None = None,
          state: OracleState | None = None, step_hook=None) -> OracleResult:
    """Restarted PDHCG (Algorithm 1 with the Section 4 heuristics).

    With ``o.penalty`` the iteration runs on the penalised problem; with
    ``o.scale`` on the scaled one (``state`` and ``step_hook`` then see scaled
    iterates).  relKKT is always taken on P at the unscaled iterate, and the
    returned x, y are unscaled.
    """
    o = o or OracleOptions()
    t0 = time.perf_counter()
    Pp = penalize(P, penalty_rho(P, o.power_iters, o.eps_zero)) if o.penalty else P
    if o.scale:
        d1, d2 = diagonal_scaling(Pp)
        Pi = scale_problem(Pp, d1, d2)
    else:
        d1, d2, Pi = np.ones(P.m), np.ones(P.n), Pp
    kkt = lambda x, y: relkkt(P, d2 * x, d1 * y)
    st = state.copy() if state is not None else initial_state(Pi, o)
    trace: list = []
    if state is None:
        k0 = kkt(st.x, st.y)
        trace.append({"k": 0, "kkt_cur": k0.relkkt, "kkt_avg": None, "restart": False,
                      "cand_avg": False, "omega": st.omega})
        st.relkkt_last = k0.relkkt
        st.kkt_anchor = k0.relkkt
        if k0.relkkt <= o.tol:
            return OracleResult(d2 * st.x, d1 * st.y, SOLVED, k0, 0, 0, 0, False, st, trace,
                                time.perf_counter() - t0)
    term = ITER_LIMIT
    best = None
    use_avg = False
    try:
        while st.attempts < o.max_iter:
            inner_step(Pi, st, o)
            if step_hook is not None:
                step_hook(st)
            if o.restart_mode == RESTART_FIXED and st.j >= o.restart_k:
                kc = kkt(st.x_avg, st.y_avg)
                restart_to(Pi, st, o, True, kc.relkkt)
            if st.attempts % o.eval_freq == 0:
                done, best, use_avg = evaluate(Pi, st, o, trace, kkt)
                if done:
                    term = SOLVED
                    break
            if time.perf_counter() - t0 > o.time_limit:
                term = TIME_LIMIT
                break
    except NumericalError:
        term = NUMERICAL_ERROR
    if term != SOLVED:
        kc = kkt(st.x, st.y)
        ka = kkt(st.x_avg, st.y_avg) if st.j > 0 else None
        use_avg = ka is not None and ka.relkkt <= kc.relkkt
        best = ka if use_avg else kc
    x = st.x_avg if use_avg else st.x
    y = st.y_avg if use_avg else st.y
    return OracleResult(d2 * x, d1 * y, term, best, st.k_total, st.cg_total, st.n_restarts,
                        use_avg, st, trace, time.perf_counter() - t0)
