"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each test fixes part of the oracle to something the paper or the mathematics
determines: hand-worked relKKT values (Section 4), closed-form QP solutions,
LAPACK solves, an exhaustive active-set search on tiny QPs, the textbook CG
error bound (Section 2), Lemma A.2(2) and Theorem 2 of the appendix, and the
trend of Table 2.  The last group plants mistakes in the oracle and checks
that a pin catches each one.  Variable bounds and the BB projected gradient
of Section 4 are pinned by a box brute force, the linear-system solution
without bounds, relKKT with bounds worked by hand, the box closed form and
brute force with the bounds written as rows.  The adaptive step size of Section 4 is pinned
by its closed form at the top singular pair of A, a lower bound that follows
from Cauchy-Schwarz and AM-GM, PDLP's update rule worked by hand, the
accept/reject invariants, step-weighted averages and the closed-form and
brute-force solutions reached with it.  The augmented penalty of Section 4
is pinned by the exact norms of a diagonal Q and a rank-one G'G, the
expansion of rho/2 ||Gx - q||^2, and the same closed-form and brute-force
solutions reached with it on.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import pdhcg_oracle as O


def _prob(Qd, Ad, c, b, m_eq=0):
    return O.OracleProblem(sp.csr_matrix(np.asarray(Qd, float)),
                           sp.csr_matrix(np.asarray(Ad, float).reshape(-1, len(c))),
                           np.asarray(c, float), np.asarray(b, float), m_eq)


def _rand_spd(rng, n, cond=10.0):
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (U * ev) @ U.T


def brute_force_qp(Qd, Ad, c, b, m_eq=0):
    """Exact solution of a tiny strictly convex QP by enumerating active sets.

    For each active set S containing the equality rows, solve the KKT system
    [[Q, A_S'], [A_S, 0]] [x; y_S] = [-c; b_S] and keep the one that is primal
    feasible with y_S >= 0 on its inequality rows.
    """
    n, m = len(c), len(b)
    ineq = list(range(m_eq, m))
    for size in range(0, min(n, m) - m_eq + 1):
        for act in itertools.combinations(ineq, size):
            S = list(range(m_eq)) + list(act)
            k = len(S)
            K = np.zeros((n + k, n + k))
            K[:n, :n] = Qd
            if k:
                K[:n, n:] = Ad[S].T
                K[n:, :n] = Ad[S]
            rhs = np.concatenate([-c, b[S]])
            try:
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                continue
            x, yS = sol[:n], sol[n:]
            if np.any(Ad @ x - b > 1e-9 * (1 + np.abs(b))) or (k and np.any(yS[m_eq:] < -1e-12)):
                continue
            if m_eq and np.any(np.abs(Ad[:m_eq] @ x - b[:m_eq]) > 1e-9):
                continue
            y = np.zeros(m)
            y[S] = yS
            return x, y
    raise AssertionError("no KKT point found")


# ---------------------------------------------------------------- relKKT
def test_relkkt_hand_worked(golden_dir):
    with open(os.path.join(golden_dir, "relkkt_hand.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        P = _prob(case["Q"], case["A"], case["c"], case["b"], case["m_eq"])
        k = O.relkkt(P, np.array(case["x"]), np.array(case["y"]))
        for key in ("r_primal", "r_dual", "r_gap", "relkkt"):
            assert getattr(k, key) == pytest.approx(case[key], rel=1e-15, abs=1e-16), (case["name"], key)


def test_relkkt_vanishes_at_closed_form_optimum():
    rng = np.random.default_rng(1)
    n = 30
    Qd = _rand_spd(rng, n, 50.0)
    c = rng.standard_normal(n)
    Ad = rng.standard_normal((5, n))
    b = np.full(5, 1e6)  # constraints far from active: x* = -Q^{-1}c, y* = 0
    x = -sla.cho_solve(sla.cho_factor(Qd), c)
    k = O.relkkt(_prob(Qd, Ad, c, b), x, np.zeros(5))
    assert k.relkkt < 1e-13
    assert k.primal_obj == pytest.approx(-0.5 * c @ sla.cho_solve(sla.cho_factor(Qd), c), rel=1e-12)


def test_relkkt_empty_constraints_and_gap_sign():
    P = _prob([[1.0]], np.zeros((0, 1)), [2.0], np.zeros(0))
    k = O.relkkt(P, np.array([-2.0]), np.zeros(0))
    assert k.r_primal == 0.0 and k.relkkt < 1e-15
    # the gap uses x'Qx + c'x + b'y: at y* = 0 and x* the dual objective equals the primal
    assert k.primal_obj == pytest.approx(k.dual_obj, rel=1e-15)


# ---------------------------------------------------------------- ||A||_2
def test_spectral_norm_rank_one_exact():
    rng = np.random.default_rng(2)
    u, v = rng.random(7) + 0.1, rng.random(11) + 0.1
    A = sp.csr_matrix(np.outer(u, v))
    assert O.spectral_norm(A, 30) == pytest.approx(np.linalg.norm(u) * np.linalg.norm(v), rel=1e-13)


def test_spectral_norm_close_to_svd_and_below_it():
    rng = np.random.default_rng(3)
    A = sp.random(120, 200, density=0.05, random_state=3, data_rvs=rng.standard_normal).tocsr()
    true = np.linalg.norm(A.toarray(), 2)
    est = O.spectral_norm(A, 30)
    assert est <= true * (1 + 1e-12)
    assert est >= 0.97 * true
    assert O.spectral_norm(A, 60) >= est * (1 - 1e-14)  # power-iteration estimates increase


# ---------------------------------------------------------------- CG (Section 2)
def test_cg_exact_in_n_steps_and_energy_bound():
    rng = np.random.default_rng(4)
    n, tau = 40, 0.7
    Qd = _rand_spd(rng, n, 30.0)
    Mfull = Qd + np.eye(n) / tau
    rhs = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    xs = sla.cho_solve(sla.cho_factor(Mfull), rhs)
    hist = []
    x, steps = O.cg(sp.csr_matrix(Qd), tau, rhs, x0, O.CG_FIXED, n_fixed=n, history=hist)
    assert steps == n
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    ev = np.linalg.eigvalsh(Mfull)
    kappa = ev[-1] / ev[0]
    r = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    en = lambda e: math.sqrt(e @ Mfull @ e)
    e0 = en(hist[0] - xs)
    for l, xl in enumerate(hist):
        assert en(xl - xs) <= 2 * r ** l * e0 * (1 + 1e-9) + 1e-12


def test_cg_adaptive_stop_guarantees_section2_criterion():
    rng = np.random.default_rng(5)
    n, tau = 60, 0.3
    Qd = _rand_spd(rng, n, 100.0)
    rhs = rng.standard_normal(n)
    xs = np.linalg.solve(Qd + np.eye(n) / tau, rhs)
    for eps in (1e-1, 1e-3, 1e-6):
        x, steps = O.cg(sp.csr_matrix(Qd), tau, rhs, np.zeros(n), O.CG_ADAPTIVE, eps=eps, cg_max=500)
        assert steps >= 1
        r = rhs - (Qd @ x + x / tau)
        assert tau * np.linalg.norm(r) <= eps
        assert np.linalg.norm(x - xs) <= eps  # ||x - x_*|| <= eps (Section 2)


def test_cg_cap_and_zero_residual():
    Qd = np.diag([1.0, 100.0, 1e4])
    rhs = np.array([1.0, 1.0, 1.0])
    _, steps = O.cg(sp.csr_matrix(Qd), 1.0, rhs, np.zeros(3), O.CG_ADAPTIVE, eps=0.0, cg_max=2)
    assert steps == 2
    xs = np.linalg.solve(Qd + np.eye(3), rhs)
    x, steps = O.cg(sp.csr_matrix(Qd), 1.0, rhs, xs, O.CG_ADAPTIVE, eps=0.0, cg_max=5)
    assert steps <= 5 and np.allclose(x, xs, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- full solver, closed forms
def _opts(**kw):
    o = O.OracleOptions(tol=1e-10, max_iter=200_000)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
def test_solver_unconstrained_m0(step):
    rng = np.random.default_rng(6)
    n = 25
    Qd = _rand_spd(rng, n, 20.0)
    c = rng.standard_normal(n)
    P = _prob(Qd, np.zeros((0, n)), c, np.zeros(0))
    res = O.solve(P, _opts(step_mode=step))
    assert res.termination == O.SOLVED
    xs = -np.linalg.solve(Qd, c)
    assert np.linalg.norm(res.x - xs) <= 1e-8 * (1 + np.linalg.norm(xs))


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
def test_solver_diagonal_box_closed_form(step):
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2
    lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    Ad = np.vstack([np.eye(n), -np.eye(n)])
    b = np.concatenate([hi, -lo])
    res = O.solve(_prob(np.diag(q), Ad, c, b), _opts(step_mode=step))
    assert res.termination == O.SOLVED
    xs = np.clip(-c / q, lo, hi)
    g = q * xs + c
    ys = np.concatenate([np.maximum(-g, 0) * (xs >= hi), np.maximum(g, 0) * (xs <= lo)])
    assert np.max(np.abs(res.x - xs)) <= 1e-8
    assert np.max(np.abs(res.y - ys)) <= 1e-7


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
@pytest.mark.parametrize("penalty", [False, True])
def test_solver_equality_hyperplane_closed_form(step, penalty):
    rng = np.random.default_rng(8)
    n = 30
    a = rng.standard_normal(n)
    c = rng.standard_normal(n)
    beta = 0.7
    res = O.solve(_prob(np.eye(n), a[None, :], c, [beta], m_eq=1),
                  _opts(step_mode=step, penalty=penalty))
    assert res.termination == O.SOLVED
    xs = -c + a * (beta + a @ c) / (a @ a)
    lam = -(beta + a @ c) / (a @ a)
    assert np.max(np.abs(res.x - xs)) <= 1e-8
    assert res.y[0] == pytest.approx(lam, abs=1e-7)


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
@pytest.mark.parametrize("seed,n,m,m_eq", [(10, 4, 6, 0), (11, 5, 8, 0), (12, 6, 7, 2), (13, 3, 8, 1)])
@pytest.mark.parametrize("penalty", [False, True])
def test_solver_matches_active_set_brute_force(seed, n, m, m_eq, step, penalty):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 3
    x0 = rng.standard_normal(n)
    b = Ad @ x0 + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    xs, ys = brute_force_qp(Qd, Ad, c, b, m_eq)
    res = O.solve(_prob(Qd, Ad, c, b, m_eq), _opts(step_mode=step, penalty=penalty))
    assert res.termination == O.SOLVED
    assert np.linalg.norm(res.x - xs) <= 1e-6 * (1 + np.linalg.norm(xs))
    fs = 0.5 * xs @ Qd @ xs + c @ xs
    assert res.kkt.primal_obj == pytest.approx(fs, rel=1e-8, abs=1e-8)


# ---------------------------------------------------------------- invariants
def test_dual_iterates_stay_nonnegative_on_inequality_rows():
    rng = np.random.default_rng(14)
    n, m, m_eq = 8, 10, 3
    Qd = _rand_spd(rng, n, 5.0)
    Ad = rng.standard_normal((m, n))
    b = Ad @ rng.standard_normal(n) + np.concatenate([np.zeros(m_eq), rng.uniform(0, 1, m - m_eq)])
    P = _prob(Qd, Ad, rng.standard_normal(n), b, m_eq)
    seen = []

    def hook(st):
        seen.append(st.y.copy())
        assert np.all(st.y[m_eq:] >= 0.0)
        assert np.all(st.y_avg[m_eq:] >= 0.0)

    O.solve(P, _opts(max_iter=500), step_hook=hook)
    assert any(np.any(y[:m_eq] < 0) for y in seen)  # equality multipliers are free


def test_lemma_a2_bounded_iterates_within_an_epoch():
    """Lemma A.2(2): ||z^k - z*||^2 <= 4 ||z^0 - z*||^2 with sigma = tau = 1/(2||A||)."""
    rng = np.random.default_rng(15)
    n, m = 6, 8
    Qd = _rand_spd(rng, n, 20.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 2
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 0.3, m)
    xs, ys = brute_force_qp(Qd, Ad, c, b)
    zs = np.concatenate([xs, ys])
    P = _prob(Qd, Ad, c, b)
    o = _opts(cg_mode=O.CG_FIXED, cg_fixed_n=n, restart_mode=O.RESTART_NONE, omega0=1.0,
              primal_weight_update=False, max_iter=400, tol=0.0)
    st0 = O.initial_state(P, o)
    st0.x, st0.y = rng.standard_normal(n), np.abs(rng.standard_normal(m))
    d0 = np.sum((np.concatenate([st0.x, st0.y]) - zs) ** 2)
    dists = []
    O.solve(P, o, state=st0,
            step_hook=lambda st: dists.append(np.sum((np.concatenate([st.x, st.y]) - zs) ** 2)))
    assert len(dists) == 400
    assert max(dists) <= 4.0 * d0
    assert dists[-1] < d0  # it also makes progress


def test_theorem2_fixed_restarts_contract():
    """Theorem 2: with exact CG, fixed K and restarts to the average the
    restart points approach the solution (checked loosely: distance shrinks
    by 10^3 and is never more than 1.5x the previous epoch's)."""
    rng = np.random.default_rng(16)
    n, m = 6, 8
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n)
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 0.3, m)
    xs, ys = brute_force_qp(Qd, Ad, c, b)
    zs = np.concatenate([xs, ys])
    P = _prob(Qd, Ad, c, b)
    o = _opts(cg_mode=O.CG_FIXED, cg_fixed_n=n, restart_mode=O.RESTART_FIXED, restart_k=50,
              omega0=1.0, primal_weight_update=False, max_iter=2000, tol=0.0, eval_freq=10**9)
    anchors = []

    def hook(st):
        if st.j == 50:
            anchors.append(np.linalg.norm(np.concatenate([st.x_avg, st.y_avg]) - zs))

    O.solve(P, o, step_hook=hook)
    d0 = np.linalg.norm(zs)
    assert anchors[-1] <= 1e-3 * d0
    for a, b_ in zip(anchors, anchors[1:]):
        assert b_ <= 1.5 * a + 1e-12


def test_table2_trend_cg_steps_grow_with_condition_number():
    """Table 2: CG steps per outer iteration grow with kappa(Q)."""
    from paper_2405_16160_b300 import workloads as W
    rng = np.random.default_rng(17)
    n, m = 60, 40
    Ad = W._bernoulli_normal(rng, m, n, 0.2)
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 1, m)
    c = rng.standard_normal(n)
    ratios = []
    for cond in (1.0, 1e2, 1e4):
        Qd = _rand_spd(np.random.default_rng(18), n, cond)
        res = O.solve(_prob(Qd, Ad, c, b), _opts(tol=1e-6, max_iter=20000))
        assert res.termination == O.SOLVED
        ratios.append(res.cg_steps / res.iterations)
    assert ratios[0] < ratios[1] < ratios[2]


# ---------------------------------------------------------------- planted mistakes
def _mutated_inner_step(kind):
    def step(P, st, o):
        tau, sigma = st.tau, st.sigma
        if o.cg_mode == O.CG_ADAPTIVE:
            st.eps = st.eps + o.cg_eps_factor * st.relkkt_last
        cterm = 0.0 if kind == "drop_c" else P.c
        rhs = st.x / tau - cterm - P.A.T @ st.y
        x_new, steps = O.cg(P.Q, tau, rhs, st.x, o.cg_mode, o.cg_fixed_n, st.eps, o.cg_max)
        sgn = -1.0 if kind == "dual_sign" else 1.0
        xbar = x_new if kind == "no_extrapolation" else 2.0 * x_new - st.x
        y_new = st.y + sgn * sigma * (P.A @ xbar - P.b)
        y_new[P.m_eq:] = np.maximum(y_new[P.m_eq:], 0.0)
        st.j += 1
        w = st.j if kind != "avg_weight" else st.j + 1
        st.x_avg = st.x_avg + (x_new - st.x_avg) / w
        st.y_avg = st.y_avg + (y_new - st.y_avg) / w
        st.x, st.y = x_new, y_new
        st.k_total += 1
        st.attempts += 1
        st.cg_total += steps
    return step


def _averages_match_epoch_means(P, o):
    """Lemma A.1(2): the averages are the plain means of the epoch's iterates."""
    xs_epoch, ys_epoch, worst = [], [], [0.0]

    def hook(st):
        if st.j == 1:
            xs_epoch.clear()
            ys_epoch.clear()
        xs_epoch.append(st.x.copy())
        ys_epoch.append(st.y.copy())
        assert len(xs_epoch) == st.j
        worst[0] = max(worst[0], np.max(np.abs(st.x_avg - np.mean(xs_epoch, axis=0))),
                       np.max(np.abs(st.y_avg - np.mean(ys_epoch, axis=0))))

    O.solve(P, o, step_hook=hook)
    return worst[0]


def _avg_problem():
    rng = np.random.default_rng(19)
    n, m = 8, 10
    Ad = rng.standard_normal((m, n))
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 1, m)
    return _prob(_rand_spd(rng, n, 5.0), Ad, rng.standard_normal(n), b, 2)


def test_averages_are_uniform_epoch_means():
    assert _averages_match_epoch_means(_avg_problem(), _opts(max_iter=700, eval_freq=16)) <= 1e-12


def test_planted_averaging_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(O, "inner_step", _mutated_inner_step("avg_weight"))
    assert _averages_match_epoch_means(_avg_problem(), _opts(max_iter=700, eval_freq=16)) > 1e-6


def _max_metric_increase(P, zs, n, iters=300):
    """Largest relative increase of ||z^k - z*||_M over the run, where
    M = [[I/tau, -A'], [-A, I/sigma]]: with exact primal solves, one PDHCG step
    (x first, y with the extrapolated 2x+ - x) is a proximal-point step in the
    M metric (the optimality conditions in the proof of Lemma A.1), so the
    distance to a saddle point never grows."""
    o = _opts(cg_mode=O.CG_FIXED, cg_fixed_n=n, restart_mode=O.RESTART_NONE, omega0=1.3,
              primal_weight_update=False, max_iter=iters, tol=0.0)
    st0 = O.initial_state(P, o)
    A = P.A.toarray()
    tau, sigma = st0.tau, st0.sigma

    def mnorm(x, y):
        dx, dy = x - zs[:n], y - zs[n:]
        return dx @ dx / tau + dy @ dy / sigma - 2 * dy @ (A @ dx)

    vals = [mnorm(st0.x, st0.y)]
    O.solve(P, o, state=st0, step_hook=lambda st: vals.append(mnorm(st.x, st.y)))
    return max((b_ - a) / vals[0] for a, b_ in zip(vals, vals[1:]))


def _fejer_problem():
    rng = np.random.default_rng(20)
    n, m = 6, 9
    Qd = _rand_spd(rng, n, 8.0) * 1e-2  # weakly convex: extrapolation matters
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 2
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 0.3, m)
    xs, ys = brute_force_qp(Qd, Ad, c, b)
    return _prob(Qd, Ad, c, b), np.concatenate([xs, ys]), n


def test_iterates_fejer_monotone_in_pdhg_metric():
    P, zs, n = _fejer_problem()
    assert _max_metric_increase(P, zs, n) <= 1e-12


def test_planted_extrapolation_mistake_is_caught(monkeypatch):
    P, zs, n = _fejer_problem()
    monkeypatch.setattr(O, "inner_step", _mutated_inner_step("no_extrapolation"))
    assert _max_metric_increase(P, zs, n) > 1e-6


@pytest.mark.parametrize("kind", ["drop_c", "dual_sign"])
def test_planted_mistakes_are_caught_by_box_pin(monkeypatch, kind):
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2
    lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    P = _prob(np.diag(q), np.vstack([np.eye(n), -np.eye(n)]), c, np.concatenate([hi, -lo]))
    xs = np.clip(-c / q, lo, hi)
    monkeypatch.setattr(O, "inner_step", _mutated_inner_step(kind))
    res = O.solve(P, _opts(max_iter=3000))
    ok = res.termination == O.SOLVED and np.max(np.abs(res.x - xs)) <= 1e-8
    assert not ok, f"planted mistake {kind} went unnoticed"


def test_planted_relkkt_mistake_is_caught(monkeypatch, golden_dir):
    with open(os.path.join(golden_dir, "relkkt_hand.json")) as f:
        case = json.load(f)["cases"][0]
    P = _prob(case["Q"], case["A"], case["c"], case["b"], case["m_eq"])
    real = O.relkkt

    def wrong(P_, x, y):  # gap numerator with 1/2 x'Qx instead of x'Qx
        k = real(P_, x, y)
        xQx = x @ (P_.Q @ x)
        k.r_gap = abs(0.5 * xQx + P_.c @ x + P_.b @ y) / (1 + max(abs(k.primal_obj), abs(k.dual_obj)))
        return k

    k = wrong(P, np.array(case["x"]), np.array(case["y"]))
    assert k.r_gap != pytest.approx(case["r_gap"], rel=1e-6)


# ---------------------------------------------------------------- preprocessing (Section 4)
def test_scaling_hand_worked():
    # K = [[0, 0, 3], [0, 0, 4], [3, 4, 0]]: Q = 0 (2 x 2), A = [[3, 4]]
    P = _prob(np.zeros((2, 2)), [[3.0, 4.0]], [0.0, 0.0], [1.0])
    d1, d2 = O.diagonal_scaling(P, ruiz_iters=0)  # Pock-Chambolle only: 1-norms 3, 4, 7
    assert np.allclose(d2, [1 / math.sqrt(3), 1 / 2], rtol=1e-15)
    assert np.allclose(d1, [1 / math.sqrt(7)], rtol=1e-15)
    # one Ruiz step (inf-norms 3, 4, 4), then Pock-Chambolle on the result
    d1, d2 = O.diagonal_scaling(P, ruiz_iters=1)
    r2 = np.array([1 / math.sqrt(3), 0.5])
    r1 = np.array([0.5])
    a = np.array([3.0, 4.0]) * r2 * r1  # scaled A after the Ruiz step
    assert np.allclose(d2, r2 / np.sqrt(a), rtol=1e-15)
    assert np.allclose(d1, r1 / math.sqrt(a.sum()), rtol=1e-15)
    # a diagonal Q alone: Pock-Chambolle makes it the identity
    d1, d2 = O.diagonal_scaling(_prob(np.diag([4.0, 9.0]), np.zeros((0, 2)), [1, 1], []), 0)
    assert np.allclose(d2, [0.5, 1 / 3], rtol=1e-15)


def test_ruiz_equilibrates_rows():
    """Ruiz iterations converge to a scaling with unit infinity-norm rows."""
    rng = np.random.default_rng(30)
    n, m = 30, 20
    Qd = _rand_spd(rng, n, 50.0) * np.exp(rng.uniform(-3, 3, n))[:, None]
    Qd = (Qd + Qd.T) / 2
    Ad = rng.standard_normal((m, n)) * np.exp(rng.uniform(-4, 4, (m, 1)))
    P = _prob(Qd, Ad, rng.standard_normal(n), rng.standard_normal(m))
    d1, d2 = O.diagonal_scaling(P, ruiz_iters=200, pock_chambolle=False)
    rn, rm = O._row_norms_K(P, d1, d2, ord_inf=True)
    assert np.allclose(rn, 1.0, atol=1e-6) and np.allclose(rm, 1.0, atol=1e-6)
    # Pock-Chambolle afterwards: unit 1-norms are not its fixed point, but a
    # second application changes an already 1-norm-balanced K by little
    d1p, d2p = O.diagonal_scaling(P, ruiz_iters=200)
    rn1, rm1 = O._row_norms_K(P, d1p, d2p, ord_inf=False)
    assert np.all(rn1 > 0) and np.all(rm1 > 0)


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
@pytest.mark.parametrize("seed,n,m,m_eq", [(10, 4, 6, 0), (12, 6, 7, 2), (13, 3, 8, 1)])
@pytest.mark.parametrize("penalty", [False, True])
def test_scaled_solver_matches_active_set_brute_force(seed, n, m, m_eq, step, penalty):
    rng = np.random.default_rng(seed)
    dsc = np.exp(rng.uniform(-2, 2, n))  # badly scaled but PSD (Eq. (1)): D Q D + 0.1 I
    Qd = dsc[:, None] * _rand_spd(rng, n, 10.0) * dsc[None, :] + np.eye(n) * 0.1
    Ad = rng.standard_normal((m, n)) * np.exp(rng.uniform(-2, 2, (m, 1)))
    c = rng.standard_normal(n) * 3
    b = Ad @ rng.standard_normal(n) + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    xs, ys = brute_force_qp(Qd, Ad, c, b, m_eq)
    res = O.solve(_prob(Qd, Ad, c, b, m_eq), _opts(scale=True, step_mode=step, penalty=penalty))
    assert res.termination == O.SOLVED
    assert np.linalg.norm(res.x - xs) <= 1e-6 * (1 + np.linalg.norm(xs))
    assert O.relkkt(_prob(Qd, Ad, c, b, m_eq), res.x, res.y).relkkt <= 1e-10


def test_scaled_solver_box_closed_form():
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n) * np.exp(rng.uniform(-3, 3, n))
    c = rng.standard_normal(n) * 2
    lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    res = O.solve(_prob(np.diag(q), np.vstack([np.eye(n), -np.eye(n)]), c,
                        np.concatenate([hi, -lo])), _opts(scale=True))
    assert res.termination == O.SOLVED
    assert np.max(np.abs(res.x - np.clip(-c / q, lo, hi))) <= 1e-8


# ---------------------------------------------------------------- adaptive step size (Section 4)
def _svd_top(Ad):
    U, sv, Vt = np.linalg.svd(Ad)
    return U[:, 0], sv[0], Vt[0]


@pytest.mark.parametrize("omega", [0.3, 1.0, 4.0])
def test_step_limit_at_the_top_singular_pair(omega):
    """Q = qI, dx = t v1, dy = -/+ omega t u1 (top singular pair of A, LAPACK SVD):
    ||dz||_w^2 = 2 omega t^2, |dy'A dx| = omega s1 t^2, dx'Q dx = q t^2, so the
    limit is 2 omega / (2 omega s1 + q); with q = 0 it is 1/||A||_2 exactly.
    Both signs of dy: the coupling enters through its absolute value."""
    rng = np.random.default_rng(30)
    n, m = 7, 5
    Ad = rng.standard_normal((m, n))
    u1, s1, v1 = _svd_top(Ad)
    x, y = rng.standard_normal(n), rng.standard_normal(m)
    for q in (0.0, 0.7):
        P = _prob(q * np.eye(n), Ad, np.zeros(n), np.zeros(m))
        for sign in (1.0, -1.0):
            t = 0.37
            L = O.step_limit(P, x, y, x + t * v1, y + sign * omega * t * u1, omega)
            assert L == pytest.approx(2 * omega / (2 * omega * s1 + q), rel=1e-12)
    P0 = _prob(np.zeros((n, n)), Ad, np.zeros(n), np.zeros(m))
    assert O.step_limit(P0, x, y, x + v1, y + omega * u1, omega) == pytest.approx(1 / s1, rel=1e-12)


def test_step_limit_lower_bound_and_no_motion():
    """2|dy'A dx| <= ||A|| (omega||dx||^2 + ||dy||^2/omega) and dx'Qdx <= ||Q|| ||dx||^2
    give L >= 1/(||A||_2 + ||Q||_2/omega) for every trial step; no motion gives no limit."""
    rng = np.random.default_rng(31)
    n, m = 9, 6
    Qd = _rand_spd(rng, n, 30.0)
    Ad = rng.standard_normal((m, n))
    P = _prob(Qd, Ad, np.zeros(n), np.zeros(m))
    nA, nQ = np.linalg.norm(Ad, 2), np.linalg.norm(Qd, 2)
    for _ in range(200):
        omega = math.exp(rng.uniform(-3, 3))
        x, y = rng.standard_normal(n), rng.standard_normal(m)
        dx = rng.standard_normal(n) * math.exp(rng.uniform(-2, 2))
        dy = rng.standard_normal(m) * math.exp(rng.uniform(-2, 2))
        L = O.step_limit(P, x, y, x + dx, y + dy, omega)
        assert L >= (1 - 1e-12) / (nA + nQ / omega)
    assert O.step_limit(P, x, y, x, y, 1.0) == math.inf


def test_next_step_size_worked_by_hand():
    """PDLP's rule with a = 3 attempts: 4^-0.3 = 0.6597539553864471 and
    4^-0.6 = 0.43527528164806206 (= 2^-0.6, 2^-1.2)."""
    o = O.OracleOptions()
    # reject eta = 0.5 against L = 0.4: min(0.4 * 0.34024604461355, 0.5 * 1.43527528164806)
    assert O.next_step_size(0.5, 0.4, 3, o) == pytest.approx(0.13609841784542116, rel=1e-14)
    # accept eta = 0.05 against L = 0.4: the growth term 0.05 * 1.435... is the smaller
    assert O.next_step_size(0.05, 0.4, 3, o) == pytest.approx(0.0717637640824031, rel=1e-14)
    # no limit: pure growth
    assert O.next_step_size(0.1, math.inf, 3, o) == pytest.approx(0.14352752816480621, rel=1e-14)


def _adaptive_problem():
    rng = np.random.default_rng(32)
    n, m, m_eq = 12, 16, 2
    Qd = _rand_spd(rng, n, 50.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 3
    b = Ad @ rng.standard_normal(n) + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    return _prob(Qd, Ad, c, b, m_eq)


def _watch_attempts(monkeypatch, P, o):
    """Run a solve, recording every attempt: (accepted, eta, limit, k before/after, z before/after)."""
    seen = []
    inner = O.inner_step

    def wrapped(Pi, st, oo):
        x0, y0, eta0, om0, k0 = st.x.copy(), st.y.copy(), st.eta, st.omega, st.k_total
        xa0, ya0, j0 = st.x_avg.copy(), st.y_avg.copy(), st.j
        inner(Pi, st, oo)
        seen.append(dict(acc=st.last_accepted, eta=eta0, eta_next=st.eta, k0=k0, k=st.k_total,
                         x0=x0, y0=y0, x=st.x.copy(), y=st.y.copy(), j0=j0, j=st.j,
                         xa0=xa0, ya0=ya0, xa=st.x_avg.copy(), ya=st.y_avg.copy(),
                         L=O.step_limit(Pi, x0, y0, st.x, st.y, om0) if st.last_accepted else None))

    monkeypatch.setattr(O, "inner_step", wrapped)
    res = O.solve(P, o)
    monkeypatch.setattr(O, "inner_step", inner)
    return res, seen


def test_adaptive_step_accept_reject_invariants(monkeypatch):
    """Every accepted step satisfies eta <= L and advances k by one; every
    rejected attempt leaves (x, y), k and the averages unchanged and shrinks eta.
    A start at 40x the fixed step forces rejections."""
    P = _adaptive_problem()
    eta0 = 40.0 / (2.0 * O.spectral_norm(P.A, 30))
    res, seen = _watch_attempts(monkeypatch, P, _opts(step_mode=O.STEP_ADAPTIVE, eta=eta0, tol=1e-8))
    assert res.termination == O.SOLVED
    rej = [s for s in seen if not s["acc"]]
    acc = [s for s in seen if s["acc"]]
    assert len(rej) >= 1 and len(acc) == res.iterations
    for s in acc:
        assert s["eta"] <= s["L"] and s["k"] == s["k0"] + 1
    for s in rej:
        assert s["k"] == s["k0"] and s["eta_next"] < s["eta"]
        assert np.array_equal(s["x"], s["x0"]) and np.array_equal(s["y"], s["y0"])
        assert np.array_equal(s["xa"], s["xa0"]) and s["j"] == s["j0"]


def _weighted_average_error(seen):
    """Largest deviation of the averages from sum eta_k z_k / sum eta_k over each epoch."""
    worst, ep = 0.0, []
    for s in seen:
        if not s["acc"]:
            continue
        if s["j"] == 1:
            ep = []
        ep.append(s)
        w = np.array([e["eta"] for e in ep])
        xs = np.average(np.array([e["x"] for e in ep]), axis=0, weights=w)
        ys = np.average(np.array([e["y"] for e in ep]), axis=0, weights=w)
        worst = max(worst, np.max(np.abs(s["xa"] - xs)) / (1 + np.max(np.abs(xs))),
                    np.max(np.abs(s["ya"] - ys)) / (1 + np.max(np.abs(ys))))
    return worst


def test_adaptive_averages_are_step_weighted(monkeypatch):
    P = _adaptive_problem()
    _, seen = _watch_attempts(monkeypatch, P, _opts(step_mode=O.STEP_ADAPTIVE, tol=1e-8))
    assert len({round(s["eta"], 12) for s in seen}) > 5  # the step really varies
    assert _weighted_average_error(seen) <= 1e-12


def test_planted_uniform_average_in_adaptive_mode_is_caught(monkeypatch):
    """The mistake: keep the fixed-step uniform mean while eta varies."""
    P = _adaptive_problem()
    real = O.inner_step

    def uniform_avg(Pi, st, oo):
        xa, ya, j0 = st.x_avg.copy(), st.y_avg.copy(), st.j
        real(Pi, st, oo)
        if st.last_accepted:
            base_x, base_y = (xa, ya) if j0 > 0 else (np.zeros_like(xa), np.zeros_like(ya))
            st.x_avg = base_x + (st.x - base_x) / st.j
            st.y_avg = base_y + (st.y - base_y) / st.j

    monkeypatch.setattr(O, "inner_step", uniform_avg)
    _, seen = _watch_attempts(monkeypatch, P, _opts(step_mode=O.STEP_ADAPTIVE, tol=1e-8, max_iter=600))
    assert _weighted_average_error(seen) > 1e-6


def test_adaptive_step_cuts_iterations_on_a_portfolio_qp():
    """The reason the rule exists: on a portfolio instance it reaches 1e-4 in fewer iterations."""
    from paper_2405_16160_b300 import workloads as W
    P = O.problem_from_instance(W.portfolio(0, 1).to_instance())
    fixed = O.solve(P, _opts(tol=1e-4))
    adaptive = O.solve(P, _opts(tol=1e-4, step_mode=O.STEP_ADAPTIVE))
    assert fixed.termination == adaptive.termination == O.SOLVED
    assert adaptive.state.attempts < 0.7 * fixed.iterations


# ---------------------------------------------------------------- augmented penalty (Section 4)
def test_symmetric_norm_of_a_diagonal_q():
    d = np.array([1.0, 0.1, 0.2, 5.0, -0.3])  # |5| dominates: (1/5)^30 below rounding
    assert O.symmetric_norm(sp.csr_matrix(np.diag(np.abs(d))), 30) == pytest.approx(5.0, rel=1e-15)


def test_penalty_rho_closed_form():
    """Q = qI and one equality row g: ||Q||_2 = q, G'G = g g' has norm ||g||^2,
    so rho = 0.1 q / ||g||^2; without equality rows rho = 0."""
    rng = np.random.default_rng(40)
    n, q = 9, 3.7
    g = rng.standard_normal(n)
    Ad = np.vstack([g, rng.standard_normal((3, n))])
    P = _prob(q * np.eye(n), Ad, np.zeros(n), np.zeros(4), m_eq=1)
    assert O.penalty_rho(P) == pytest.approx(0.1 * q / (g @ g), rel=1e-12)
    assert O.penalty_rho(_prob(q * np.eye(n), Ad, np.zeros(n), np.zeros(4), m_eq=0)) == 0.0


def test_penalized_objective_is_the_original_plus_the_penalty():
    """1/2 x'Q^x + c^'x = 1/2 x'Qx + c'x + rho/2 ||Gx - q||^2 - rho/2 ||q||^2 for every x."""
    rng = np.random.default_rng(41)
    n, m, m_eq = 8, 6, 3
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c, b = rng.standard_normal(n), rng.standard_normal(m)
    P = _prob(Qd, Ad, c, b, m_eq)
    rho = 0.37
    Pp = O.penalize(P, rho)
    for _ in range(5):
        x = rng.standard_normal(n)
        f = 0.5 * x @ Qd @ x + c @ x
        fp = 0.5 * x @ (Pp.Q @ x) + Pp.c @ x
        r = Ad[:m_eq] @ x - b[:m_eq]
        assert fp == pytest.approx(f + 0.5 * rho * (r @ r) - 0.5 * rho * (b[:m_eq] @ b[:m_eq]),
                                   rel=1e-12, abs=1e-12)
    assert np.array_equal(Pp.A.toarray(), P.A.toarray()) and np.array_equal(Pp.b, P.b)


# ---------------------------------------------------------------- theoretical CG precision (Section 3)
def _theory_problem(seed=50, n=10, m=12, cond=30.0):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, cond)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 2
    b = Ad @ rng.standard_normal(n) + rng.uniform(0, 0.5, m)
    return Qd, Ad, c, b


def test_theory_zeta_meets_the_section3_bound():
    """With sigma = tau = 1/(2||A||) the default zeta = ||A|| / (4 K^2) satisfies
    2 zeta <= min{(1 - sqrt(st)||A||)/(2 sqrt(st) K^2), (1 - sqrt(st)||A||)/(2 tau K^2)}
    (with equality), and twice it would not."""
    Qd, Ad, c, b = _theory_problem()
    P = _prob(Qd, Ad, c, b)
    o = _opts(cg_mode=O.CG_THEORY, omega0=1.0)
    st = O.initial_state(P, o)
    nA, K = O.spectral_norm(P.A, 30), o.eval_freq
    sig = tau = st.eta  # omega = 1
    rst = math.sqrt(sig * tau)
    bound = min((1 - rst * nA) / (2 * rst * K ** 2), (1 - rst * nA) / (2 * tau * K ** 2))
    assert 2 * st.zeta <= bound * (1 + 1e-12)
    assert 2 * (2 * st.zeta) > bound
    lmax = np.linalg.eigvalsh(Qd)[-1]  # power iteration approaches it from below
    assert lmax * (1 - 1e-6) <= st.norm_Q <= lmax * (1 + 1e-12)


def test_proposition1_bounds_the_cg_steps():
    """Proposition 1 with the precision sequence of Section 3: after the first
    iteration of an epoch every CG solve stops within log_r(zeta / (2 tau l_max
    (1 + tau||A||)(1 + tau||Q||))) steps, r = (sqrt(k) - 1)/(sqrt(k) + 1), k the
    condition number of Q + I/tau.  (tau l_max, l_max = ||Q + I/tau||, turns
    the paper's error test into the residual test tau ||r|| <= epsilon used
    here, through the energy-norm CG bound; exact CG bounds computed with
    LAPACK eigenvalues.)"""
    Qd, Ad, c, b = _theory_problem()
    P = _prob(Qd, Ad, c, b)
    o = _opts(cg_mode=O.CG_THEORY, cg_max=100_000, omega0=1.0, primal_weight_update=False,
              restart_mode=O.RESTART_FIXED, restart_k=64, tol=0.0, max_iter=640)
    seen = []
    O.solve(P, o, step_hook=lambda st: seen.append((st.j, st.last_cg_steps, st.tau)))
    ev = np.linalg.eigvalsh(Qd)
    nA = np.linalg.norm(Ad, 2)
    checked = 0
    for j, steps, tau in seen:
        if j <= 1:  # epsilon^1 comes from the restart point's dual step
            continue
        lmin, lmax = ev[0] + 1 / tau, ev[-1] + 1 / tau
        kappa = lmax / lmin
        r = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
        zeta = O.initial_state(P, o).zeta
        bound = math.log(zeta / (2 * tau * lmax * (1 + tau * nA) * (1 + tau * ev[-1]))) / math.log(r)
        assert steps <= max(1, math.ceil(bound)) + 1, (steps, bound)
        checked += 1
    assert checked > 500


@pytest.mark.parametrize("seed,n,m,m_eq", [(10, 4, 6, 0), (12, 6, 7, 2)])
def test_theory_rule_reaches_the_brute_force_solution(seed, n, m, m_eq):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 3
    b = Ad @ rng.standard_normal(n) + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    xs, ys = brute_force_qp(Qd, Ad, c, b, m_eq)
    res = O.solve(_prob(Qd, Ad, c, b, m_eq), _opts(cg_mode=O.CG_THEORY))
    assert res.termination == O.SOLVED
    assert np.linalg.norm(res.x - xs) <= 1e-6 * (1 + np.linalg.norm(xs))


def test_theory_precision_grows_within_an_epoch_and_restarts_at_zero_increment(monkeypatch):
    """epsilon^k is non-decreasing inside an epoch; each epoch's first value is
    the restart point's own (zeta ||y^ - y|| / (1 + tau||Q||)), not a sum."""
    Qd, Ad, c, b = _theory_problem(seed=51)
    P = _prob(Qd, Ad, c, b)
    o = _opts(cg_mode=O.CG_THEORY, restart_mode=O.RESTART_FIXED, restart_k=64, tol=0.0,
              max_iter=256)
    eps = []
    O.solve(P, o, step_hook=lambda st: eps.append((st.j, st.eps)))
    for (j0, e0), (j1, e1) in zip(eps, eps[1:]):
        if j1 == j0 + 1:
            assert e1 >= e0
    firsts = [e for j, e in eps if j == 1]
    assert len(firsts) >= 3 and all(e >= 0 for e in firsts)


# ---------------------------------------------------------------- variable bounds and BB (Section 4)
def _box_brute_force(M, rhs, lo, hi):
    """min 1/2 x'Mx - rhs'x over the box, exactly: every assignment of the
    variables to lower bound / upper bound / free, the free ones solved by
    LAPACK, kept when feasible with the right multiplier signs."""
    n = len(rhs)
    best = None
    for pat in itertools.product((0, 1, 2), repeat=n):
        x = np.zeros(n)
        fixed = [j for j in range(n) if pat[j] != 2]
        for j in fixed:
            x[j] = lo[j] if pat[j] == 0 else hi[j]
        if not np.all(np.isfinite(x[fixed])):
            continue
        free = [j for j in range(n) if pat[j] == 2]
        if free:
            r = rhs[free] - M[np.ix_(free, fixed)] @ x[fixed]
            x[free] = np.linalg.solve(M[np.ix_(free, free)], r)
        if np.any(x < lo - 1e-12) or np.any(x > hi + 1e-12):
            continue
        g = M @ x - rhs
        if any((pat[j] == 0 and g[j] < -1e-10) or (pat[j] == 1 and g[j] > 1e-10) for j in range(n)):
            continue
        best = x
        break
    assert best is not None
    return best


def test_bb_without_bounds_solves_the_linear_system():
    rng = np.random.default_rng(60)
    n = 12
    Qd = _rand_spd(rng, n, 50.0)
    rhs = rng.standard_normal(n)
    tau = 0.7
    x, steps = O.bb(sp.csr_matrix(Qd), tau, rhs, np.zeros(n), np.full(n, -np.inf),
                    np.full(n, np.inf), O.CG_ADAPTIVE, eps=1e-13, bb_max=10_000)
    assert np.allclose(x, np.linalg.solve(Qd + np.eye(n) / tau, rhs), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_bb_matches_box_brute_force_and_stays_in_the_box(seed):
    rng = np.random.default_rng(seed)
    n = 6
    Qd = _rand_spd(rng, n, 20.0)
    rhs = rng.standard_normal(n) * 3
    lo = np.where(rng.random(n) < 0.7, -rng.uniform(0.1, 1, n), -np.inf)
    hi = np.where(rng.random(n) < 0.7, rng.uniform(0.1, 1, n), np.inf)
    tau = 1.3
    xs = _box_brute_force(Qd + np.eye(n) / tau, rhs, lo, hi)
    x, steps = O.bb(sp.csr_matrix(Qd), tau, rhs, np.clip(np.zeros(n), lo, hi), lo, hi,
                    O.CG_ADAPTIVE, eps=1e-14, bb_max=20_000)
    assert np.all(x >= lo) and np.all(x <= hi)
    assert np.allclose(x, xs, rtol=1e-9, atol=1e-10)


def test_relkkt_with_bounds_worked_by_hand():
    """min x^2 - 6x on x <= 1 (Q = [2], c = -6, no rows).  At x* = 1: g = -4, the
    upper bound's multiplier -4 (lambda^- = 4): r_dual = 0, dual objective
    -1 - 1*4 = -5 = primal objective.  At x = 0.5: g = -5 is still allowed
    (r_dual = 0) but the gap catches it: pobj = -2.75, dobj = -0.25 - 5 = -5.25,
    r_gap = 2.5 / (1 + 5.25) = 0.4."""
    P = _prob([[2.0]], np.zeros((0, 1)), [-6.0], np.zeros(0))
    P.lo, P.hi = np.array([-np.inf]), np.array([1.0])
    k = O.relkkt(P, np.array([1.0]), np.zeros(0))
    assert k.r_dual == 0.0 and k.r_gap == 0.0 and k.primal_obj == -5.0 and k.dual_obj == -5.0
    k = O.relkkt(P, np.array([0.5]), np.zeros(0))
    assert k.r_dual == 0.0
    assert k.primal_obj == -2.75 and k.dual_obj == -5.25
    assert k.r_gap == pytest.approx(0.4, rel=1e-15)
    # a lower bound alone cannot absorb a negative gradient: x = 0.5 with x >= 0
    P.lo, P.hi = np.array([0.0]), np.array([np.inf])
    k = O.relkkt(P, np.array([0.5]), np.zeros(0))
    assert k.r_dual == pytest.approx(5.0 / (1.0 + 6.0), rel=1e-15)


@pytest.mark.parametrize("step", [O.STEP_FIXED, O.STEP_ADAPTIVE])
def test_solver_box_bounds_closed_form(step):
    """Diagonal Q with the box as variable bounds (no rows): x* = clip(-c/q, lo, hi)."""
    rng = np.random.default_rng(64)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2
    P = _prob(np.diag(q), np.zeros((0, n)), c, np.zeros(0))
    P.lo, P.hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    res = O.solve(P, _opts(step_mode=step))
    assert res.termination == O.SOLVED
    assert np.max(np.abs(res.x - np.clip(-c / q, P.lo, P.hi))) <= 1e-8


@pytest.mark.parametrize("seed,n,m,m_eq", [(70, 4, 5, 0), (71, 5, 6, 1), (72, 3, 4, 2)])
@pytest.mark.parametrize("scale", [False, True])
def test_solver_with_bounds_matches_brute_force_with_the_bounds_as_rows(seed, n, m, m_eq, scale):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 3
    x0 = rng.uniform(-0.3, 0.3, n)
    b = Ad @ x0 + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    lo = np.where(rng.random(n) < 0.6, -rng.uniform(0.4, 1, n), -np.inf)
    hi = np.where(rng.random(n) < 0.6, rng.uniform(0.4, 1, n), np.inf)
    rows = [j for j in range(n) if np.isfinite(hi[j])], [j for j in range(n) if np.isfinite(lo[j])]
    Ab = np.vstack([Ad, np.eye(n)[rows[0]], -np.eye(n)[rows[1]]])
    bb_ = np.concatenate([b, hi[rows[0]], -lo[rows[1]]])
    xs, _ = brute_force_qp(Qd, Ab, c, bb_, m_eq)
    P = _prob(Qd, Ad, c, b, m_eq)
    P.lo, P.hi = lo, hi
    res = O.solve(P, _opts(scale=scale))
    assert res.termination == O.SOLVED
    assert np.all(res.x >= lo - 1e-12) and np.all(res.x <= hi + 1e-12)
    assert np.linalg.norm(res.x - xs) <= 1e-6 * (1 + np.linalg.norm(xs))
    assert res.kkt.primal_obj == pytest.approx(0.5 * xs @ Qd @ xs + c @ xs, rel=1e-8, abs=1e-8)


def test_long_only_bounds_match_long_only_rows_on_a_portfolio():
    """The portfolio's long-only rows -x <= 0 as the bound x >= 0: the same solution."""
    from paper_2405_16160_b300 import workloads as W
    lr = W.portfolio(0, 5, n_lo=30, n_hi=60)
    P_rows = O.problem_from_instance(lr.to_instance())
    keep = [i for i in range(P_rows.m) if not (P_rows.A[i].nnz == 1 and P_rows.A[i].data[0] < 0
                                                and P_rows.b[i] == 0.0)]
    P = O.OracleProblem(P_rows.Q, P_rows.A[keep], P_rows.c, P_rows.b[keep], P_rows.m_eq,
                        np.zeros(P_rows.n), np.full(P_rows.n, np.inf))
    assert P.m == P_rows.m - P_rows.n
    r1 = O.solve(P_rows, _opts(tol=1e-9))
    r2 = O.solve(P, _opts(tol=1e-9))
    assert r1.termination == r2.termination == O.SOLVED
    assert np.max(np.abs(r1.x - r2.x)) <= 1e-6
