"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each test fixes part of the oracle to something the paper or the mathematics
determines: hand-worked relKKT values (Section 4), closed-form QP solutions,
LAPACK solves, an exhaustive active-set search on tiny QPs, the textbook CG
error bound (Section 2), Lemma A.2(2) and Theorem 2 of the appendix, and the
trend of Table 2.  The last group plants mistakes in the oracle and checks
that a pin catches each one.
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


def test_solver_unconstrained_m0():
    rng = np.random.default_rng(6)
    n = 25
    Qd = _rand_spd(rng, n, 20.0)
    c = rng.standard_normal(n)
    P = _prob(Qd, np.zeros((0, n)), c, np.zeros(0))
    res = O.solve(P, _opts())
    assert res.termination == O.SOLVED
    xs = -np.linalg.solve(Qd, c)
    assert np.linalg.norm(res.x - xs) <= 1e-8 * (1 + np.linalg.norm(xs))


def test_solver_diagonal_box_closed_form():
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2
    lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    Ad = np.vstack([np.eye(n), -np.eye(n)])
    b = np.concatenate([hi, -lo])
    res = O.solve(_prob(np.diag(q), Ad, c, b), _opts())
    assert res.termination == O.SOLVED
    xs = np.clip(-c / q, lo, hi)
    g = q * xs + c
    ys = np.concatenate([np.maximum(-g, 0) * (xs >= hi), np.maximum(g, 0) * (xs <= lo)])
    assert np.max(np.abs(res.x - xs)) <= 1e-8
    assert np.max(np.abs(res.y - ys)) <= 1e-7


def test_solver_equality_hyperplane_closed_form():
    rng = np.random.default_rng(8)
    n = 30
    a = rng.standard_normal(n)
    c = rng.standard_normal(n)
    beta = 0.7
    res = O.solve(_prob(np.eye(n), a[None, :], c, [beta], m_eq=1), _opts())
    assert res.termination == O.SOLVED
    xs = -c + a * (beta + a @ c) / (a @ a)
    lam = -(beta + a @ c) / (a @ a)
    assert np.max(np.abs(res.x - xs)) <= 1e-8
    assert res.y[0] == pytest.approx(lam, abs=1e-7)


@pytest.mark.parametrize("seed,n,m,m_eq", [(10, 4, 6, 0), (11, 5, 8, 0), (12, 6, 7, 2), (13, 3, 8, 1)])
def test_solver_matches_active_set_brute_force(seed, n, m, m_eq):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, 10.0)
    Ad = rng.standard_normal((m, n))
    c = rng.standard_normal(n) * 3
    x0 = rng.standard_normal(n)
    b = Ad @ x0 + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    xs, ys = brute_force_qp(Qd, Ad, c, b, m_eq)
    res = O.solve(_prob(Qd, Ad, c, b, m_eq), _opts())
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


@pytest.mark.parametrize("seed,n,m,m_eq", [(10, 4, 6, 0), (12, 6, 7, 2), (13, 3, 8, 1)])
def test_scaled_solver_matches_active_set_brute_force(seed, n, m, m_eq):
    rng = np.random.default_rng(seed)
    Qd = _rand_spd(rng, n, 10.0) * np.exp(rng.uniform(-2, 2, n))[:, None]
    Qd = (Qd + Qd.T) / 2 + np.eye(n) * 0.1
    Ad = rng.standard_normal((m, n)) * np.exp(rng.uniform(-2, 2, (m, 1)))
    c = rng.standard_normal(n) * 3
    b = Ad @ rng.standard_normal(n) + np.concatenate([np.zeros(m_eq), rng.uniform(0, 0.5, m - m_eq)])
    xs, ys = brute_force_qp(Qd, Ad, c, b, m_eq)
    res = O.solve(_prob(Qd, Ad, c, b, m_eq), _opts(scale=True))
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
