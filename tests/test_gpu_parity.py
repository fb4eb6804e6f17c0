"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (FP64 on both sides; the two differ only in summation order and
in fused multiply-adds):
  * ||A||_2, relKKT terms: 1e-12 relative;
  * one iteration from a shared state: 1e-10 relative (infinity norm);
  * end to end: both reach relKKT <= tol, the oracle re-scores the GPU
    solution at <= tol, the restart decisions agree, and the objectives
    agree within 1e-4 relative.  The solver's own relKKT of its result
    agrees with the oracle's re-score to 1e-9 relative or 1e-12 absolute:
    relKKT's numerators (Ax - b, Qx + A'y + c, the gap) cancel near a
    solution, and two FP64 evaluations that sum in different orders agree
    to a few ulps of the terms, not of the small difference.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pdhcg_oracle as O
from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import workloads as W
from paper_2405_16160_b300.solver import QPOptions, QPSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2405_16160_b300 import build
    build.build()


def _ragged_eq():
    return W.sparse_dd(3, n=1237, m=611, m_eq=17)


def _unconstrained():
    rng = np.random.default_rng(5)
    n = 37
    M = rng.standard_normal((n, n))
    Qd = M @ M.T / n + np.eye(n)
    return W.from_dense(Qd, np.zeros((0, n)), rng.standard_normal(n), np.zeros(0), name="m=0")


def _all_equalities():
    rng = np.random.default_rng(6)
    n, m = 40, 12
    Qd = np.diag(rng.uniform(0.5, 2, n))
    Ad = W._bernoulli_normal(rng, m, n, 0.3)
    return W.from_dense(Qd, Ad, rng.standard_normal(n), Ad @ rng.standard_normal(n), m_eq=m,
                        name="all equalities")


def _empty_rows():
    rng = np.random.default_rng(7)
    n, m = 50, 30
    Qd = np.diag(rng.uniform(0.5, 2, n))
    Qd[3, 3] = 0.0  # an empty row/column of Q (PSD)
    Ad = W._bernoulli_normal(rng, m, n, 0.2)
    Ad[[0, 7, 29], :] = 0.0  # empty rows of A
    Ad[:, [4, 9]] = 0.0  # empty rows of A'
    return W.from_dense(Qd, Ad, rng.standard_normal(n), Ad @ rng.standard_normal(n) + 0.5,
                        name="empty rows")


def _single():
    return W.from_dense(np.array([[2.0]]), np.array([[1.0]]), np.array([-3.0]), np.array([1.0]),
                        name="n=1")


def _long_rows():
    """Rows longer than the 4096-entry long-row threshold in A, A' and Q, and
    medium rows (a few hundred entries among rows of a handful, taken by a
    whole warp) in each of them."""
    import scipy.sparse as sp
    rng = np.random.default_rng(8)
    n, m = 10_000, 6_000
    A = sp.random(m, n, density=6 / n, random_state=8, data_rvs=rng.standard_normal).tolil()
    A[:, 3] = rng.standard_normal((m, 1))        # A' row 3: 6000 entries
    A[0, :5000] = rng.standard_normal(5000)      # A rows 0, 1: 5000 entries
    A[1, 2000:7000] = rng.standard_normal(5000)
    A[:300, 7] = rng.standard_normal((300, 1))   # A' row 7: 300 entries (medium)
    A[2, 7000:7150] = rng.standard_normal(150)   # A row 2: 150 entries (medium)
    A = A.tocsr()
    S = sp.random(n, n, density=3 / n, random_state=9, data_rvs=lambda k: rng.normal(0, 0.1, k))
    S = sp.lil_matrix(S + S.T)
    S[5, 100:5100] = rng.normal(0, 0.01, 5000)   # Q row/column 5: > 5000 entries
    S[100:5100, 5] = S[5, 100:5100].T
    S[9, 6000:6200] = rng.normal(0, 0.01, 200)   # Q row/column 9: 200 entries (medium)
    S[6000:6200, 9] = S[9, 6000:6200].T
    S = S.tocsr()
    Q = S + sp.diags(np.asarray(abs(S).sum(axis=1)).ravel() + rng.uniform(0.5, 2, n))
    x0 = rng.standard_normal(n)
    b = A @ x0 + rng.uniform(0, 1, m)
    return W.from_dense(Q.toarray(), A.toarray(), rng.standard_normal(n), b, name="long rows")


CASES = {
    "dense_small": lambda: W.dense_small(0),
    "dense_small_eq": lambda: W.dense_small(1, m_eq=10),
    "sparse_small": lambda: W.sparse_dd(0, n=20_000, m=10_000),
    "ragged_eq": _ragged_eq,
    "unconstrained": _unconstrained,
    "all_equalities": _all_equalities,
    "empty_rows": _empty_rows,
    "single": _single,
    "long_rows": _long_rows,
    "zipf_small": lambda: W.zipf_dd(0, n=20_000, m=10_000),
}


def _relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _shared_state(inst, P, seed):
    rng = np.random.default_rng(seed)
    n, m, me = inst.n, inst.m, inst.m_eq

    def yv():
        y = np.abs(rng.standard_normal(m))
        y[:me] = rng.standard_normal(me)
        return y

    eta = 1.0 / (2.0 * max(O.spectral_norm(P.A, 30), 1e-10))
    return {"x": rng.standard_normal(n), "y": yv(), "x_avg": rng.standard_normal(n),
            "y_avg": yv(), "x_anchor": rng.standard_normal(n), "y_anchor": yv(),
            "eta": eta, "omega": 1.3, "eps": 1e-3, "relkkt_last": 0.2, "kkt_anchor": 0.5,
            "kkt_prev_cand": math.inf, "j": 3, "k_total": 10, "restarts": 0, "cg_total": 0}


def _oracle_state(s):
    return O.OracleState(x=s["x"].copy(), y=s["y"].copy(), x_avg=s["x_avg"].copy(),
                         y_avg=s["y_avg"].copy(), x_anchor=s["x_anchor"].copy(),
                         y_anchor=s["y_anchor"].copy(), eta=s["eta"], omega=s["omega"],
                         eps=s["eps"], j=s["j"], k_total=s["k_total"],
                         relkkt_last=s["relkkt_last"], kkt_anchor=s["kkt_anchor"],
                         kkt_prev_cand=s["kkt_prev_cand"])


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name):
        if name not in cache:
            inst = CASES[name]()
            cache[name] = (inst, O.problem_from_instance(inst), QPSolver(inst))
        return cache[name]

    yield get
    for _, _, s in cache.values():
        s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_norm_A_matches_oracle(built, name):
    inst, P, s = built(name)
    assert s.norm_A(30) == pytest.approx(O.spectral_norm(P.A, 30), rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_relkkt_terms_match_oracle(built, name):
    inst, P, s = built(name)
    st = _shared_state(inst, P, 1)
    s.set_state(st)
    kc, ka = s.evaluate()
    for got, (x, y) in ((kc, (st["x"], st["y"])), (ka, (st["x_avg"], st["y_avg"]))):
        ref = O.relkkt(P, x, y)
        for key in ("r_primal", "r_dual", "r_gap", "relkkt", "primal_obj", "dual_obj"):
            assert got[key] == pytest.approx(getattr(ref, key), rel=1e-12, abs=1e-14), key


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode,iters", [("fixed3", 1), ("adaptive", 1), ("adaptive", 4)])
def test_iterations_match_oracle(built, name, mode, iters):
    inst, P, s = built(name)
    st = _shared_state(inst, P, 2)
    s.set_state(st)
    kw = dict(cg_mode=L.CG_FIXED, cg_fixed_n=3) if mode == "fixed3" else {}
    s.iterate(iters, **kw)
    got = s.get_state()
    o = O.OracleOptions(**({"cg_mode": O.CG_FIXED, "cg_fixed_n": 3} if mode == "fixed3" else {}))
    ost = _oracle_state(st)
    for _ in range(iters):
        O.inner_step(P, ost, o)
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-10, key
    assert got["cg_total"] == ost.cg_total
    assert got["j"] == ost.j and got["k_total"] == ost.k_total
    assert got["eps"] == pytest.approx(ost.eps, rel=1e-15)
    if inst.m > inst.m_eq:
        assert np.all(got["y"][inst.m_eq:] >= 0.0)


@pytest.mark.parametrize("name,tol", [("dense_small", 1e-6), ("dense_small_eq", 1e-6),
                                      ("sparse_small", 1e-4), ("ragged_eq", 1e-4),
                                      ("unconstrained", 1e-6), ("all_equalities", 1e-6),
                                      ("empty_rows", 1e-6), ("single", 1e-8),
                                      ("long_rows", 1e-5)])
def test_end_to_end_matches_oracle(built, name, tol):
    inst, P, s = built(name)
    ores = O.solve(P, O.OracleOptions(tol=tol))
    info = s.solve(tol=tol)
    x, y = s.solution()
    assert ores.termination == O.SOLVED
    assert info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= tol
    assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
    assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
    if name == "unconstrained":
        # m = 0 gives ||A|| = 0, so tau = 1/(2 eps_zero) = 5e9 and the adaptive CG
        # tolerance eps/tau sits at the rounding level of r0: step counts then
        # depend on summation order and only the result is comparable.
        assert _relerr(x, ores.x) <= 1e-6
        return
    # same trajectory: iteration count, restarts, CG steps and restart decisions
    trace = s.trace()
    orestarts = [(r["k"], int(r["restart"]) * (2 if r["cand_avg"] else 1)) for r in ores.trace[1:]]
    grestarts = [(t["k"], t["restart"]) for t in trace]
    assert grestarts == orestarts
    assert info["iterations"] == ores.iterations
    assert info["restarts"] == ores.restarts
    assert info["cg_steps"] == ores.cg_steps
    assert _relerr(x, ores.x) <= 1e-8


def test_solves_are_deterministic_and_allocator_independent(built):
    inst, P, s = built("sparse_small")
    s.solve(tol=1e-4)
    x1, y1 = s.solution()
    s.solve(tol=1e-4)
    x2, y2 = s.solution()
    with QPSolver(inst, torch_memory=False) as s2:
        s2.solve(tol=1e-4)
        x3, y3 = s2.solution()
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    assert np.array_equal(x1, x3) and np.array_equal(y1, y3)


def test_checkpoint_resume_is_bit_identical(built):
    inst, P, s = built("sparse_small")
    s.solve(tol=0.0, max_iter=256)
    full = s.get_state()
    s.solve(tol=0.0, max_iter=128)
    mid = s.get_state()
    with QPSolver(inst) as s2:
        s2.set_state(mid)
        s2.solve(tol=0.0, max_iter=256, warm_start=2)
        resumed = s2.get_state()
    for key in ("x", "y", "x_avg", "y_avg", "x_anchor", "y_anchor"):
        assert np.array_equal(full[key], resumed[key]), key
    for key in ("omega", "eps", "j", "k_total", "restarts", "cg_total"):
        assert full[key] == resumed[key], key


def test_warm_start_from_solution_stops_at_once(built):
    inst, P, s = built("dense_small")
    s.solve(tol=1e-6)
    x, y = s.solution()
    s.set_warm_start(x, y)
    info = s.solve(tol=1e-6, warm_start=1)
    assert info["termination"] == L.TERM_SOLVED and info["iterations"] == 0


def test_iteration_limit_returns_best_iterate(built):
    inst, P, s = built("sparse_small")
    info = s.solve(tol=1e-12, max_iter=100)
    assert info["termination"] == L.TERM_ITER_LIMIT and info["iterations"] == 100
    x, y = s.solution()
    assert O.relkkt(P, x, y).relkkt == pytest.approx(info["relkkt"], rel=1e-9)


def test_numerical_error_on_indefinite_q():
    n = 20
    inst = W.from_dense(-100.0 * np.eye(n), np.ones((1, n)), np.ones(n), np.array([1.0]))
    ores = O.solve(O.problem_from_instance(inst), O.OracleOptions())
    assert ores.termination == O.NUMERICAL_ERROR
    with QPSolver(inst) as s:
        info = s.solve()
    assert info["termination"] == L.TERM_NUMERICAL


def test_barrier_timeout_returns_status_and_context_survives(built):
    inst, P, s = built("sparse_small")
    with pytest.raises(L.QPError) as e:
        s.solve(debug_flags=L.DEBUG_BARRIER_NEVER_RELEASES)
    assert e.value.status == 5
    info = s.solve(tol=1e-4)  # the same handle keeps working
    assert info["termination"] == L.TERM_SOLVED


# ------------------------------------------------------------- full size
GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "sparse_dd_n1000000_m500000_seed0_trace.json")


@pytest.fixture(scope="module")
def big():
    inst = W.sparse_dd(0)
    s = QPSolver(inst)
    yield inst, O.problem_from_instance(inst), s
    s.close()


def test_full_size_one_iteration_parity(big):
    inst, P, s = big
    st = _shared_state(inst, P, 3)
    s.set_state(st)
    s.iterate(1)
    got = s.get_state()
    ost = _oracle_state(st)
    O.inner_step(P, ost, O.OracleOptions())
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-10, key
    assert got["cg_total"] == ost.cg_total


def test_full_size_solve_matches_oracle_trace(big):
    inst, P, s = big
    info = s.solve(tol=1e-4)
    x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= 1e-4
    with open(GOLDEN) as f:
        g = json.load(f)
    assert info["iterations"] == g["iterations"]
    assert info["restarts"] == g["restarts"]
    assert info["cg_steps"] == g["cg_steps"]
    assert rescored.primal_obj == pytest.approx(g["primal_obj"], rel=1e-4)
    assert info["norm_A"] == pytest.approx(1.0 / (2.0 * g["eta"]), rel=1e-12)


# ------------------------------------------------------------- mixed precision
# FP32 values/iterates/SpMVs with FP64-accurate reductions: one iteration
# from a shared state agrees with the FP64 oracle to 1e-5 relative; a solve
# ends with an FP64 re-evaluation (and FP64 refinement if needed), so the
# oracle re-scores its result at <= tol.
MIXED_ITER_CASES = ["dense_small", "dense_small_eq", "sparse_small", "ragged_eq", "empty_rows",
                    "long_rows", "zipf_small"]


@pytest.mark.parametrize("name", MIXED_ITER_CASES)
@pytest.mark.parametrize("n_cg", [1, 3])
def test_mixed_one_iteration_matches_oracle(built, name, n_cg):
    inst, P, s = built(name)
    st = _shared_state(inst, P, 4)
    s.set_state(st)
    s.iterate(1, cg_mode=L.CG_FIXED, cg_fixed_n=n_cg, precision=L.PREC_MIXED)
    got = s.get_state()
    ost = _oracle_state(st)
    O.inner_step(P, ost, O.OracleOptions(cg_mode=O.CG_FIXED, cg_fixed_n=n_cg))
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-5, key
    assert got["cg_total"] == ost.cg_total


@pytest.mark.parametrize("name,tol", [("dense_small", 1e-6), ("dense_small_eq", 1e-6),
                                      ("sparse_small", 1e-4), ("ragged_eq", 1e-4),
                                      ("unconstrained", 1e-6), ("all_equalities", 1e-6),
                                      ("empty_rows", 1e-6), ("single", 1e-8)])
def test_mixed_solve_meets_tolerance_in_fp64(built, name, tol):
    inst, P, s = built(name)
    ores = O.solve(P, O.OracleOptions(tol=tol))
    info = s.solve(tol=tol, precision=L.PREC_MIXED)
    x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= tol
    assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
    assert info["check_relkkt"] >= 0.0 and info["mixed_iterations"] > 0
    assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)


def test_mixed_full_size_meets_tolerance(big):
    inst, P, s = big
    info = s.solve(tol=1e-4, precision=L.PREC_MIXED)
    x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= 1e-4
    with open(GOLDEN) as f:
        g = json.load(f)
    assert rescored.primal_obj == pytest.approx(g["primal_obj"], rel=1e-4)


# ------------------------------------------------------- Section 4 scaling
# QP_CREATE_SCALE: D1, D2 from 10 Ruiz steps and one Pock-Chambolle step;
# the solver iterates on the scaled problem and measures relKKT on the
# original one.  The oracle computes its own scaling from the paper's steps.
SCALED_CASES = ["dense_small", "sparse_small", "ragged_eq", "empty_rows", "long_rows",
                "zipf_small"]


@pytest.fixture(scope="module")
def built_scaled():
    cache = {}

    def get(name):
        if name not in cache:
            inst = CASES[name]()
            P = O.problem_from_instance(inst)
            d1, d2 = O.diagonal_scaling(P)
            cache[name] = (inst, P, d1, d2, QPSolver(inst, scale=True))
        return cache[name]

    yield get
    for v in cache.values():
        v[-1].close()


@pytest.mark.parametrize("name", SCALED_CASES)
def test_scaling_matches_oracle(built_scaled, name):
    inst, P, d1, d2, s = built_scaled(name)
    g1, g2 = s.scaling()
    assert _relerr(g1, d1) <= 1e-12 and _relerr(g2, d2) <= 1e-12


@pytest.mark.parametrize("name", SCALED_CASES)
def test_scaled_relkkt_is_measured_on_the_original_problem(built_scaled, name):
    inst, P, d1, d2, s = built_scaled(name)
    st = _shared_state(inst, P, 5)  # taken as scaled iterates
    s.set_state(st)
    kc, ka = s.evaluate()
    for got, (x, y) in ((kc, (st["x"], st["y"])), (ka, (st["x_avg"], st["y_avg"]))):
        ref = O.relkkt(P, d2 * x, d1 * y)
        for key in ("r_primal", "r_dual", "r_gap", "relkkt", "primal_obj", "dual_obj"):
            assert got[key] == pytest.approx(getattr(ref, key), rel=1e-12, abs=1e-14), key


@pytest.mark.parametrize("name", SCALED_CASES)
def test_scaled_iteration_matches_oracle(built_scaled, name):
    inst, P, d1, d2, s = built_scaled(name)
    Ps = O.scale_problem(P, d1, d2)
    st = _shared_state(inst, Ps, 6)
    s.set_state(st)
    s.iterate(1, cg_mode=L.CG_FIXED, cg_fixed_n=3)
    got = s.get_state()
    ost = _oracle_state(st)
    O.inner_step(Ps, ost, O.OracleOptions(cg_mode=O.CG_FIXED, cg_fixed_n=3))
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-10, key


@pytest.mark.parametrize("name,tol", [("dense_small", 1e-6), ("sparse_small", 1e-4),
                                      ("ragged_eq", 1e-4), ("long_rows", 1e-5),
                                      ("zipf_small", 1e-4)])
def test_scaled_end_to_end_matches_oracle(built_scaled, name, tol):
    inst, P, d1, d2, s = built_scaled(name)
    ores = O.solve(P, O.OracleOptions(tol=tol, scale=True))
    info = s.solve(tol=tol)
    x, y = s.solution()
    assert ores.termination == O.SOLVED and info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= tol
    assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
    assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
    assert info["iterations"] == ores.iterations and info["restarts"] == ores.restarts
    assert info["cg_steps"] == ores.cg_steps
    assert _relerr(x, ores.x) <= 1e-8


@pytest.mark.parametrize("name,tol", [("sparse_small", 1e-4), ("long_rows", 1e-5),
                                      ("zipf_small", 1e-4)])
def test_scaled_mixed_solve_meets_tolerance(built_scaled, name, tol):
    inst, P, d1, d2, s = built_scaled(name)
    info = s.solve(tol=tol, precision=L.PREC_MIXED)
    x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED
    assert O.relkkt(P, x, y).relkkt <= tol


# ------------------------------------------- mixed path: state representation
# The mixed path keeps x as the restart point (a compensated FP32 pair) plus
# an FP32 displacement, and y as a compensated pair.  Moving a state into it
# and reading it back therefore loses at most one FP32 rounding of the
# displacement x - x_anchor and ~2^-47 of everything else.
def test_mixed_state_round_trip_keeps_the_restart_point(built):
    inst, P, s = built("sparse_small")
    st = _shared_state(inst, P, 6)
    st["x"] = st["x_anchor"] + 1e-3 * st["x"]      # an iterate near its restart point
    st["x_avg"] = st["x_anchor"] + 1e-3 * st["x_avg"]
    s.set_state(st)
    s.iterate(0, precision=L.PREC_MIXED)
    got = s.get_state()
    a = st["x_anchor"]
    assert np.all(np.abs(got["x_anchor"] - a) <= 2.0 ** -46 * np.abs(a))
    for key in ("x", "x_avg"):
        bound = 2.0 ** -24 * np.abs(st[key] - a) + 2.0 ** -46 * np.abs(a)
        assert np.all(np.abs(got[key] - st[key]) <= bound), key
    for key in ("y", "y_avg"):
        assert np.all(np.abs(got[key] - st[key]) <= 2.0 ** -46 * np.abs(st[key])), key


# A scaled instance with power-law column popularity: diagonal scaling makes
# the iterate large on the popular columns, where thousands of rows share one
# coordinate.  The mixed path must converge like FP64 there (it once stalled
# near relKKT 1e-2 when those coordinates moved in FP32 ulp steps).
def test_mixed_tracks_fp64_on_a_scaled_power_law_instance():
    inst = W.zipf_dd(0, n=200_000, m=100_000)
    with QPSolver(inst, scale=True) as s:
        f64 = s.solve(tol=1e-4, precision=L.PREC_FP64, max_iter=20000)
        mix = s.solve(tol=1e-4, precision=L.PREC_MIXED, max_iter=20000)
    assert f64["termination"] == L.TERM_SOLVED and mix["termination"] == L.TERM_SOLVED
    assert mix["check_relkkt"] <= 1e-4 and mix["refine_iterations"] == 0
    assert mix["iterations"] <= 1.15 * f64["iterations"]


# ------------------------------------------- full size, Section 4 scaling
GOLDEN_SCALED = os.path.join(os.path.dirname(__file__), "golden",
                             "sparse_dd_n1000000_m500000_seed0_scaled_trace.json")


def test_full_size_scaled_solve_matches_oracle_trace():
    inst = W.sparse_dd(0)
    with open(GOLDEN_SCALED) as f:
        g = json.load(f)
    with QPSolver(inst, scale=True) as s:
        info = s.solve(tol=1e-4)
        x, y = s.solution()
        mix = s.solve(tol=1e-4, precision=L.PREC_MIXED)
        xm, ym = s.solution()
    P = O.problem_from_instance(inst)
    rescored = O.relkkt(P, x, y)
    assert info["termination"] == L.TERM_SOLVED and rescored.relkkt <= 1e-4
    assert info["iterations"] == g["iterations"]
    assert info["restarts"] == g["restarts"]
    assert info["cg_steps"] == g["cg_steps"]
    assert rescored.primal_obj == pytest.approx(g["primal_obj"], rel=1e-4)
    # mixed precision on the same scaled instance
    assert mix["termination"] == L.TERM_SOLVED
    assert O.relkkt(P, xm, ym).relkkt <= 1e-4
    assert O.relkkt(P, xm, ym).primal_obj == pytest.approx(g["primal_obj"], rel=1e-4)


# ------------------------------------------------- Section 4 adaptive step size
# Each attempt runs the iteration into a trial point, the step test accepts
# or rejects it (a rejection keeps z) and eta moves either way.  From a
# shared state the GPU's attempts match the oracle's: the same decisions,
# eta to 1e-12 and the iterates to 1e-10 (FP64).  A start at 30x the fixed
# step makes the first attempts rejections.
ADAPTIVE_ITER_CASES = ["dense_small", "dense_small_eq", "sparse_small", "ragged_eq",
                       "empty_rows", "single", "long_rows", "zipf_small"]


@pytest.mark.parametrize("name", ADAPTIVE_ITER_CASES)
@pytest.mark.parametrize("eta_mult,iters", [(1.0, 1), (1.0, 4), (30.0, 4)])
def test_adaptive_step_attempts_match_oracle(built, name, eta_mult, iters):
    inst, P, s = built(name)
    st = _shared_state(inst, P, 5)
    st["eta"] *= eta_mult
    s.set_state(st)
    s.iterate(iters, step_mode=L.STEP_ADAPTIVE)
    got = s.get_state()
    ost = _oracle_state(st)
    ost.attempts = st["k_total"]  # a state without attempts counts every iteration as one
    o = O.OracleOptions(step_mode=O.STEP_ADAPTIVE)
    for _ in range(iters):
        O.inner_step(P, ost, o)
    assert got["k_total"] == ost.k_total and got["j"] == ost.j
    assert got["attempts"] == ost.attempts == st["k_total"] + iters
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-10, key
    assert got["eta"] == pytest.approx(ost.eta, rel=1e-12)
    assert got["weight_sum"] == pytest.approx(ost.weight_sum, rel=1e-12)
    assert got["cg_total"] == ost.cg_total
    assert got["eps"] == pytest.approx(ost.eps, rel=1e-15)
    if eta_mult > 1.0 and name != "single":
        assert ost.k_total < st["k_total"] + iters  # the big start was rejected at least once


@pytest.mark.parametrize("name,tol", [("dense_small", 1e-6), ("dense_small_eq", 1e-6),
                                      ("sparse_small", 1e-4), ("ragged_eq", 1e-4),
                                      ("all_equalities", 1e-6), ("empty_rows", 1e-6),
                                      ("single", 1e-8), ("long_rows", 1e-5)])
def test_adaptive_step_end_to_end_matches_oracle(built, name, tol):
    inst, P, s = built(name)
    ores = O.solve(P, O.OracleOptions(tol=tol, step_mode=O.STEP_ADAPTIVE))
    info = s.solve(tol=tol, step_mode=L.STEP_ADAPTIVE)
    x, y = s.solution()
    assert ores.termination == O.SOLVED and info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= tol
    assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
    assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
    trace = s.trace()
    orestarts = [(r["k"], int(r["restart"]) * (2 if r["cand_avg"] else 1)) for r in ores.trace[1:]]
    if [(t["k"], t["restart"]) for t in trace] == orestarts:
        assert info["iterations"] == ores.iterations
        assert info["attempts"] == ores.state.attempts
        assert info["restarts"] == ores.restarts
        # a CG stop test (tau ||r|| <= eps_k) met at the rounding level can
        # take one step more or less without moving any decision
        assert abs(info["cg_steps"] - ores.cg_steps) <= max(2, 0.005 * ores.cg_steps)
        # the same decisions; eta moves with the iterates, so rounding drifts a
        # little further than with the fixed step (1e-8 there)
        assert _relerr(x, ores.x) <= 1e-7
    else:
        # eta is a continuous function of the iterates: over thousands of
        # attempts rounding-level differences (summation order, fused
        # multiply-adds) can move a restart decision, after which the two
        # trajectories part.  Attempt-level parity is the test above; here the
        # work and the answer must agree.
        assert abs(info["attempts"] - ores.state.attempts) <= 0.15 * ores.state.attempts + 64
        assert _relerr(x, ores.x) <= 100 * tol


@pytest.mark.parametrize("name,tol", [("dense_small", 1e-6), ("sparse_small", 1e-4),
                                      ("ragged_eq", 1e-4), ("long_rows", 1e-5),
                                      ("zipf_small", 1e-4)])
def test_adaptive_step_mixed_meets_tolerance_in_fp64(built, name, tol):
    inst, P, s = built(name)
    ores = O.solve(P, O.OracleOptions(tol=tol, step_mode=O.STEP_ADAPTIVE))
    info = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE)
    x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED
    rescored = O.relkkt(P, x, y)
    assert rescored.relkkt <= tol
    assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
    assert info["attempts"] >= info["iterations"] > 0


def test_adaptive_step_checkpoint_resume_is_bit_identical(built):
    inst, P, s = built("sparse_small")
    s.solve(tol=0.0, max_iter=256, step_mode=L.STEP_ADAPTIVE)
    full = s.get_state()
    s.solve(tol=0.0, max_iter=128, step_mode=L.STEP_ADAPTIVE)
    mid = s.get_state()
    with QPSolver(inst) as s2:
        s2.set_state(mid)
        s2.solve(tol=0.0, max_iter=256, warm_start=2, step_mode=L.STEP_ADAPTIVE)
        resumed = s2.get_state()
    for key in ("x", "y", "x_avg", "y_avg", "x_anchor", "y_anchor"):
        assert np.array_equal(full[key], resumed[key]), key
    for key in ("eta", "omega", "eps", "j", "k_total", "attempts", "weight_sum", "restarts",
                "cg_total"):
        assert full[key] == resumed[key], key


GOLDEN_ADAPTIVE = os.path.join(os.path.dirname(__file__), "golden",
                               "sparse_dd_n1000000_m500000_seed0_scaled_adaptive_trace.json")


def test_full_size_scaled_adaptive_step_matches_oracle_trace():
    """The bench instance (n = 1e6, Section 4 scaling) with the adaptive step:
    the oracle's attempts, iterations, CG steps and restarts, and its objective."""
    inst = W.sparse_dd(0)
    P = O.problem_from_instance(inst)
    with open(GOLDEN_ADAPTIVE) as f:
        g = json.load(f)
    with QPSolver(inst, scale=True) as s:
        info = s.solve(tol=1e-4, step_mode=L.STEP_ADAPTIVE)
        x, y = s.solution()
        assert info["termination"] == L.TERM_SOLVED
        rescored = O.relkkt(P, x, y)
        assert rescored.relkkt <= 1e-4
        assert info["iterations"] == g["iterations"]
        assert info["attempts"] == g["attempts"]
        assert info["restarts"] == g["restarts"]
        assert info["cg_steps"] == g["cg_steps"]
        assert rescored.primal_obj == pytest.approx(g["primal_obj"], rel=1e-4)
        mixed = s.solve(tol=1e-4, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE)
        xm, ym = s.solution()
        assert mixed["termination"] == L.TERM_SOLVED
        assert O.relkkt(P, xm, ym).relkkt <= 1e-4


# ------------------------------------------------- Section 4 augmented penalty
# QP_CREATE_PENALTY: the iteration runs on Q + rho G'G and c - rho G'q
# (G x = q the equality rows), relKKT is measured on the problem as given.
PENALTY_CASES = [("dense_small_eq", 1e-6), ("ragged_eq", 1e-4), ("all_equalities", 1e-6)]


@pytest.mark.parametrize("name,tol", PENALTY_CASES)
@pytest.mark.parametrize("scale", [False, True])
def test_penalty_matches_oracle(name, tol, scale):
    inst = CASES[name]()
    P = O.problem_from_instance(inst)
    ores = O.solve(P, O.OracleOptions(tol=tol, penalty=True, scale=scale))
    with QPSolver(inst, penalty=True, scale=scale) as s:
        assert s.penalty_rho() == pytest.approx(O.penalty_rho(P), rel=1e-12)
        info = s.solve(tol=tol)
        x, y = s.solution()
        assert ores.termination == O.SOLVED and info["termination"] == L.TERM_SOLVED
        rescored = O.relkkt(P, x, y)  # the problem as given
        assert rescored.relkkt <= tol
        assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
        assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
        assert info["iterations"] == ores.iterations and info["restarts"] == ores.restarts
        assert info["cg_steps"] == ores.cg_steps
        assert _relerr(x, ores.x) <= 1e-8
        mixed = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE)
        xm, ym = s.solution()
        assert mixed["termination"] == L.TERM_SOLVED
        assert O.relkkt(P, xm, ym).relkkt <= tol


def test_penalty_without_equality_rows_changes_nothing(built):
    inst, P, s = built("sparse_small")
    s.solve(tol=1e-4)
    x0, y0 = s.solution()
    with QPSolver(inst, penalty=True) as s2:
        assert s2.penalty_rho() == 0.0
        s2.solve(tol=1e-4)
        x1, y1 = s2.solution()
    assert np.array_equal(x0, x1) and np.array_equal(y0, y1)


def test_penalty_rejects_a_dense_equality_row():
    """A budget-like row over 20 000 variables: G'G would need 4e8 products."""
    import scipy.sparse as sp
    n = 20_000
    Q = sp.identity(n, format="csr")
    A = sp.csr_matrix(np.ones((1, n)))
    inst = W.QPInstance(n, 1, 1, Q.indptr.astype(np.int32), Q.indices.astype(np.int32), Q.data,
                        A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data,
                        np.ones(n), np.ones(1), name="dense equality row")
    with pytest.raises(L.QPError) as e:
        QPSolver(inst, penalty=True)
    assert e.value.status == 1  # QP_ERR_INVALID_ARG
    with QPSolver(inst) as s:  # without the penalty the same problem is fine
        assert s.solve(tol=1e-6)["termination"] == L.TERM_SOLVED


def test_gather_rate_measures_a_plausible_ceiling():
    """qp_gather_rate on the bench's shape (9e6 reads of a 1e6-float vector):
    positive, and no slower than the solver's own SpMV of that shape."""
    from ctypes import byref, c_double
    import torch
    lib = L.load_library()
    out = c_double()
    assert lib.qp_gather_rate(9_000_000, 1_000_000, 3, 1, byref(out)) == 0
    assert 1e10 < out.value < 1e13
    inst = W.sparse_dd(0, n=1_000_000, m=10)
    with QPSolver(inst) as s:
        s.solve(tol=0.0, max_iter=64, kernel_timing=1, precision=L.PREC_MIXED)
        info = s.solve(tol=0.0, max_iter=64, kernel_timing=1, precision=L.PREC_MIXED)
    torch.cuda.synchronize()
    spmv_rate = info["cg_kernel_spmvs"] * inst.nnz_Q / (info["cg_kernel_ms"] / 1e3)
    assert spmv_rate < 1.05 * out.value


# ------------------------------------------- variable bounds, BB x-step (Section 4)
# qp_set_bounds: with box constraints the x-step is the Barzilai-Borwein
# projected gradient; relKKT takes the bounds' reduced costs.  The oracle
# runs the same BB steps from the same points.
def _random_bounds(n, seed, frac=0.6):
    rng = np.random.default_rng(seed)
    lo = np.where(rng.random(n) < frac, -rng.uniform(0.2, 1.5, n), -np.inf)
    hi = np.where(rng.random(n) < frac, rng.uniform(0.2, 1.5, n), np.inf)
    return lo, hi


def _oracle_bounded(inst, lo, hi):
    P = O.problem_from_instance(inst)
    P.lo, P.hi = lo.copy(), hi.copy()
    return P


def _feasible_bounds(inst, seed, frac=0.6):
    """Bounds around a feasible point x_f (the oracle's solution with another,
    random cost vector), so the bounded problem stays feasible while, at its own
    optimum, many bounds are active."""
    rng = np.random.default_rng(seed)
    P = O.problem_from_instance(inst)
    P.c = rng.standard_normal(inst.n)
    xf = O.solve(P, O.OracleOptions(tol=1e-7)).x
    n = inst.n
    lo = np.where(rng.random(n) < frac, xf - rng.uniform(0.02, 0.3, n), -np.inf)
    hi = np.where(rng.random(n) < frac, xf + rng.uniform(0.02, 0.3, n), np.inf)
    return lo, hi


BB_ITER_CASES = ["dense_small", "dense_small_eq", "sparse_small", "ragged_eq", "long_rows"]


@pytest.mark.parametrize("name", BB_ITER_CASES)
@pytest.mark.parametrize("mode,iters", [("fixed3", 1), ("adaptive", 1), ("adaptive", 3)])
def test_bb_iterations_match_oracle(built, name, mode, iters):
    inst, _, s = built(name)
    lo, hi = _random_bounds(inst.n, 9)
    P = _oracle_bounded(inst, lo, hi)
    st = _shared_state(inst, P, 10)
    for key in ("x", "x_avg", "x_anchor"):
        st[key] = np.clip(st[key], lo, hi)
    s.set_bounds(lo, hi)
    try:
        s.set_state(st)
        kw = dict(cg_mode=L.CG_FIXED, cg_fixed_n=3) if mode == "fixed3" else {}
        s.iterate(iters, **kw)
        got = s.get_state()
    finally:
        s.set_bounds(None, None)
    ost = _oracle_state(st)
    o = O.OracleOptions(**({"cg_mode": O.CG_FIXED, "cg_fixed_n": 3} if mode == "fixed3" else {}))
    for _ in range(iters):
        O.inner_step(P, ost, o)
    for key in ("x", "y", "x_avg", "y_avg"):
        assert _relerr(got[key], getattr(ost, key)) <= 1e-10, key
    assert got["cg_total"] == ost.cg_total
    assert np.all(got["x"] >= lo) and np.all(got["x"] <= hi)


BOUNDED_CASES = [("dense_small", 1e-6), ("dense_small_eq", 1e-6), ("sparse_small", 1e-4),
                 ("ragged_eq", 1e-4), ("empty_rows", 1e-6)]


@pytest.mark.parametrize("name,tol", BOUNDED_CASES)
@pytest.mark.parametrize("scale", [False, True])
def test_bounds_end_to_end_matches_oracle(name, tol, scale):
    inst = CASES[name]()
    lo, hi = _feasible_bounds(inst, 11)
    P = _oracle_bounded(inst, lo, hi)
    ores = O.solve(P, O.OracleOptions(tol=tol, scale=scale))
    with QPSolver(inst, scale=scale) as s:
        s.set_bounds(lo, hi)
        info = s.solve(tol=tol)
        x, y = s.solution()
        assert ores.termination == O.SOLVED and info["termination"] == L.TERM_SOLVED
        assert np.all(x >= lo) and np.all(x <= hi)
        active = np.sum(np.isclose(x, lo, atol=1e-9) | np.isclose(x, hi, atol=1e-9))
        assert active > 0  # the bounds really bind
        rescored = O.relkkt(P, x, y)  # with the bounds' reduced costs
        assert rescored.relkkt <= tol
        assert info["relkkt"] == pytest.approx(rescored.relkkt, rel=1e-9, abs=1e-12)
        assert rescored.primal_obj == pytest.approx(ores.kkt.primal_obj, rel=1e-4, abs=1e-8)
        orestarts = [(r["k"], int(r["restart"]) * (2 if r["cand_avg"] else 1))
                     for r in ores.trace[1:]]
        if [(t["k"], t["restart"]) for t in s.trace()] == orestarts:
            assert info["iterations"] == ores.iterations and info["cg_steps"] == ores.cg_steps
            assert _relerr(x, ores.x) <= 1e-7
        else:  # projections decided at rounding level can part long trajectories
            assert abs(info["iterations"] - ores.iterations) <= 0.15 * ores.iterations + 64
            assert _relerr(x, ores.x) <= 100 * tol
        mixed = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE)
        xm, ym = s.solution()
        assert mixed["termination"] == L.TERM_SOLVED
        assert np.all(xm >= lo) and np.all(xm <= hi)
        assert O.relkkt(P, xm, ym).relkkt <= tol


def test_bounds_box_closed_form():
    """Diagonal Q, no rows, the box as bounds: x* = clip(-c/q, lo, hi)."""
    rng = np.random.default_rng(12)
    n = 300
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2
    lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    inst = W.from_dense(np.diag(q), np.zeros((0, n)), c, np.zeros(0), name="box bounds")
    with QPSolver(inst) as s:
        s.set_bounds(lo, hi)
        # FP64 to 1e-9; mixed to 1e-6 (its FP32 iterate stalls near 5e-9 here)
        for prec, tol, err in ((L.PREC_FP64, 1e-9, 1e-9), (L.PREC_MIXED, 1e-6, 1e-5)):
            info = s.solve(tol=tol, precision=prec)
            x, _ = s.solution()
            assert info["termination"] == L.TERM_SOLVED
            assert np.max(np.abs(x - np.clip(-c / q, lo, hi))) <= err


@pytest.mark.parametrize("bounded", [True, False])
def test_mixed_stall_hands_over_to_fp64(built, bounded):
    """Below the FP32 rounding floor the mixed phase stops improving; after
    mixed_stall_evals evaluations without a 10% gain FP64 refinement takes
    over and reaches a tolerance the FP32 iterate cannot (the box closed form
    with bounds; dense_small without).  With the rule off the FP32 phase runs
    into the iteration limit."""
    if bounded:
        rng = np.random.default_rng(12)
        n = 300
        q = rng.uniform(0.5, 2.0, n)
        c = rng.standard_normal(n) * 2
        lo, hi = -rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
        inst = W.from_dense(np.diag(q), np.zeros((0, n)), c, np.zeros(0), name="box bounds")
        s = QPSolver(inst)
        s.set_bounds(lo, hi)
        x_star = np.clip(-c / q, lo, hi)
        P = None
    else:
        inst, P, s = built("dense_small")
        x_star = None
    tol = 1e-10
    try:
        info = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE,
                       max_iter=200_000)
        x, y = s.solution()
        assert info["termination"] == L.TERM_SOLVED
        assert info["mixed_relkkt"] > tol          # the FP32 phase stalled above tol
        assert info["refine_iterations"] > 0       # and FP64 finished the solve
        assert info["relkkt"] <= tol
        if x_star is not None:
            assert np.max(np.abs(x - x_star)) <= 1e-9
        else:
            assert O.relkkt(P, x, y).relkkt <= tol
        off = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE,
                      max_iter=info["mixed_iterations"] + 1024, mixed_stall_evals=0)
        assert off["termination"] == L.TERM_ITER_LIMIT and off["refine_iterations"] == 0
    finally:
        if bounded:
            s.close()


def test_clearing_bounds_returns_to_the_cg_path(built):
    inst, P, s = built("dense_small")
    s.solve(tol=1e-6)
    x0, _ = s.solution()
    lo, hi = _random_bounds(inst.n, 13)
    s.set_bounds(lo, hi)
    s.solve(tol=1e-6)
    s.set_bounds(None, None)
    s.solve(tol=1e-6)
    x1, _ = s.solution()
    assert np.array_equal(x0, x1)


def test_set_bounds_rejects_invalid_bounds(built):
    inst, P, s = built("dense_small")
    n = inst.n
    with pytest.raises(L.QPError):
        s.set_bounds(np.ones(n), np.zeros(n))  # lo > hi
    with pytest.raises(L.QPError):
        s.set_bounds(np.full(n, np.inf), None)
    with pytest.raises(L.QPError):
        s.set_bounds(np.full(n, np.nan), None)
    s.set_bounds(None, None)


def test_unsorted_and_duplicate_entries_are_canonicalised():
    """qp_create accepts rows in any column order with duplicate entries
    (summed): a shuffled copy of the instance whose every tenth entry is
    split in two solves to the canonical instance's iterates."""
    inst = W.sparse_dd(3, n=5_000, m=2_500)
    rng = np.random.default_rng(4)

    def scramble(rowptr, col, val):
        rp, cs, vs = [0], [], []
        for i in range(len(rowptr) - 1):
            c = col[rowptr[i]:rowptr[i + 1]].copy()
            v = val[rowptr[i]:rowptr[i + 1]].copy()
            split = rng.random(len(c)) < 0.1
            c = np.concatenate([c, c[split]])
            v = np.concatenate([np.where(split, v * 0.5, v)[:len(split)], v[split] * 0.5])
            perm = rng.permutation(len(c))
            cs.append(c[perm])
            vs.append(v[perm])
            rp.append(rp[-1] + len(c))
        return (np.asarray(rp, np.int32), np.concatenate(cs).astype(np.int32),
                np.concatenate(vs))

    Qr, Qc, Qv = scramble(inst.Q_rowptr, inst.Q_col, inst.Q_val)
    Ar, Ac, Av = scramble(inst.A_rowptr, inst.A_col, inst.A_val)
    messy = W.QPInstance(inst.n, inst.m, inst.m_eq, Qr, Qc, Qv, Ar, Ac, Av, inst.c, inst.b)
    assert len(Qc) > len(inst.Q_col) and len(Ac) > len(inst.A_col)
    with QPSolver(inst) as a, QPSolver(messy) as b:
        ia = a.solve(tol=1e-6)
        ib = b.solve(tol=1e-6)
        xa, _ = a.solution()
        xb, _ = b.solution()
    assert ia["termination"] == ib["termination"] == L.TERM_SOLVED
    assert ia["iterations"] == ib["iterations"]
    assert _relerr(xb, xa) <= 1e-10
