"""Pins for the oracle's restart and primal-weight control.

Section 4 of the paper fixes three things here and this file checks each
against values worked out by hand:

* "Adaptive restart": the rule of the cited rAPDHG (its Section 6) with
  beta_sufficient = 0.2, beta_necessary = 0.8 and beta_artificial = 0.2.  A
  restart to the candidate happens when (i) its relKKT is at most
  beta_sufficient times the relKKT of the epoch's restart point, or (ii) it is
  at most beta_necessary times that value and above the candidate's value at
  the previous evaluation (progress has stalled), or (iii) the epoch has run
  for at least beta_artificial times the total iteration count.  The
  candidate is the lower-relKKT one of the current iterate and the average.
* "Primal weight adjustment": at the start of an epoch, with theta = 0.2 and
  Delta x, Delta y the distances between consecutive restart points,
  omega <- exp(theta log(Delta y / Delta x) + (1 - theta) log omega) when
  both distances exceed eps_zero, else omega is kept.  (The printed formula
  has no log on the old omega; the pin below shows that the literal reading
  would not even keep omega fixed when Delta y / Delta x = omega.)
* The starting weight omega_0 = ||c||_2 / ||b||_2 (1 when either norm is
  below eps_zero) with tau = eta / omega and sigma = eta * omega, eta =
  1 / (2 ||A||_2) (Section 3.2).

Every expected value below is written out with its arithmetic.  The last
group plants a mistake in each function and checks that a pin catches it.
"""
import math
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhcg_oracle as O

INF = math.inf

# (kkt_cand, kkt_anchor, kkt_prev_cand, j, k_total, restart?, why)
# anchor 0.5: beta_suff * 0.5 = 0.1, beta_nec * 0.5 = 0.4; k_total 100:
# beta_art * 100 = 20 iterations.
DECISION_TABLE = [
    (0.1, 0.5, INF, 1, 100, True, "(i) at equality: 0.1 <= 0.2 * 0.5"),
    (0.09, 0.5, INF, 1, 100, True, "(i): 0.09 <= 0.1"),
    (0.1000001, 0.5, INF, 1, 100, False, "just above (i); no rise for (ii); 1 < 20 for (iii)"),
    (0.3, 0.5, INF, 1, 100, False, "0.3 <= 0.4 but nothing to rise from (first evaluation of the epoch)"),
    (0.3, 0.5, 0.25, 1, 100, True, "(ii): 0.3 <= 0.4 and 0.3 > 0.25"),
    (0.4, 0.5, 0.35, 1, 100, True, "(ii) at equality of the bound: 0.4 <= 0.8 * 0.5, 0.4 > 0.35"),
    (0.41, 0.5, 0.35, 1, 100, False, "(ii) fails on the bound: 0.41 > 0.4, though it rose"),
    (0.3, 0.5, 0.3, 1, 100, False, "(ii) needs a strict rise: 0.3 == 0.3"),
    (0.3, 0.5, 0.35, 1, 100, False, "still falling: 0.3 < 0.35"),
    (0.45, 0.5, 0.3, 20, 100, True, "(iii) at equality: 20 >= 0.2 * 100"),
    (0.45, 0.5, 0.3, 19, 100, False, "(iii) fails: 19 < 20; (i), (ii) fail on their bounds"),
    (0.45, 0.5, 0.3, 100, 500, True, "(iii): 100 >= 0.2 * 500"),
    (0.45, 0.5, 0.3, 99, 500, False, "(iii) fails: 99 < 100"),
    (0.6, 0.5, 0.3, 64, 64, True, "(iii): the first epoch's first evaluation, j = k_total"),
    (2.0, 0.5, 0.3, 5, 100, False, "relKKT far above the anchor: no test holds"),
]


def _state(n=2, m=1, **kw):
    z = lambda k: np.zeros(k)
    st = O.OracleState(z(n), z(m), z(n), z(m), z(n), z(m), eta=0.1, omega=1.0)
    for k, v in kw.items():
        setattr(st, k, v)
    return st


def _table_mismatches(restart_test):
    o = O.OracleOptions()
    bad = []
    for cand, anchor, prev, j, k, want, why in DECISION_TABLE:
        st = _state(kkt_anchor=anchor, kkt_prev_cand=prev, j=j, k_total=k)
        if bool(restart_test(cand, st, o)) != want:
            bad.append(why)
    return bad


def test_paper_constants_are_the_defaults():
    o = O.OracleOptions()
    assert (o.beta_suff, o.beta_nec, o.beta_art, o.theta_pw) == (0.2, 0.8, 0.2, 0.2)
    assert o.eps_zero == 1e-10


def test_restart_decision_table():
    assert _table_mismatches(O.restart_test) == []


class _FakeKKT:
    """relKKT values chosen per evaluation, for the current iterate (the
    arrays st.x / st.y) and for the average (st.x_avg / st.y_avg)."""

    def __init__(self, st):
        self.st, self.cur, self.avg = st, None, None

    def __call__(self, x, y):
        v = self.avg if x is self.st.x_avg else self.cur
        return SimpleNamespace(relkkt=v)


def test_evaluation_sequence_worked_by_hand():
    # One epoch watched over five evaluations (eval_freq 64) with the primal
    # weight update off; k_total is large so that (iii) only fires where the
    # table says.  Each line: the two relKKT values, the candidate, the tests.
    P = O.OracleProblem(sp.csr_matrix(np.eye(2)), sp.csr_matrix(np.ones((1, 2))),
                        np.zeros(2), np.ones(1), 0)
    o = O.OracleOptions(tol=1e-4, primal_weight_update=False)
    st = _state(kkt_anchor=1.0, kkt_prev_cand=INF, j=64, k_total=1000)
    st.x, st.x_avg = np.array([1.0, 2.0]), np.array([3.0, 4.0])
    st.y, st.y_avg = np.array([5.0]), np.array([6.0])
    fk = _FakeKKT(st)
    rec = []

    def ev(cur, avg):
        fk.cur, fk.avg = cur, avg
        return O.evaluate(P, st, o, rec, fk)

    # E1: cur 0.9, avg 0.85 -> candidate avg 0.85.  (i) 0.85 > 0.2; (ii) 0.85 > 0.8;
    # (iii) 64 < 200.  No restart; prev <- 0.85; relkkt_last <- cur 0.9.
    done, best, use_avg = ev(0.9, 0.85)
    assert (done, best.relkkt, use_avg, rec[-1]["restart"]) == (False, 0.85, True, False)
    assert (st.kkt_prev_cand, st.relkkt_last, st.kkt_anchor) == (0.85, 0.9, 1.0)
    # E2: cur 0.75, avg 0.78 -> candidate cur 0.75.  (ii) 0.75 <= 0.8 but
    # 0.75 < 0.85 (still falling).  No restart; prev <- 0.75.
    st.j, st.k_total = 128, 1064
    done, best, use_avg = ev(0.75, 0.78)
    assert (done, best.relkkt, use_avg, rec[-1]["restart"]) == (False, 0.75, False, False)
    assert st.kkt_prev_cand == 0.75
    # E3: cur 0.79, avg 0.77 -> candidate avg 0.77.  (ii) 0.77 <= 0.8 and
    # 0.77 > 0.75: restart to the average.  Anchor <- 0.77, prev <- inf, j <- 0,
    # (x, y) and the anchors <- the average, CG precision reset.
    st.j, st.k_total, st.eps = 192, 1128, 0.3
    done, best, use_avg = ev(0.79, 0.77)
    assert (done, best.relkkt, use_avg, rec[-1]["restart"], rec[-1]["cand_avg"]) == \
        (False, 0.77, True, True, True)
    assert (st.kkt_anchor, st.kkt_prev_cand, st.relkkt_last, st.j, st.eps, st.n_restarts) == \
        (0.77, INF, 0.77, 0, 0.0, 1)
    assert np.array_equal(st.x, [3.0, 4.0]) and np.array_equal(st.x_anchor, [3.0, 4.0])
    assert np.array_equal(st.y, [6.0]) and np.array_equal(st.y_anchor, [6.0])
    # E4: a tie, cur = avg = 0.1 -> the average is the candidate.  (i) 0.1 <= 0.154.
    st.j, st.k_total = 64, 1192
    st.x_avg, st.y_avg = np.array([7.0, 8.0]), np.array([9.0])
    done, best, use_avg = ev(0.1, 0.1)
    assert (done, use_avg, rec[-1]["restart"]) == (False, True, True)
    assert st.kkt_anchor == 0.1 and np.array_equal(st.x, [7.0, 8.0])
    # E5: cur 5e-5 <= tol 1e-4 -> done with the current iterate; nothing else moves.
    st.j, st.k_total = 64, 1256
    done, best, use_avg = ev(5e-5, 2e-4)
    assert (done, best.relkkt, use_avg) == (True, 5e-5, False)
    assert st.n_restarts == 2 and st.kkt_anchor == 0.1


def _pw_state(dx_vec, dy_vec, omega):
    # anchors at 1.5 and -2.0 where the distances survive the subtraction
    # exactly, at 0 for the cases at the eps_zero boundary
    tiny = min(np.abs(np.asarray(dx_vec + dy_vec))[np.nonzero(dx_vec + dy_vec)]) < 1e-6
    st = _state(n=len(dx_vec), m=len(dy_vec), omega=omega)
    st.x_anchor = np.full(len(dx_vec), 0.0 if tiny else 1.5)
    st.y_anchor = np.full(len(dy_vec), 0.0 if tiny else -2.0)
    st.x = st.x_anchor + np.asarray(dx_vec, float)
    st.y = st.y_anchor + np.asarray(dy_vec, float)
    st.x_avg, st.y_avg = st.x.copy(), st.y.copy()
    return st


def _pw_after(restart_to, dx_vec, dy_vec, omega):
    P = O.OracleProblem(sp.csr_matrix(np.eye(len(dx_vec))),
                        sp.csr_matrix(np.ones((len(dy_vec), len(dx_vec)))),
                        np.zeros(len(dx_vec)), np.ones(len(dy_vec)), 0)
    st = _pw_state(dx_vec, dy_vec, omega)
    restart_to(P, st, O.OracleOptions(), False, 0.5)
    return st


PW_CASES = [
    # (dx, dy, omega_old, omega_new, arithmetic)
    ([3.0, 4.0], [12.0, 16.0], 2.0, 2.0 ** 1.2,
     "dx 5, dy 20: exp(0.2 log 4 + 0.8 log 2) = 2^0.4 * 2^0.8 = 2^1.2"),
    ([0.0, 2.0], [0.0, 2.0], 5.0, 5.0 ** 0.8,
     "dx = dy = 2: exp(0.2 log 1 + 0.8 log 5) = 5^0.8"),
    ([1.0, 0.0], [0.0, 3.0], 3.0, 3.0,
     "dy/dx = 3 = omega: the update keeps omega (a fixed point)"),
    ([1e-11, 0.0], [0.0, 7.0], 2.0, 2.0, "dx = 1e-11 <= eps_zero: omega kept"),
    ([4.0, 0.0], [0.0, 0.0], 2.0, 2.0, "dy = 0: omega kept"),
    ([1e-10, 0.0], [0.0, 1.0], 2.0, 2.0, "dx = eps_zero exactly: not above it, omega kept"),
]


@pytest.mark.parametrize("dx,dy,old,new,why", PW_CASES)
def test_primal_weight_update_worked_by_hand(dx, dy, old, new, why):
    st = _pw_after(O.restart_to, dx, dy, old)
    assert st.omega == pytest.approx(new, rel=1e-14), why
    # tau = eta / omega and sigma = eta * omega follow the new weight
    assert st.tau == pytest.approx(0.1 / new, rel=1e-14)
    assert st.sigma == pytest.approx(0.1 * new, rel=1e-14)


def test_primal_weight_update_just_above_eps_zero():
    # dx = 2e-10 > eps_zero, dy = 8e-10: exp(0.2 log 4 + 0.8 log 1) = 4^0.2
    st = _pw_after(O.restart_to, [2e-10, 0.0], [0.0, 8e-10], 1.0)
    assert st.omega == pytest.approx(4.0 ** 0.2, rel=1e-12)


def test_primal_weight_distances_are_to_the_previous_restart_point():
    # restart to the average: the distances are avg - anchor, not cur - anchor
    P = O.OracleProblem(sp.csr_matrix(np.eye(2)), sp.csr_matrix(np.ones((1, 2))),
                        np.zeros(2), np.ones(1), 0)
    st = _state(omega=1.0)
    st.x_anchor, st.y_anchor = np.zeros(2), np.zeros(1)
    st.x, st.y = np.array([100.0, 0.0]), np.array([1.0])           # cur: dx 100, dy 1
    st.x_avg, st.y_avg = np.array([0.0, 1.0]), np.array([32.0])    # avg: dx 1, dy 32
    O.restart_to(P, st, O.OracleOptions(), True, 0.5)
    assert st.omega == pytest.approx(32.0 ** 0.2, rel=1e-14)  # exp(0.2 log 32) = 2
    assert st.omega == pytest.approx(2.0, rel=1e-14)


OMEGA0_CASES = [
    # (c, b, omega0 option, expected omega_0, arithmetic)
    ([3.0, 4.0], [1.0, 2.0, 2.0], 0.0, 5.0 / 3.0, "||c|| = 5, ||b|| = 3"),
    ([0.0, 0.0], [1.0, 2.0, 2.0], 0.0, 1.0, "c = 0: 1"),
    ([3.0, 4.0], [0.0, 0.0, 0.0], 0.0, 1.0, "b = 0: 1"),
    ([3.0, 4.0], [1e-11, 0.0, 0.0], 0.0, 1.0, "||b|| = 1e-11 <= eps_zero: 1"),
    ([3.0, 4.0], [1.0, 2.0, 2.0], 7.0, 7.0, "an explicit omega_0 wins"),
]


@pytest.mark.parametrize("c,b,opt,want,why", OMEGA0_CASES)
def test_initial_primal_weight_rule(c, b, opt, want, why):
    # A = u v' with u = (1, 0, 0), v = (3, 4): ||A||_2 = ||u|| ||v|| = 5 exactly,
    # so eta = 1 / (2 * 5) = 0.1
    A = sp.csr_matrix(np.array([[3.0, 4.0], [0.0, 0.0], [0.0, 0.0]]))
    P = O.OracleProblem(sp.csr_matrix(np.eye(2)), A, np.array(c), np.array(b), 0)
    st = O.initial_state(P, O.OracleOptions(omega0=opt))
    assert st.omega == pytest.approx(want, rel=1e-15), why
    assert st.eta == pytest.approx(0.1, rel=1e-14)
    assert st.tau == pytest.approx(0.1 / want, rel=1e-14)
    assert st.sigma == pytest.approx(0.1 * want, rel=1e-14)
    assert not st.x.any() and not st.y.any() and not st.x_avg.any() and st.j == 0


# ---------------------------------------------------------------- planted mistakes
def _swapped_betas(kkt_cand, st, o):
    if kkt_cand <= o.beta_nec * st.kkt_anchor:
        return True
    if kkt_cand <= o.beta_suff * st.kkt_anchor and kkt_cand > st.kkt_prev_cand:
        return True
    return st.j >= o.beta_art * st.k_total


def _no_rise_clause(kkt_cand, st, o):
    if kkt_cand <= o.beta_suff * st.kkt_anchor:
        return True
    if kkt_cand <= o.beta_nec * st.kkt_anchor:
        return True
    return st.j >= o.beta_art * st.k_total


def _rise_reversed(kkt_cand, st, o):
    if kkt_cand <= o.beta_suff * st.kkt_anchor:
        return True
    if kkt_cand <= o.beta_nec * st.kkt_anchor and kkt_cand < st.kkt_prev_cand:
        return True
    return st.j >= o.beta_art * st.k_total


def _counters_swapped(kkt_cand, st, o):
    if kkt_cand <= o.beta_suff * st.kkt_anchor:
        return True
    if kkt_cand <= o.beta_nec * st.kkt_anchor and kkt_cand > st.kkt_prev_cand:
        return True
    return st.k_total >= o.beta_art * st.j


def _strict_bounds(kkt_cand, st, o):
    if kkt_cand < o.beta_suff * st.kkt_anchor:
        return True
    if kkt_cand < o.beta_nec * st.kkt_anchor and kkt_cand > st.kkt_prev_cand:
        return True
    return st.j > o.beta_art * st.k_total


@pytest.mark.parametrize("mutant", [_swapped_betas, _no_rise_clause, _rise_reversed,
                                    _counters_swapped, _strict_bounds])
def test_planted_restart_mistakes_are_caught(mutant):
    assert _table_mismatches(mutant), f"{mutant.__name__} went unnoticed"


def _mutant_restart_to(kind):
    def restart_to(P, st, o, use_avg, kkt_cand):
        xc = st.x_avg.copy() if use_avg else st.x.copy()
        yc = st.y_avg.copy() if use_avg else st.y.copy()
        dx = float(np.linalg.norm(xc - st.x_anchor))
        dy = float(np.linalg.norm(yc - st.y_anchor))
        if dx > o.eps_zero and dy > o.eps_zero:
            if kind == "printed_literally":  # (1 - theta) omega inside exp, no log
                st.omega = math.exp(o.theta_pw * math.log(dy / dx) + (1 - o.theta_pw) * st.omega)
            elif kind == "theta_swapped":
                st.omega = math.exp((1 - o.theta_pw) * math.log(dy / dx)
                                    + o.theta_pw * math.log(st.omega))
            elif kind == "ratio_inverted":
                st.omega = math.exp(o.theta_pw * math.log(dx / dy)
                                    + (1 - o.theta_pw) * math.log(st.omega))
            elif kind == "squared_distances":
                st.omega = math.exp(o.theta_pw * math.log(dy * dy / (dx * dx))
                                    + (1 - o.theta_pw) * math.log(st.omega))
        st.x, st.y = xc, yc
        st.x_anchor, st.y_anchor = xc.copy(), yc.copy()
        st.j, st.eps, st.kkt_anchor, st.kkt_prev_cand = 0, 0.0, kkt_cand, math.inf
    return restart_to


@pytest.mark.parametrize("kind", ["printed_literally", "theta_swapped", "ratio_inverted",
                                  "squared_distances"])
def test_planted_primal_weight_mistakes_are_caught(kind):
    caught = False
    for dx, dy, old, new, _ in PW_CASES:
        st = _pw_after(_mutant_restart_to(kind), dx, dy, old)
        caught |= not math.isclose(st.omega, new, rel_tol=1e-12)
    assert caught, f"{kind} went unnoticed"


def test_planted_omega0_mistake_is_caught(monkeypatch):
    real = O.initial_state

    def inverted(P, o):
        st = real(P, o)
        nc, nb = float(np.linalg.norm(P.c)), float(np.linalg.norm(P.b))
        if o.omega0 <= 0 and nc > o.eps_zero and nb > o.eps_zero:
            st.omega = nb / nc  # ||b|| / ||c|| instead of ||c|| / ||b||
        return st

    monkeypatch.setattr(O, "initial_state", inverted)
    c, b, opt, want, _ = OMEGA0_CASES[0]
    A = sp.csr_matrix(np.array([[3.0, 4.0], [0.0, 0.0], [0.0, 0.0]]))
    P = O.OracleProblem(sp.csr_matrix(np.eye(2)), A, np.array(c), np.array(b), 0)
    assert not math.isclose(O.initial_state(P, O.OracleOptions(omega0=opt)).omega, want,
                            rel_tol=1e-12)
