"""The largest single QP of the workloads at its full size, re-scored by the oracle.

n = 10^7 variables, m = 5 * 10^6 rows: Q diagonal plus a mirrored random part
(~6 * 10^7 entries, diagonally dominant), A with 8 entries per row whose
columns follow a Zipf(1.1) popularity law (A' has rows of millions of
entries), Section 4 scaling, mixed precision and the adaptive step size, as
the benchmark runs it.  The oracle cannot solve a problem of this size in a
test, but it can score one: its FP64 relKKT of the returned (x, y), on the
problem as given, must meet the tolerance and agree with the solver's own
FP64 evaluation.  A time limit keeps a regression from running away.
"""
import math

import numpy as np
import pytest

from oracle import pdhcg_oracle as O
from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import workloads as W
from paper_2405_16160_b300.solver import QPSolver

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2405_16160_b300 import build
    build.build()


def test_largest_qp_solution_rescored_by_the_oracle():
    tol = 1e-4
    inst = W.zipf_dd(0, n=10_000_000, m=5_000_000)
    with QPSolver(inst, scale=True) as s:
        info = s.solve(tol=tol, precision=L.PREC_MIXED, step_mode=L.STEP_ADAPTIVE,
                       time_limit_s=300.0)
        x, y = s.solution()
    assert info["termination"] == L.TERM_SOLVED, info
    P = O.problem_from_instance(inst)
    k = O.relkkt(P, x, y)
    assert k.relkkt <= tol, k
    # the solver's final FP64 check and the oracle's score of the same point.
    # Both sum the objectives' ~7e7 terms (x'Qx over Q's entries, c'x, b'y) in
    # FP64, in different orders: the sums agree to about sqrt(N) u ~ 1e-12 of
    # their magnitude, so the gap term |p - d| / (1 + |p| + |d|) to about 1e-12
    # absolute, 1e-8 of a relKKT near 1e-4..1e-5.  Ten times that:
    assert info["relkkt"] == pytest.approx(k.relkkt, rel=1e-7, abs=1e-11)
    assert math.isfinite(k.primal_obj) and math.isfinite(k.dual_obj)
    assert np.all(y >= 0.0)  # every row is an inequality
    assert max(k.r_primal, k.r_dual, k.r_gap) <= tol
