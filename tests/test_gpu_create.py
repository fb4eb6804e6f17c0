"""qp_create's checks of the problem on the device.

With a device visible, qp_create copies Q, A, c and b as given and checks
their entries there (row pointers monotone, columns in range, values finite,
rows sorted); with QP_CREATE_CHECK_SYMMETRY (or without a device) the host
checks them first.  Both must report the same error with the same message
(the first failure: Q before A before c before b, row pointers before
entries, the lowest index), and a problem with unsorted rows or duplicate
entries must be solved as its canonical form either way.
"""
import dataclasses

import numpy as np
import pytest

from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import workloads as W
from paper_2405_16160_b300.solver import QPSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2405_16160_b300 import build
    build.build()


def _error(inst, **kw):
    with pytest.raises(L.QPError) as e:
        QPSolver(inst, torch_memory=False, **kw)
    return e.value


def _both_paths(inst):
    """The device check's error and the host check's (the symmetry flag keeps
    the host path; the instances are symmetric, so it adds no error)."""
    dev, host = _error(inst), _error(inst, check_symmetry=True)
    assert dev.status == host.status == 1
    assert str(dev) == str(host)
    return str(dev)


def _copy(inst, **arrays):
    return dataclasses.replace(inst, **{k: v.copy() for k, v in arrays.items()})


BASE = W.sparse_dd(5, n=3000, m=1200)


def test_non_finite_and_out_of_range_entries():
    inst = _copy(BASE, Q_val=BASE.Q_val, A_col=BASE.A_col, A_val=BASE.A_val)
    inst.Q_val[4011] = np.inf
    inst.A_col[900] = inst.n           # out of range, later
    inst.A_val[37] = np.nan            # non-finite, earlier in A
    msg = _both_paths(inst)
    assert "Q: non-finite value at entry 4011" in msg, msg  # Q before A
    inst.Q_val[4011] = 1.0
    msg = _both_paths(inst)
    assert "A: non-finite value at entry 37" in msg, msg    # the lowest entry of A
    inst.A_val[37] = 1.0
    msg = _both_paths(inst)
    assert "A: column index out of range at entry 900" in msg, msg
    inst.A_col[900] = -1
    assert "entry 900" in _both_paths(inst)


def test_row_pointers_before_entries():
    inst = _copy(BASE, Q_rowptr=BASE.Q_rowptr, Q_val=BASE.Q_val)
    inst.Q_val[3] = np.nan
    r = inst.Q_rowptr
    r[12], r[13] = r[13], r[12]        # rows 11 and 12 run backwards
    msg = _both_paths(inst)
    assert "Q: rowptr is not monotone at row" in msg, msg


def test_c_and_b():
    inst = _copy(BASE, c=BASE.c, b=BASE.b)
    inst.b[7] = np.inf
    inst.c[2999] = np.nan
    assert "c[2999] is not finite" in _both_paths(inst)
    inst.c[2999] = 0.0
    assert "b[7] is not finite" in _both_paths(inst)


def test_unsorted_rows_and_duplicates_solve_as_the_canonical_problem():
    """Rows reversed, and the first entry of every row of Q split in two
    halves: the device check finds them not canonical and the host's
    canonical copy (sorted, duplicates summed) is what gets solved."""
    inst = BASE
    n = inst.n
    rows_q, cols_q, vals_q = [], [], []
    for i in range(n):
        s, e = inst.Q_rowptr[i], inst.Q_rowptr[i + 1]
        cols = list(inst.Q_col[s:e][::-1])
        vals = list(inst.Q_val[s:e][::-1])
        cols.append(cols[-1])            # the row's first column, twice
        vals[-1] *= 0.5
        vals.append(vals[-1])
        rows_q.append(len(cols))
        cols_q += cols
        vals_q += vals
    rp = np.concatenate([[0], np.cumsum(rows_q)]).astype(np.int32)
    messy = dataclasses.replace(inst, Q_rowptr=rp, Q_col=np.array(cols_q, dtype=np.int32),
                                Q_val=np.array(vals_q))
    with QPSolver(inst) as s:
        ref = s.solve(tol=1e-6)
        x0, y0 = s.solution()
    with QPSolver(messy) as s:
        got = s.solve(tol=1e-6)
        x1, y1 = s.solution()
    assert got["iterations"] == ref["iterations"]
    assert np.max(np.abs(x1 - x0)) <= 1e-12 * max(1.0, np.max(np.abs(x0)))
    assert np.max(np.abs(y1 - y0)) <= 1e-12 * max(1.0, np.max(np.abs(y0)))


def _rule_lanes(lens, fp32, cg=False):
    """The mean-row-length rule of qp_create: the mean over the rows of at
    most 64 entries when some rows are longer, else over all rows; FP32 Q
    (cg, its products in the CG kernel) takes the fewest lanes G with a mean
    of at most 8 G entries."""
    short = lens <= 64
    if 0 < short.sum() < lens.size:
        avg = lens[short].sum() / short.sum()
    else:
        avg = lens.sum() / max(lens.size, 1)
    if fp32 and cg:
        steps = [(8.0, 1), (16.0, 2), (32.0, 4), (64.0, 8)]
    elif fp32:
        steps = [(3.0, 1), (6.0, 2), (20.0, 4), (64.0, 8)]
    else:
        steps = [(24.0, 1), (64.0, 4), (256.0, 8)]
    for bound, g in steps:
        if avg <= bound:
            return g
    return 32


@pytest.mark.parametrize("make", [lambda: W.sparse_dd(1, n=30_000, m=12_000),
                                  lambda: W.zipf_dd(1, n=40_000, m=20_000),
                                  lambda: W.dense_small(0)],
                         ids=["uniform", "power_law", "dense"])
def test_row_census_gives_the_rule_of_the_row_lengths(make):
    """The row counts behind the lanes per row are taken on the device; the
    choice must be the rule applied to the row lengths of Q, A and A', and
    the row layouts the rule's: warp ranges for Q, grid-stride groups for A
    and A'."""
    inst = make()
    lens = [np.diff(inst.Q_rowptr), np.diff(inst.A_rowptr),
            np.bincount(inst.A_col, minlength=inst.n)]
    with QPSolver(inst) as s:
        sh = s.shapes()
    rule = sh["lanes_rule"]
    for p, fp32 in ((0, False), (1, True)):
        assert rule[p] == [_rule_lanes(l, fp32, k == 0) for k, l in enumerate(lens)], (p, rule)
        assert sh["lanes"][p] == rule[p]
        assert sh["layout"][p] == [1, 0, 0], sh["layout"]
