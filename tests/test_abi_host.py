"""Host-side tests of the C ABI (no GPU needed).

The library must load on a machine without a GPU, export every function
include/pdhcg.h declares, agree with the ctypes mirror on struct layouts, and
do its host work (CSR validation, the stable transpose behind the explicit
A', option defaults) correctly.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import solver as S
from paper_2405_16160_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_16160_b300 import build
    build.build()
    return L.load_library()


def _declared_functions():
    text = open(L.HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(n for n, _, _ in L.SIGNATURES) == names


def test_abi_version_and_status_strings(lib):
    assert lib.qp_abi_version() == 2
    assert lib.qp_status_string(0) == b"ok"
    assert lib.qp_status_string(5) == b"device barrier timeout"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layouts_match_ctypes(tmp_path):
    structs = {"qp_options": L.QPOptionsC, "qp_info": L.QPInfoC,
               "qp_state_scalars": L.QPStateScalarsC, "qp_state_vectors": L.QPStateVectorsC,
               "qp_trace_entry": L.QPTraceEntryC, "qp_device_ctx": L.QPDeviceCtxC,
               "qp_shapes": L.QPShapesC, "qp_instance": L.QPInstanceC,
               "qp_instance_result": L.QPInstanceResultC}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdhcg.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, py in structs.items():
        assert int(got[f"{cname} size"]) == __import__("ctypes").sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
    # QPBatch passes its instance table as a numpy structured array
    dt = S._INSTANCE_DTYPE
    assert dt.itemsize == int(got["qp_instance size"])
    for f, _ in L.QPInstanceC._fields_:
        assert dt.fields[f][1] == int(got[f"qp_instance.{f}"]), f


def test_option_defaults_follow_the_paper(lib):
    o = S.QPOptions()
    # Section 4: beta_suff, beta_nec, beta_art, theta; 0.05 relKKT increments of eps_k
    assert (o.beta_suff, o.beta_nec, o.beta_art, o.theta_pw) == (0.2, 0.8, 0.2, 0.2)
    assert o.cg_eps_factor == 0.05
    assert o.power_iters == 30 and o.eval_freq == 64 and o.tol == 1e-4
    assert o.cg_mode == L.CG_ADAPTIVE and o.restart_mode == L.RESTART_ADAPTIVE
    # the mixed path's FP64 handover: 32 evaluations without a 10% relKKT gain
    assert o.refine == 1 and o.mixed_stall_evals == 32


def test_csr_validate_rejects_bad_inputs(lib):
    ok = S.csr_validate(2, 3, [0, 1, 3], [0, 1, 2], [1.0, 2.0, 3.0])
    assert ok == 0
    bad = [
        (2, 3, [1, 1, 3], [0, 1, 2], [1.0, 2.0, 3.0]),  # rowptr[0] != 0
        (2, 3, [0, 2, 1], [0, 1, 2], [1.0, 2.0, 3.0]),  # not monotone
        (2, 3, [0, 1, 3], [0, 3, 2], [1.0, 2.0, 3.0]),  # column out of range
        (2, 3, [0, 1, 3], [0, -1, 2], [1.0, 2.0, 3.0]),  # negative column
        (2, 3, [0, 1, 3], [0, 1, 2], [1.0, np.nan, 3.0]),  # NaN
        (2, 3, [0, 1, 3], [0, 1, 2], [1.0, np.inf, 3.0]),  # Inf
    ]
    for args in bad:
        assert S.csr_validate(*args) == 1, args


def test_csr_validate_accepts_any_valid_layout_and_reports_the_first_bad_entry(lib):
    """Unsorted rows, duplicates and empty rows are valid input (qp_create
    canonicalises them); on a large matrix, checked in parallel ranges, the
    error names the lowest bad entry."""
    assert S.csr_validate(4, 5, [0, 3, 3, 5, 5], [4, 0, 4, 2, 1], [1.0, 2.0, 3.0, 4.0, 5.0]) == 0
    assert S.csr_validate(3, 3, [0, 0, 0, 0], [], []) == 0
    rng = np.random.default_rng(0)
    rows, per = 200_000, 6
    rp = np.arange(0, rows * per + 1, per, dtype=np.int32)
    col = rng.integers(0, rows, rows * per).astype(np.int32)
    val = rng.standard_normal(rows * per)
    assert S.csr_validate(rows, rows, rp, col, val) == 0
    col[900_001] = rows         # out of range, late
    val[500_003] = np.inf       # non-finite, earlier
    col[700_000] = -3           # out of range, in between
    assert S.csr_validate(rows, rows, rp, col, val) == 1
    msg = L.load_library().qp_last_error().decode()
    assert "500003" in msg and "non-finite" in msg, msg


def test_csr_transpose_is_stable_and_exact(lib):
    rng = np.random.default_rng(0)
    M = sp.random(300, 170, density=0.03, random_state=1, format="csr")
    M.data = rng.standard_normal(M.nnz)
    tr, tc, tv = S.csr_transpose(300, 170, M.indptr, M.indices, M.data)
    T = sp.csr_matrix((tv, tc, tr), shape=(170, 300))
    assert (T != M.T).nnz == 0
    for j in range(170):  # entries keep increasing input-row order
        assert np.all(np.diff(tc[tr[j]:tr[j + 1]]) > 0)
    # empty matrix and empty rows
    tr, tc, tv = S.csr_transpose(3, 4, [0, 0, 0, 0], [], [])
    assert list(tr) == [0, 0, 0, 0, 0] and tc.size == 0


def test_create_validates_before_touching_a_device(lib):
    inst = W.dense_small(0)
    bad = W.dense_small(0)
    bad.c = bad.c.copy()
    bad.c[3] = np.nan
    with pytest.raises(L.QPError) as e:
        S.QPSolver(bad, torch_memory=False)
    assert e.value.status == 1
    bad2 = W.dense_small(0)
    bad2.A_col = bad2.A_col.copy()
    bad2.A_col[0] = inst.n  # out of range
    with pytest.raises(L.QPError) as e:
        S.QPSolver(bad2, torch_memory=False)
    assert e.value.status == 1
    with pytest.raises(L.QPError) as e:  # m_eq > m
        inst.m_eq = inst.m + 1
        S.QPSolver(inst, torch_memory=False)
    assert e.value.status == 1


def test_create_without_gpu_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.QPError) as e:
        S.QPSolver(W.dense_small(0), torch_memory=False)
    assert e.value.status == 6


def test_batch_create_without_gpu_reports_no_device(lib):
    """The batch binding builds its instance table (a structured array of
    addresses) for many instances and the library reports the missing
    device, on a machine without one."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    insts = W.portfolio_batch(3, count=300, n_lo=20, n_hi=60, bounds=True)
    with pytest.raises(L.QPError) as e:
        S.QPBatch(insts, torch_memory=False)
    assert e.value.status == 6


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(FileNotFoundError):
        L.load_library(str(tmp_path / "libpdhcg.so"))


def test_parallel_transpose_matches_scipy_and_is_stable(lib):
    # large enough for several worker threads (>= 2^18 entries each)
    rng = np.random.default_rng(3)
    rows, cols, per = 200_000, 150_000, 8
    colidx = np.sort(rng.integers(0, cols, size=(rows, per)), axis=1)
    keep = np.ones_like(colidx, dtype=bool)
    keep[:, 1:] = colidx[:, 1:] != colidx[:, :-1]
    counts = keep.sum(axis=1)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    col = colidx[keep].astype(np.int32)
    val = rng.standard_normal(col.size)
    tr, tc, tv = S.csr_transpose(rows, cols, rowptr, col, val)
    M = sp.csr_matrix((val, col, rowptr), shape=(rows, cols))
    ref = M.T.tocsr()
    ref.sort_indices()
    assert np.array_equal(tr, ref.indptr)
    assert np.array_equal(tc, ref.indices)  # stable: each output row in input-row order
    assert np.array_equal(tv, ref.data)


def test_gather_rate_rejects_bad_arguments(lib):
    from ctypes import byref, c_double
    out = c_double()
    assert lib.qp_gather_rate(0, 10, 1, 1, byref(out)) == 1  # QP_ERR_INVALID_ARG
    assert lib.qp_gather_rate(10, 0, 1, 1, byref(out)) == 1
    assert lib.qp_gather_rate(10, 10, 1, 1, None) == 1


def test_tuner_rejects_bad_arguments(lib):
    from ctypes import byref
    out = L.QPShapesC()
    assert lib.qp_tune(None, 10, byref(out)) == 1  # QP_ERR_INVALID_ARG
    assert lib.qp_get_shapes(None, byref(out)) == 1
