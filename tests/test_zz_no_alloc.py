"""qp_norm_A_static: the allocation-free ||A||_2 estimate, checked against
qp_norm_A and against the CPU oracle's power iteration.

Callers that cannot allocate device memory (a control loop held to a memory
budget fixed at start-up, code running while another framework owns all
device memory, code that must not risk an allocation's device-wide
synchronisation) use qp_norm_A_static, which keeps its work vectors in a
static device array.  This file is collected last so that a failure here
does not hide the rest of the suite; it also passes when run on its own.
"""
import ctypes

import numpy as np
import pytest

from oracle import pdhcg_oracle as O
from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import workloads as W
from paper_2405_16160_b300.solver import QPSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2405_16160_b300 import build
    build.build()
    return torch


def _device_csr(torch, inst):
    A = inst.scipy_A().tocsr()
    A.sort_indices()
    At = A.T.tocsr()
    At.sort_indices()
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return [dev(A.indptr, np.int32), dev(A.indices, np.int32), dev(A.data, np.float64),
            dev(At.indptr, np.int32), dev(At.indices, np.int32), dev(At.data, np.float64)], A.nnz


def _static_norm(torch, lib, inst, iters=30):
    arrs, nnz = _device_csr(torch, inst)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.qp_norm_A_static(inst.m, inst.n, nnz, *[a.data_ptr() for a in arrs], iters,
                              out.data_ptr(), stream.cuda_stream)
    L.check(st, "qp_norm_A_static")
    stream.synchronize()
    return float(out.item())


def test_static_norm_matches_handle_norm_on_two_calls(torch_cuda):
    lib = L.load_library()
    cases = [W.sparse_dd(11, n=30_000, m=12_000), W.dense_small(12, m_eq=5)]
    for inst in cases:  # two calls in a row on different problems share the array
        got = _static_norm(torch_cuda, lib, inst)
        with QPSolver(inst) as s:
            ref = s.norm_A(30)
        assert got == pytest.approx(ref, rel=1e-12)
        # the same 30 power iterations from the normalised all-ones vector, in
        # FP64 on the CPU (Section 3.2's ||A||_2 of the step size)
        assert got == pytest.approx(O.spectral_norm(inst.scipy_A().tocsr(), 30), rel=1e-12)


def test_static_norm_rejects_sizes_beyond_its_scratch(torch_cuda):
    lib = L.load_library()
    one = torch_cuda.zeros(2, dtype=torch_cuda.int32, device="cuda")
    out = torch_cuda.zeros(1, dtype=torch_cuda.float64, device="cuda")
    n = L.QP_NORM_A_STATIC_MAX_DOUBLES // 2  # 2n alone exceeds the capacity
    st = lib.qp_norm_A_static(0, n, 0, one.data_ptr(), None, None, one.data_ptr(), None, None, 30,
                              out.data_ptr(), None)
    assert st == 1
    assert b"exceeds the static scratch limit" in lib.qp_last_error()
