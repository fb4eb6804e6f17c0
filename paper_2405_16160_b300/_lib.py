"""ctypes mirror of include/pdhcg.h.  Marshalling only: no solver arithmetic here."""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_float, c_int32, c_int64,
                    c_size_t, c_uint32, c_uint64, c_void_p)

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpdhcg.so")
HEADER_PATH = os.path.join(os.path.dirname(PKG), "include", "pdhcg.h")

QP_OK = 0
STATUS_NAMES = {0: "QP_OK", 1: "QP_ERR_INVALID_ARG", 2: "QP_ERR_OOM", 3: "QP_ERR_CUDA",
                4: "QP_ERR_NOT_SOLVED", 5: "QP_ERR_DEVICE_TIMEOUT", 6: "QP_ERR_NO_DEVICE"}
TERM_NONE, TERM_SOLVED, TERM_ITER_LIMIT, TERM_TIME_LIMIT, TERM_NUMERICAL = -1, 0, 1, 2, 3
CG_ADAPTIVE, CG_FIXED = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
RESTART_ADAPTIVE, RESTART_NONE = 0, 2
STEP_FIXED, STEP_ADAPTIVE = 0, 1
CREATE_CHECK_SYMMETRY = 1
CREATE_SCALE = 2
CREATE_PENALTY = 4
DEBUG_BARRIER_NEVER_RELEASES = 1
QP_NORM_A_STATIC_MAX_DOUBLES = 1 << 20  # capacity of qp_norm_A_static's static scratch


class QPOptionsC(Structure):
    _fields_ = [
        ("tol", c_double), ("max_iter", c_int64), ("time_limit_s", c_double),
        ("eval_freq", c_int32), ("cg_mode", c_int32), ("cg_fixed_n", c_int32), ("cg_max", c_int32),
        ("cg_eps_factor", c_double), ("restart_mode", c_int32), ("power_iters", c_int32),
        ("beta_suff", c_double), ("beta_nec", c_double), ("beta_art", c_double),
        ("theta_pw", c_double), ("eps_zero", c_double), ("primal_weight_update", c_int32),
        ("warm_start", c_int32), ("omega0", c_double), ("eta", c_double),
        ("kernel_timing", c_int32), ("debug_flags", c_uint32), ("precision", c_int32),
        ("refine", c_int32), ("step_mode", c_int32), ("mixed_stall_evals", c_int32),
        ("reserved", c_int64 * 6),
    ]


class QPInfoC(Structure):
    _fields_ = [
        ("termination", c_int32), ("returned_avg", c_int32), ("iterations", c_int64),
        ("cg_steps", c_int64), ("restarts", c_int64), ("evaluations", c_int64),
        ("relkkt", c_double), ("r_primal", c_double), ("r_dual", c_double), ("r_gap", c_double),
        ("primal_obj", c_double), ("dual_obj", c_double), ("norm_A", c_double), ("eta", c_double),
        ("omega", c_double), ("tau", c_double), ("sigma", c_double), ("setup_ms", c_double),
        ("solve_ms", c_double), ("cg_kernel_ms", c_double), ("cg_kernel_launches", c_int64),
        ("cg_kernel_spmvs", c_int64), ("device_error", c_int32), ("cooperative", c_int32),
        ("precision", c_int32), ("pad0", c_int32), ("mixed_iterations", c_int64),
        ("refine_iterations", c_int64), ("mixed_relkkt", c_double), ("check_relkkt", c_double),
        ("attempts", c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class QPStateScalarsC(Structure):
    _fields_ = [
        ("eta", c_double), ("omega", c_double), ("eps", c_double), ("relkkt_last", c_double),
        ("kkt_anchor", c_double), ("kkt_prev_cand", c_double), ("j", c_int64),
        ("k_total", c_int64), ("restarts", c_int64), ("cg_total", c_int64),
        ("attempts", c_int64), ("weight_sum", c_double),
    ]


class QPStateVectorsC(Structure):
    _fields_ = [("x", POINTER(c_double)), ("y", POINTER(c_double)), ("x_avg", POINTER(c_double)),
                ("y_avg", POINTER(c_double)), ("x_anchor", POINTER(c_double)),
                ("y_anchor", POINTER(c_double))]


class QPTraceEntryC(Structure):
    _fields_ = [("k", c_int64), ("kkt_cur", c_double), ("kkt_avg", c_double), ("omega", c_double),
                ("restart", c_int32), ("cg_last", c_int32)]


class QPInstanceC(Structure):
    _fields_ = [("n", c_int32), ("m", c_int32), ("m_eq", c_int32), ("k", c_int32),
                ("F", POINTER(c_double)), ("qd", POINTER(c_double)),
                ("A_rowptr", POINTER(c_int32)), ("A_col", POINTER(c_int32)),
                ("A_val", POINTER(c_double)), ("c", POINTER(c_double)), ("b", POINTER(c_double))]


class QPInstanceResultC(Structure):
    _fields_ = [("termination", c_int32), ("returned_avg", c_int32), ("iterations", c_int64),
                ("cg_steps", c_int64), ("restarts", c_int64), ("r_primal", c_double),
                ("r_dual", c_double), ("r_gap", c_double), ("relkkt", c_double),
                ("primal_obj", c_double), ("dual_obj", c_double), ("eta", c_double),
                ("omega", c_double), ("norm_A", c_double), ("attempts", c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class QPShapesC(Structure):
    _fields_ = [("lanes", (c_int32 * 3) * 2), ("lanes_rule", (c_int32 * 3) * 2),
                ("layout", (c_int32 * 3) * 2), ("product_us", (c_double * 3) * 2), ("product_us_rule", (c_double * 3) * 2),
                ("waves", c_int32), ("tuned", c_int32), ("waves_us", c_double * 3)]

    def as_dict(self) -> dict:
        grid = lambda a: [list(row) for row in a]
        return {"lanes": grid(self.lanes), "lanes_rule": grid(self.lanes_rule),
                "layout": grid(self.layout),
                "product_us": grid(self.product_us),
                "product_us_rule": grid(self.product_us_rule), "waves": self.waves,
                "tuned": self.tuned, "waves_us": list(self.waves_us)}


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class QPDeviceCtxC(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p), ("stream", c_void_p)]


_I32P = POINTER(c_int32)
_F64P = POINTER(c_double)
_H = c_void_p

# (name, restype, argtypes) for every function declared in include/pdhcg.h
SIGNATURES = [
    ("qp_status_string", c_char_p, [c_int32]),
    ("qp_abi_version", c_int32, []),
    ("qp_last_error", c_char_p, []),
    ("qp_options_default", None, [POINTER(QPOptionsC)]),
    ("qp_create", c_int32, [POINTER(_H), c_int32, c_int32, c_int32, _I32P, _I32P, _F64P, _I32P,
                            _I32P, _F64P, _F64P, _F64P, POINTER(QPDeviceCtxC), c_uint32]),
    ("qp_destroy", None, [_H]),
    ("qp_solve", c_int32, [_H, POINTER(QPOptionsC), POINTER(QPInfoC)]),
    ("qp_get_solution", c_int32, [_H, _F64P, _F64P]),
    ("qp_get_scaling", c_int32, [_H, _F64P, _F64P]),
    ("qp_get_stats", c_int32, [_H, POINTER(QPInfoC)]),
    ("qp_get_trace", c_int32, [_H, POINTER(QPTraceEntryC), c_int64, POINTER(c_int64)]),
    ("qp_set_warm_start", c_int32, [_H, _F64P, _F64P]),
    ("qp_get_state", c_int32, [_H, POINTER(QPStateVectorsC), POINTER(QPStateScalarsC)]),
    ("qp_set_state", c_int32, [_H, POINTER(QPStateVectorsC), POINTER(QPStateScalarsC)]),
    ("qp_iterate", c_int32, [_H, POINTER(QPOptionsC), c_int64]),
    ("qp_evaluate", c_int32, [_H, _F64P, _F64P]),
    ("qp_norm_A", c_int32, [_H, c_int32, _F64P]),
    ("qp_get_penalty", c_int32, [_H, _F64P]),
    ("qp_set_bounds", c_int32, [_H, _F64P, _F64P]),
    ("qp_tune", c_int32, [_H, c_int32, POINTER(QPShapesC)]),
    ("qp_get_shapes", c_int32, [_H, POINTER(QPShapesC)]),
    ("qp_gather_rate", c_int32, [c_int64, c_int32, c_int32, c_uint64, _F64P]),
    ("qp_norm_A_static", c_int32, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("qp_csr_validate", c_int32, [c_int32, c_int32, _I32P, _I32P, _F64P]),
    ("qp_csr_transpose", c_int32, [c_int32, c_int32, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P]),
    ("qp_batch_create", c_int32, [POINTER(_H), c_int32, POINTER(QPInstanceC),
                                  POINTER(QPDeviceCtxC), c_uint32]),
    ("qp_batch_destroy", None, [_H]),
    ("qp_batch_solve", c_int32, [_H, POINTER(QPOptionsC), _F64P]),
    ("qp_batch_results", c_int32, [_H, POINTER(QPInstanceResultC)]),
    ("qp_batch_solution", c_int32, [_H, _F64P, _F64P]),
    ("qp_batch_set_warm_start", c_int32, [_H, _F64P, _F64P]),
    ("qp_batch_set_bounds", c_int32, [_H, _F64P, _F64P]),
    ("qp_batch_set_bounds_each", c_int32, [_H, c_void_p, c_void_p]),
    ("qp_batch_set_threads", c_int32, [_H, c_int32]),
    ("qp_batch_tune", c_int32, [_H, POINTER(QPOptionsC), c_int32, c_int32, _I32P]),
    ("qp_mlp_create", c_int32, [POINTER(_H), c_int32, _I32P, c_int32, POINTER(QPDeviceCtxC)]),
    ("qp_mlp_destroy", None, [_H]),
    ("qp_mlp_param_count", c_int64, [_H]),
    ("qp_mlp_set_params", c_int32, [_H, POINTER(c_float)]),
    ("qp_mlp_get_params", c_int32, [_H, POINTER(c_float)]),
    ("qp_mlp_forward", c_int32, [_H, c_int32, c_void_p, c_void_p]),
    ("qp_mlp_loss_grad", c_int32, [_H, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_double)]),
    ("qp_mlp_adam_step", c_int32, [_H, c_float]),
]

_lock = threading.Lock()
_lib = None


class QPError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}"
                         + (f" ({detail})" if detail else ""))


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libpdhcg.so (built in-tree by paper_2405_16160_b300.build).

    Raises FileNotFoundError when the library is missing: there is no other
    implementation to fall back to.
    """
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise FileNotFoundError(
                f"{p} is missing; build it with `python -m paper_2405_16160_b300.build`")
        lib = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != QP_OK:
        lib = load_library()
        raise QPError(status, where, (lib.qp_last_error() or b"").decode(errors="replace"))
