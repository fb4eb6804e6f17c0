"""Python face of the C ABI: argument marshalling only.

Every step of the solve runs in libpdhcg.so's CUDA kernels; this module
converts numpy arrays to the C types, lends PyTorch's caching allocator and
current stream to the library, and turns status codes into exceptions.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p

import numpy as np

from . import _lib as L


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} entries, got {a.size}")
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _host_f64(n, pinned):
    """An n-entry float64 host array, page-locked (through PyTorch) if asked."""
    if pinned and n > 0:
        import torch
        return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    return np.empty(n)


def _ptr(a, ctype):
    return a.ctypes.data_as(POINTER(ctype)) if a is not None else None


def _addr(a):
    """The address of an array's data (0, NULL, for None), as _ptr gives it."""
    return 0 if a is None else a.__array_interface__["data"][0]


# struct qp_instance of include/pdhcg.h: four int32 sizes, then seven pointers
_INSTANCE_DTYPE = np.dtype([("n", np.int32), ("m", np.int32), ("m_eq", np.int32), ("k", np.int32),
                            ("F", np.uint64), ("qd", np.uint64), ("A_rowptr", np.uint64),
                            ("A_col", np.uint64), ("A_val", np.uint64), ("c", np.uint64),
                            ("b", np.uint64)])


class QPOptions:
    """Solver options (see qp_options in include/pdhcg.h); defaults from the library."""

    def __init__(self, **overrides):
        lib = L.load_library()
        self._c = L.QPOptionsC()
        lib.qp_options_default(byref(self._c))
        for k, v in overrides.items():
            setattr(self, k, v)

    def __getattr__(self, name):
        c = self.__dict__.get("_c")
        if c is not None and name in dict(L.QPOptionsC._fields_):
            return getattr(c, name)
        raise AttributeError(name)

    def __setattr__(self, name, value):
        if name == "_c":
            object.__setattr__(self, name, value)
        elif name in dict(L.QPOptionsC._fields_):
            setattr(self._c, name, value)
        else:
            raise AttributeError(f"unknown option {name}")

    def as_dict(self) -> dict:
        return {n: getattr(self._c, n) for n, _ in L.QPOptionsC._fields_ if n != "reserved"}


class QPSolver:
    """One QP resident on the current CUDA device.

    ``QPSolver(inst)`` copies the instance (``workloads.QPInstance`` or any
    object with the same CSR fields) through ``qp_create``.  With
    ``torch_memory=True`` (default) the device buffers come from PyTorch's
    caching allocator and the work is ordered after PyTorch's current stream.
    Variable bounds the instance carries (``lo``/``hi``, None when absent)
    are passed on to ``qp_set_bounds``.
    """

    def __init__(self, inst, torch_memory: bool = True, check_symmetry: bool = False,
                 scale: bool = False, penalty: bool = False):
        self.lib = L.load_library()
        self.n, self.m, self.m_eq = int(inst.n), int(inst.m), int(inst.m_eq)
        self._keep = []
        ctx = None
        if torch_memory:
            ctx = self._torch_ctx()
        Qr, Qc, Qv = _i32(inst.Q_rowptr), _i32(inst.Q_col), _f64(inst.Q_val)
        Ar, Ac, Av = _i32(inst.A_rowptr), _i32(inst.A_col), _f64(inst.A_val)
        c, b = _f64(inst.c, self.n), _f64(inst.b, self.m)
        h = c_void_p()
        st = self.lib.qp_create(byref(h), self.n, self.m, self.m_eq,
                                _ptr(Qr, c_int32), _ptr(Qc, c_int32), _ptr(Qv, c_double),
                                _ptr(Ar, c_int32), _ptr(Ac, c_int32), _ptr(Av, c_double),
                                _ptr(c, c_double), _ptr(b, c_double),
                                byref(ctx) if ctx is not None else None,
                                (L.CREATE_CHECK_SYMMETRY if check_symmetry else 0)
                                | (L.CREATE_SCALE if scale else 0)
                                | (L.CREATE_PENALTY if penalty else 0))
        L.check(st, "qp_create")
        self.h = h
        self._ctx = ctx
        lo, hi = getattr(inst, "lo", None), getattr(inst, "hi", None)
        if lo is not None or hi is not None:
            self.set_bounds(lo, hi)

    def _torch_ctx(self):
        import torch

        dev = torch.cuda.current_device()
        stream = torch.cuda.current_stream()

        def _alloc(nbytes, user, s):
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

        def _free(ptr, nbytes, user, s):
            torch.cuda.caching_allocator_delete(ptr)

        fa, ff = L.ALLOC_FN(_alloc), L.FREE_FN(_free)
        self._keep += [fa, ff, stream]
        return L.QPDeviceCtxC(fa, ff, None, c_void_p(stream.cuda_stream))

    # ------------------------------------------------------------------ solve
    def solve(self, options: QPOptions | None = None, **overrides) -> dict:
        o = options or QPOptions()
        for k, v in overrides.items():
            setattr(o, k, v)
        info = L.QPInfoC()
        st = self.lib.qp_solve(self.h, byref(o._c), byref(info))
        L.check(st, "qp_solve")
        return info.as_dict()

    def solution(self):
        """(x, y) in host arrays; page-locked ones when PyTorch has allocated
        this handle's memory, so that the copies run at DMA speed."""
        x = _host_f64(self.n, self._ctx is not None)
        y = _host_f64(self.m, self._ctx is not None)
        L.check(self.lib.qp_get_solution(self.h, _ptr(x, c_double), _ptr(y, c_double)),
                "qp_get_solution")
        return x, y

    def scaling(self):
        d1 = np.empty(self.m)
        d2 = np.empty(self.n)
        L.check(self.lib.qp_get_scaling(self.h, _ptr(d1, c_double), _ptr(d2, c_double)),
                "qp_get_scaling")
        return d1, d2

    def stats(self) -> dict:
        info = L.QPInfoC()
        L.check(self.lib.qp_get_stats(self.h, byref(info)), "qp_get_stats")
        return info.as_dict()

    def trace(self) -> list:
        cnt = c_int64()
        L.check(self.lib.qp_get_trace(self.h, None, 0, byref(cnt)), "qp_get_trace")
        buf = (L.QPTraceEntryC * max(cnt.value, 1))()
        L.check(self.lib.qp_get_trace(self.h, buf, cnt.value, byref(cnt)), "qp_get_trace")
        return [{n: getattr(buf[i], n) for n, _ in L.QPTraceEntryC._fields_}
                for i in range(cnt.value)]

    # ----------------------------------------------------------------- state
    _VEC = ("x", "y", "x_avg", "y_avg", "x_anchor", "y_anchor")

    def get_state(self) -> dict:
        arrs = {k: np.empty(self.n if k.startswith("x") else self.m) for k in self._VEC}
        v = L.QPStateVectorsC(*[_ptr(arrs[k], c_double) for k in self._VEC])
        s = L.QPStateScalarsC()
        L.check(self.lib.qp_get_state(self.h, byref(v), byref(s)), "qp_get_state")
        arrs.update({n: getattr(s, n) for n, _ in L.QPStateScalarsC._fields_})
        return arrs

    def set_state(self, state: dict) -> None:
        arrs = {k: (_f64(state[k], self.n if k.startswith("x") else self.m)
                    if state.get(k) is not None else None) for k in self._VEC}
        v = L.QPStateVectorsC(*[_ptr(arrs[k], c_double) for k in self._VEC])
        # a state without the adaptive-step scalars is a fixed-step state:
        # every iteration was one attempt and the epoch has no step weights
        defaults = {"attempts": state.get("k_total"), "weight_sum": 0.0}
        s = L.QPStateScalarsC(*[state[n] if n in state else defaults[n]
                                for n, _ in L.QPStateScalarsC._fields_])
        L.check(self.lib.qp_set_state(self.h, byref(v), byref(s)), "qp_set_state")

    def set_warm_start(self, x0=None, y0=None) -> None:
        x0 = _f64(x0, self.n) if x0 is not None else None
        y0 = _f64(y0, self.m) if y0 is not None else None
        L.check(self.lib.qp_set_warm_start(self.h, _ptr(x0, c_double), _ptr(y0, c_double)),
                "qp_set_warm_start")

    def iterate(self, iters: int, options: QPOptions | None = None, **overrides) -> None:
        o = options or QPOptions()
        for k, v in overrides.items():
            setattr(o, k, v)
        L.check(self.lib.qp_iterate(self.h, byref(o._c), int(iters)), "qp_iterate")

    def evaluate(self):
        kc = np.empty(6)
        ka = np.empty(6)
        L.check(self.lib.qp_evaluate(self.h, _ptr(kc, c_double), _ptr(ka, c_double)), "qp_evaluate")
        keys = ("r_primal", "r_dual", "r_gap", "relkkt", "primal_obj", "dual_obj")
        return dict(zip(keys, kc)), dict(zip(keys, ka))

    def norm_A(self, iters: int = 30) -> float:
        out = c_double()
        L.check(self.lib.qp_norm_A(self.h, int(iters), byref(out)), "qp_norm_A")
        return out.value

    def set_bounds(self, lo=None, hi=None) -> None:
        """Variable bounds lo <= x <= hi (None: no bound on that side; +-inf allowed)."""
        lo = _f64(lo, self.n) if lo is not None else None
        hi = _f64(hi, self.n) if hi is not None else None
        L.check(self.lib.qp_set_bounds(self.h, _ptr(lo, c_double), _ptr(hi, c_double)),
                "qp_set_bounds")

    def penalty_rho(self) -> float:
        out = c_double()
        L.check(self.lib.qp_get_penalty(self.h, byref(out)), "qp_get_penalty")
        return out.value

    def tune(self, reps: int = 20) -> dict:
        """qp_tune: time the row kernels' launch shapes on this problem's
        matrices and keep the fastest; returns the shapes in use."""
        out = L.QPShapesC()
        L.check(self.lib.qp_tune(self.h, int(reps), byref(out)), "qp_tune")
        return out.as_dict()

    def shapes(self) -> dict:
        """qp_get_shapes: the launch shapes in use."""
        out = L.QPShapesC()
        L.check(self.lib.qp_get_shapes(self.h, byref(out)), "qp_get_shapes")
        return out.as_dict()

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.qp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ batches
class QPBatch:
    """Many small QPs with Q = F F' + diag(qd), solved in one launch.

    ``instances`` is a list of ``workloads.LowRankQP`` (or objects with the
    same fields).  Solutions and warm starts are lists of per-instance arrays.
    Variable bounds the instances carry (``lo``/``hi``) are packed and passed
    on to ``qp_batch_set_bounds``.
    """

    def __init__(self, instances, torch_memory: bool = True):
        self.lib = L.load_library()
        self.count = len(instances)
        self.ns = [int(q.n) for q in instances]
        self.ms = [int(q.m) for q in instances]
        self._keep = []  # the allocator callbacks (alive as long as the handle)
        arrays = []      # instance arrays (read during qp_batch_create only)
        # the qp_instance table as a structured array with the C layout (its
        # pointers are the arrays' addresses, 0 for NULL): no ctypes object
        # per array, which dominates the marshalling of thousands of instances
        table = np.zeros(self.count, dtype=_INSTANCE_DTYPE)
        ints = np.empty((self.count, 4), dtype=np.int32)
        ptrs = np.zeros((self.count, 7), dtype=np.uint64)
        for i, q in enumerate(instances):
            F = _f64(q.F).reshape(-1) if q.k > 0 else None
            qd, c = _f64(q.qd, q.n), _f64(q.c, q.n)
            b = _f64(q.b, q.m)
            Ar, Ac, Av = _i32(q.A_rowptr), _i32(q.A_col), _f64(q.A_val)
            arrays += [F, qd, c, b, Ar, Ac, Av]
            ints[i] = (q.n, q.m, q.m_eq, q.k)
            ptrs[i] = [_addr(a) for a in (F, qd, Ar, Ac, Av, c, b)]
        for j, name in enumerate(("n", "m", "m_eq", "k")):
            table[name] = ints[:, j]
        for j, name in enumerate(("F", "qd", "A_rowptr", "A_col", "A_val", "c", "b")):
            table[name] = ptrs[:, j]
        ctx = QPSolver._torch_ctx(self) if torch_memory else None
        h = c_void_p()
        st = self.lib.qp_batch_create(byref(h), self.count,
                                      table.ctypes.data_as(POINTER(L.QPInstanceC)),
                                      byref(ctx) if ctx is not None else None, 0)
        del arrays, table
        L.check(st, "qp_batch_create")
        self.h = h
        self._ctx = ctx
        if any(getattr(q, "lo", None) is not None or getattr(q, "hi", None) is not None
               for q in instances):
            self.set_bounds([getattr(q, "lo", None) for q in instances],
                            [getattr(q, "hi", None) for q in instances])

    def solve(self, options: QPOptions | None = None, **overrides) -> float:
        """Solve every instance; returns the launch's device time in ms."""
        o = options or QPOptions()
        for k, v in overrides.items():
            setattr(o, k, v)
        ms = c_double()
        L.check(self.lib.qp_batch_solve(self.h, byref(o._c), byref(ms)), "qp_batch_solve")
        return ms.value

    def results(self) -> list:
        out = (L.QPInstanceResultC * self.count)()
        L.check(self.lib.qp_batch_results(self.h, out), "qp_batch_results")
        return [out[i].as_dict() for i in range(self.count)]

    def solution(self):
        x = np.empty(sum(self.ns))
        y = np.empty(max(sum(self.ms), 1))
        L.check(self.lib.qp_batch_solution(self.h, _ptr(x, c_double), _ptr(y, c_double)),
                "qp_batch_solution")
        return np.split(x, np.cumsum(self.ns)[:-1]), np.split(y[:sum(self.ms)],
                                                              np.cumsum(self.ms)[:-1])

    def set_warm_start(self, xs=None, ys=None) -> None:
        """Per-instance starting points: lists of arrays, or the packed arrays
        (instance after instance) as they are."""
        def pack(vs, total):
            if vs is None:
                return None
            if isinstance(vs, np.ndarray) and vs.ndim == 1:
                return _f64(vs, total)
            return _f64(np.concatenate(vs), total)
        x0, y0 = pack(xs, sum(self.ns)), pack(ys, sum(self.ms))
        L.check(self.lib.qp_batch_set_warm_start(self.h, _ptr(x0, c_double), _ptr(y0, c_double)),
                "qp_batch_set_warm_start")

    def set_bounds(self, los=None, his=None) -> None:
        """Per-instance bounds: lists of arrays (an entry None: no bound on
        that side), passed as one pointer per instance (qp_batch_set_bounds_each:
        no packed copy on either side of the call)."""
        def table(vs):
            if vs is None:
                return None, None
            if len(vs) != self.count:
                raise ValueError(f"expected {self.count} bound arrays, got {len(vs)}")
            arrs = [None if v is None else _f64(v, n) for v, n in zip(vs, self.ns)]
            return arrs, np.array([_addr(a) for a in arrs], dtype=np.uint64)
        lo_keep, lo = table(los)
        hi_keep, hi = table(his)
        L.check(self.lib.qp_batch_set_bounds_each(
            self.h, None if lo is None else lo.ctypes.data, None if hi is None else hi.ctypes.data),
            "qp_batch_set_bounds_each")
        del lo_keep, hi_keep

    def set_threads(self, threads: int) -> None:
        L.check(self.lib.qp_batch_set_threads(self.h, int(threads)), "qp_batch_set_threads")

    def tune(self, options: QPOptions | None = None, sample_count: int = 1 << 30,
             sample_iters: int = 128, **overrides) -> int:
        o = options or QPOptions()
        for k, v in overrides.items():
            setattr(o, k, v)
        t = c_int32()
        L.check(self.lib.qp_batch_tune(self.h, byref(o._c), int(sample_count), int(sample_iters),
                                       byref(t)), "qp_batch_tune")
        return t.value

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.qp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ host-only helpers
def csr_validate(rows, cols, rowptr, col, val) -> int:
    lib = L.load_library()
    rp, cc, vv = _i32(rowptr), _i32(col), _f64(val)
    return lib.qp_csr_validate(int(rows), int(cols), _ptr(rp, c_int32), _ptr(cc, c_int32),
                               _ptr(vv, c_double))


def csr_transpose(rows, cols, rowptr, col, val):
    lib = L.load_library()
    rp, cc, vv = _i32(rowptr), _i32(col), _f64(val)
    nnz = int(rp[-1])
    tr = np.empty(cols + 1, np.int32)
    tc = np.empty(max(nnz, 1), np.int32)
    tv = np.empty(max(nnz, 1), np.float64)
    L.check(lib.qp_csr_transpose(int(rows), int(cols), _ptr(rp, c_int32), _ptr(cc, c_int32),
                                 _ptr(vv, c_double), _ptr(tr, c_int32), _ptr(tc, c_int32),
                                 _ptr(tv, c_double)), "qp_csr_transpose")
    return tr, tc[:nnz], tv[:nnz]
