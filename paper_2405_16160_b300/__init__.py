"""B300-native restarted PDHCG solver for convex QP (arXiv 2405.16160).

min 1/2 x'Qx + c'x  s.t.  Ax <= b  (Q PSD; leading m_eq rows are equalities).

The solver lives in ``libpdhcg.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/pdhcg.h``).  This package only marshals arguments:
``solver.QPSolver`` wraps the C calls, ``workloads`` draws seeded synthetic
instances.  Importing the package does not load the library; the first call
that needs it does, and it raises if the library is missing.
"""
import importlib

__all__ = ["QPSolver", "QPOptions", "load_library"]


def __getattr__(name):
    if name in ("QPSolver", "QPOptions"):
        return getattr(importlib.import_module(".solver", __name__), name)
    if name == "load_library":
        return importlib.import_module("._lib", __name__).load_library
    raise AttributeError(name)
