"""Build libpdhcg.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2405_16160_b300.build [--force]

The library is plain C ABI (include/pdhcg.h); no PyTorch headers are used.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libpdhcg.so")
SOURCES = ["pdhcg.cu", "batch.cu", "mlp.cu", "norm_static.cu", "diag.cu", "host_csr.cpp"]
# the batched solver's kernel, one object per value type and block size
BATCH_INST = [(v, nt) for v in ("float", "double") for nt in (64, 128, 256, 512)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    """(source, extra flags, object name) of every compile unit."""
    units = [(src, [], src + ".o") for src in SOURCES]
    units += [("batch_inst.cu", [f"-DBATCH_V={v}", f"-DBATCH_NT={nt}"], f"batch_inst_{v}_{nt}.o")
              for v, nt in BATCH_INST]
    return units


def _deps(obj: str):
    """The files an object was built from, from the dependency file nvcc wrote
    beside it (None when there is none)."""
    try:
        text = open(obj + ".d").read()
    except OSError:
        return None
    text = text.replace("\\\n", " ")
    _, _, rest = text.partition(":")
    return [f for f in rest.split() if f]


def _stale(obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = _deps(obj)
    if deps is None:
        return True
    t = os.path.getmtime(obj)
    deps.append(os.path.abspath(__file__))
    return any(not os.path.exists(f) or os.path.getmtime(f) > t for f in deps)


def up_to_date() -> bool:
    """The library is newer than everything it is built from: its objects and
    their dependencies, or, where the objects are absent (a copy of the tree
    that carries the library alone), every source and header of the package."""
    if not os.path.exists(LIB):
        return False
    objdir = os.path.join(PKG, "_build")
    t = os.path.getmtime(LIB)
    objs = [os.path.join(objdir, name) for _, _, name in _units()]
    if all(os.path.exists(o) for o in objs):
        return all(not _stale(o) and os.path.getmtime(o) <= t for o in objs)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(ROOT, "include", "pdhcg.h"), os.path.abspath(__file__)]
    return all(os.path.getmtime(f) <= t for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every stale unit to an object in parallel (an object is stale
    when a file it was built from is newer), then link the library."""
    if not force and up_to_date():
        return LIB
    from concurrent.futures import ThreadPoolExecutor

    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
             "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")

    def compile_one(unit) -> str:
        src, extra, name = unit
        obj = os.path.join(objdir, name)
        if not force and not _stale(obj):
            return obj
        cmd = [nvcc(), *flags, *extra, "-MD", "-MF", obj + ".d", "-c", os.path.join(CSRC, src),
               "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        return obj

    units = _units()
    with ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, units))
    subprocess.run([nvcc(), *ARCH, "-shared", *objs, "-o", LIB + ".tmp"], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(path)
