"""Solve a generated workload from the command line.

    python -m paper_2405_16160_b300.solve --workload zipf_dd --max-iter 64 --repeat 2

Builds the library if needed, creates the instance on the current CUDA
device (with the Section 4 scaling unless --no-scale) and prints one JSON
line per solve: the qp_info fields, the solve's device time and, for the
first, the create time.  Every step runs in libpdhcg.so.
"""
from __future__ import annotations

import argparse
import json
import time

from . import _lib as L
from . import build as B
from . import workloads as W

GENERATORS = {
    "sparse_dd": W.sparse_dd,
    "zipf_dd": W.zipf_dd,
    "dense_small": W.dense_small,
}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=sorted(GENERATORS), default="sparse_dd")
    ap.add_argument("--n", type=int, default=None, help="override the workload's n")
    ap.add_argument("--m", type=int, default=None, help="override the workload's m")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=100_000,
                    help="iteration limit (attempts with the adaptive step)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--step", choices=["adaptive", "fixed"], default="adaptive")
    ap.add_argument("--no-scale", action="store_true")
    ap.add_argument("--mixed-stall-evals", type=int, default=None,
                    help="mixed: hand over to FP64 after this many evaluations without a "
                         "10%% gain (0: off; default: the library's)")
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    from .solver import QPSolver

    B.build()
    kw = {k: v for k, v in (("n", args.n), ("m", args.m)) if v is not None}
    inst = GENERATORS[args.workload](args.seed, **kw)
    t0 = time.perf_counter()
    solver = QPSolver(inst, scale=not args.no_scale)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    opts = dict(tol=args.tol, max_iter=args.max_iter,
                precision=L.PREC_MIXED if args.precision == "mixed" else L.PREC_FP64,
                step_mode=L.STEP_ADAPTIVE if args.step == "adaptive" else L.STEP_FIXED)
    if args.mixed_stall_evals is not None:
        opts["mixed_stall_evals"] = args.mixed_stall_evals
    with solver:
        for r in range(args.repeat):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = solver.solve(**opts)
            e1.record(stream)
            e1.synchronize()
            out = {"workload": args.workload, "n": inst.n, "m": inst.m, "solve": r,
                   "device_s": e0.elapsed_time(e1) / 1e3, **info}
            if r == 0:
                out["create_s"] = create_s
            print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
