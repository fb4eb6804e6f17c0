"""Write oracle-only expected values for the large parity cases.

    python oracle/make_golden.py [--n 1000000 --m 500000 --seed 0] [--scale] [--adaptive-step]

Runs the CPU oracle (and nothing else: the CUDA library is not loaded) on
the seeded large sparse instance and stores its trajectory summary under
tests/golden/.  The instance comes from the shared seeded generator, which
holds none of the solver's arithmetic.  With --scale the oracle applies its
own Section 4 diagonal scaling (10 Ruiz steps, then Pock-Chambolle); with
--adaptive-step it uses the Section 4 adaptive step size.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import pdhcg_oracle as O  # noqa: E402
from paper_2405_16160_b300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=500_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--scale", action="store_true")
    ap.add_argument("--adaptive-step", action="store_true")
    args = ap.parse_args()
    inst = W.sparse_dd(args.seed, n=args.n, m=args.m)
    P = O.problem_from_instance(inst)
    t0 = time.perf_counter()
    step = O.STEP_ADAPTIVE if args.adaptive_step else O.STEP_FIXED
    res = O.solve(P, O.OracleOptions(tol=args.tol, scale=args.scale, step_mode=step))
    secs = time.perf_counter() - t0
    out = {
        "source": "oracle/pdhcg_oracle.py (CPU FP64), instance workloads.sparse_dd",
        "instance": {"n": args.n, "m": args.m, "seed": args.seed, "tol": args.tol,
                     "scale": args.scale, "nnz_Q": inst.nnz_Q, "nnz_A": inst.nnz_A,
                     "step_mode": "adaptive" if args.adaptive_step else "fixed"},
        "termination": res.termination, "iterations": res.iterations, "cg_steps": res.cg_steps,
        "attempts": res.state.attempts,
        "restarts": res.restarts, "returned_avg": res.returned_avg,
        "relkkt": res.kkt.relkkt, "primal_obj": res.kkt.primal_obj, "dual_obj": res.kkt.dual_obj,
        "eta": res.state.eta, "omega": res.state.omega,
        "trace": res.trace, "oracle_seconds": secs,
    }
    name = (f"sparse_dd_n{args.n}_m{args.m}_seed{args.seed}"
            f"{'_scaled' if args.scale else ''}{'_adaptive' if args.adaptive_step else ''}"
            "_trace.json")
    path = os.path.join(ROOT, "tests", "golden", name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, res.iterations, res.cg_steps, res.restarts, res.kkt.relkkt, f"{secs:.1f}s")


if __name__ == "__main__":
    main()
