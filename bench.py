"""Benchmark: time to relKKT <= 1e-4 of restarted PDHCG on the large sparse QP.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete qp_solve (set-up power iteration, every PDHCG
iteration, relKKT evaluations, restarts, the final FP64 check) of the seeded
n=1e6, m=5e5 sparse QP (Q diagonally dominant with ~9 nnz/row, A with 10
uniform nnz/row) in mixed precision, with the problem already resident on
the device, diagonally scaled as Section 4 prescribes (10 Ruiz steps and
one Pock-Chambolle step, done once by qp_create) and with the Section 4
adaptive step size (``--step fixed``: eta = 1/(2||A||_2)).  The same solve in
plain FP64 is timed beside it, and both again with the other step rule.  The solve measured end to end through the C ABI
from host arrays (qp_create with the scaling and the host-to-device copies,
qp_solve, qp_get_solution, qp_destroy) is reported as ``e2e``.

``--impl reference`` times the CPU FP64 oracle (the reference arm of this
build): every timed step is one complete oracle solve of the same instance
to 1e-4 on the host's cores.
Under torchrun (N > 1) every rank solves its own instance (replicas; the
path has no cross-GPU exchange) and rank 0 prints the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "large sparse QP: n=1e6, m=5e5, Q = diag U[0.5,2] + mirrored N(0,0.1) "
                        "(~9 nnz/row, diagonally dominant), A 10 uniform N(0,1) nnz/row, "
                        "c ~ N(0,1), b = A x0 + U[0,1]",
            "n": 1_000_000, "m": 500_000, "seed": 0, "tol": 1e-4, "precision": "mixed",
            "scaling": "Section 4: 10 Ruiz steps + Pock-Chambolle on [[Q, A'], [A, 0]]",
            "step": "Section 4 adaptive step size",
            "l2": "inputs larger than L2 (~470 MB resident working set vs 126 MB L2)"}
METRIC = "time to 1e-4 rel. KKT (restarted PDHCG; FP32 data/iterates, FP64 reductions) vs plain FP64 GPU PDHCG"

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def cg_kernel_bytes(nnz_q: int, n: int, cg_steps: int, w: int, k_v: int = 11) -> float:
    """Algorithmic DRAM bytes of the CG kernel: per CG step, one product with
    Q, (w + 4) B per stored entry (value + int32 column) and 4 (n + 1) B of
    row pointers, plus k_v vector streams of n values of w bytes.  k_v = 11
    counts textbook CG's vector statements with each operand read once and
    each result written once (q = Q p: read p, write q; x += a p: 3;
    r -= a q: 3; p = r + b p: 3); k_v = 6 is the fully fused floor (p, q, x
    and r each once, x and r written back).  Streams the implementation adds
    (the tracked Q x, the adaptive step's sums) are not counted."""
    return cg_steps * ((w + 4.0) * nnz_q + 4.0 * (n + 1) + k_v * float(w) * n)


def mixed_solve_launches(chunks: int, power_iters: int, eval_freq: int) -> int:
    """Kernel launches of one mixed-precision qp_solve on an instance without
    long rows (each SpMV is then one launch).

    set-up: k_init_vectors; cache refresh (k_materialize, A x_a, k_shift_rhs,
    A dx, A'y, Q x, k_prepare); power iteration (k_pow_start, 2 per step,
    k_setup_finish); the first evaluation (k_materialize, 4 SpMVs, k_kkt_n,
    k_kkt_m, k_control).  Per chunk: 3 per iteration or attempt (k_cg, k_dual,
    k_atv; the adaptive step commits inside k_atv), an evaluation (8), the
    restart kernels (3) and k_prepare.  At the end the FP64 check: 2
    conversions, the FP64 cache refresh (3 SpMVs, k_prepare) and an FP64
    evaluation (4 SpMVs, k_kkt_n, k_kkt_m, k_control)."""
    setup = 1 + 7 + (1 + 2 * power_iters + 1) + 8
    chunk = 3 * eval_freq + 8 + 3 + 1
    final = 2 + 4 + 7
    return setup + chunks * chunk + final


def gather_ceiling(count: int, n: int) -> float | None:
    """The device's random-gather rate (qp_gather_rate) over `count` reads of an
    n-float vector: the ceiling of an SpMV over uniformly random columns."""
    from ctypes import byref, c_double
    from paper_2405_16160_b300 import _lib as L
    out = c_double()
    st = L.load_library().qp_gather_rate(int(count), int(n), 10, 1, byref(out))
    return out.value if st == 0 else None


def _profiled_traffic():
    """DRAM bytes per k_cg launch from the committed ncu capture, or None when
    the kernel source has changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_cg_traffic.json")
    src = os.path.join(ROOT, "paper_2405_16160_b300", "csrc", "kernels.cuh")
    try:
        with open(prof) as f:
            rec = json.load(f)
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return rec.get("dram_bytes_per_launch_full_size") if rec.get("kernels_cuh_sha256_16") == sha \
        else None


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
               "NUMEXPR_NUM_THREADS")


def host_cpu():
    """(logical cores this process may use, CPU model name) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


def oracle_full_solve(step: str = "adaptive", max_iter: int = 100_000, inst=None) -> dict:
    """The oracle as it stands, one complete solve of the bench instance to
    relKKT <= 1e-4: its Section 4 scaling, set-up (power iteration, omega_0),
    every attempt, the relKKT evaluations and restarts.  Instance generation
    is outside the timed region.  max_iter caps the attempts (untimed
    warm-ups only)."""
    from oracle import pdhcg_oracle as O
    from paper_2405_16160_b300 import workloads as W
    if inst is None:
        inst = W.sparse_dd(WORKLOAD["seed"], n=WORKLOAD["n"], m=WORKLOAD["m"])
    P = O.problem_from_instance(inst)
    o = O.OracleOptions(tol=WORKLOAD["tol"], max_iter=max_iter, eval_freq=64, scale=True,
                        step_mode=O.STEP_ADAPTIVE if step == "adaptive" else O.STEP_FIXED)
    c0, t0 = time.process_time(), time.perf_counter()
    r = O.solve(P, o)
    wall = time.perf_counter() - t0
    return {"s": wall, "cpu_s": time.process_time() - c0, "attempts": r.state.attempts,
            "iterations": r.iterations, "relkkt": r.kkt.relkkt, "termination": r.termination}


def oracle_solve_subprocess(threads: int, step: str) -> dict:
    """oracle_full_solve in a fresh interpreter whose BLAS/OpenMP pools are
    limited to `threads` (the variables must be set before numpy loads)."""
    env = dict(os.environ)
    for v in THREAD_VARS:
        env[v] = str(threads)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-solve",
                          "--step", step], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_record(step: str) -> dict:
    """The oracle's time to 1e-4 on the host: one full solve with every core
    available to its BLAS/OpenMP pools (value) and one with them pinned to
    a single thread."""
    cores, model = host_cpu()
    full = oracle_solve_subprocess(cores, step)
    one = oracle_solve_subprocess(1, step)
    return {"value": full["s"], "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"one full oracle solve of the same instance to relKKT <= 1e-4 (Section 4 "
                      f"scaling, set-up, {full['attempts']} attempts, final relKKT "
                      f"{full['relkkt']:.2e}), numpy/scipy with BLAS/OpenMP threads = {cores}",
            "cpu_model": model, "process_cpu_s": full["cpu_s"],
            "single_thread_s": one["s"], "single_thread_attempts": one["attempts"],
            "single_thread_note": "the same full solve with every BLAS/OpenMP pool limited to "
                                  "one thread"}


def run_reference(args):
    """The CPU FP64 oracle, as it stands, on the bench instance: every timed
    step is one complete solve to relKKT <= 1e-4 on the host's cores; the
    untimed warm-up steps run the same solve capped at 8 attempts (imports,
    scipy set-up, first touch of the instance)."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2405_16160_b300 import workloads as W
    inst = W.sparse_dd(WORKLOAD["seed"], n=WORKLOAD["n"], m=WORKLOAD["m"])
    cores, model = host_cpu()
    for _ in range(args.warmup):
        oracle_full_solve(args.step, max_iter=8, inst=inst)
    runs = [oracle_full_solve(args.step, inst=inst) for _ in range(args.steps)]
    v = statistics.mean(r["s"] for r in runs)
    sample = (f"one full oracle solve of the instance to relKKT <= 1e-4 per step ("
              f"{runs[-1]['attempts']} attempts, final relKKT {runs[-1]['relkkt']:.2e}); "
              f"warm-up steps capped at 8 attempts")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, step=args.step, precision="fp64 (oracle)"),
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": model,
                         "process_cpu_s": statistics.mean(r["cpu_s"] for r in runs)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def _timed_solves(solver, steps, stream, **opts):
    import torch
    infos, times = [], []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = solver.solve(**opts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        infos.append(info)
    return infos, times


LARGEST = {"workload": "largest single QP: n=1e7, m=5e6, Q ~5 nnz/row diagonally dominant, A 8 "
                       "nnz/row with Zipf(1.1) column popularity, Section 4 scaling",
           "n": 10_000_000, "m": 5_000_000, "seed": 0, "attempts": 256}


def largest_qp_record(stream, step: int, steps: int = 2) -> dict:
    """The largest single QP (n = 1e7, m = 5e6) on the same GPU: the first
    LARGEST['attempts'] attempts of its solve, timed in mixed precision and in
    plain FP64 (ms per attempt and their ratio), and the CG kernel's
    roofline over a kernel-timed run of the same attempts.  A full solve of
    this instance takes about 40 s (bench.py --workload zipf_dd)."""
    import torch

    from paper_2405_16160_b300 import _lib as L
    from paper_2405_16160_b300 import workloads as W
    from paper_2405_16160_b300.solver import QPSolver

    inst = W.zipf_dd(LARGEST["seed"], n=LARGEST["n"], m=LARGEST["m"])
    cap = LARGEST["attempts"]
    out = {"workload": LARGEST["workload"], "attempts_timed": cap}
    with QPSolver(inst, scale=True) as s:
        out["tuned_shapes"] = s.tune(reps=5)
        runs = {}
        for name, prec in (("mixed", L.PREC_MIXED), ("fp64", L.PREC_FP64)):
            opts = dict(tol=1e-4, precision=prec, step_mode=step, max_iter=cap)
            s.solve(**opts)  # warm-up: graph capture
            infos, times = _timed_solves(s, steps, stream, **opts)
            runs[name] = statistics.mean(times)
            out[f"{name}_ms_per_attempt"] = runs[name] * 1e3 / infos[-1]["attempts"]
            out[f"{name}_relkkt_after"] = infos[-1]["relkkt"]
        out["fp64_over_mixed"] = runs["fp64"] / runs["mixed"]
        kinfos, _ = _timed_solves(s, 1, stream, tol=1e-4, precision=L.PREC_MIXED, step_mode=step,
                                  max_iter=cap, kernel_timing=1)
    ki = kinfos[-1]
    ks = ki["cg_kernel_ms"] / 1e3
    peak, peak_kind = _peaks()
    if ks > 0:
        achieved = cg_kernel_bytes(inst.nnz_Q, inst.n, ki["cg_kernel_spmvs"], 4) / ks / 1e9
        out["roofline"] = {"kernel": "k_cg<float>", "bound": "hbm", "achieved": achieved,
                           "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                           "peak_kind": peak_kind,
                           "avg_launch_us": ks / max(ki["cg_kernel_launches"], 1) * 1e6,
                           "cg_steps_per_launch": ki["cg_kernel_spmvs"]
                           / max(ki["cg_kernel_launches"], 1)}
    del inst
    torch.cuda.synchronize()
    return out


def run_ours(args):
    import torch

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2405_16160_b300 import _lib as L
    from paper_2405_16160_b300 import build as B
    from paper_2405_16160_b300 import workloads as W
    from paper_2405_16160_b300.solver import QPSolver

    B.build()
    inst = W.sparse_dd(WORKLOAD["seed"] + rank, n=WORKLOAD["n"], m=WORKLOAD["m"])
    tol = WORKLOAD["tol"]
    stream = torch.cuda.current_stream()
    step = L.STEP_ADAPTIVE if args.step == "adaptive" else L.STEP_FIXED
    other = L.STEP_FIXED if step == L.STEP_ADAPTIVE else L.STEP_ADAPTIVE
    mixed = dict(tol=tol, precision=L.PREC_MIXED, step_mode=step)
    fp64 = dict(tol=tol, precision=L.PREC_FP64, step_mode=step)

    # ---- device-resident solves (value): mixed precision, CUDA-graph replay,
    # with the row kernels' launch shapes picked by qp_tune (the solve with
    # the mean-row-length rule's shapes is timed first, for the comparison)
    solver = QPSolver(inst, scale=True)
    for _ in range(args.warmup):
        solver.solve(**mixed)
    _, rule_times = _timed_solves(solver, max(2, args.steps // 2), stream, **mixed)
    t_tune = time.perf_counter()
    # --shapes rule keeps the rule's shapes (profiling: under ncu the tuner's
    # timings, and so its choices, are not those of a plain run)
    shapes = solver.tune(reps=20) if args.shapes == "tuned" else solver.shapes()
    tune_s = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        solver.solve(**mixed)
    solver.solve(**fp64)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        _barrier(ws)
        torch.cuda.synchronize()
        infos, times = _timed_solves(solver, args.steps, stream, **mixed)
        torch.cuda.synchronize()
        _barrier(ws)
    trace_len = len(solver.trace())
    # the same solve in plain FP64 (the ratio the metric asks for)
    infos64, times64 = _timed_solves(solver, max(1, args.steps // 2), stream, **fp64)
    # both again with the other step rule
    oth = {}
    for name, opts in (("mixed", mixed), ("fp64", fp64)):
        o2 = dict(opts, step_mode=other)
        solver.solve(**o2)
        inf2, t2 = _timed_solves(solver, max(1, args.steps // 4), stream, **o2)
        oth[name] = (statistics.mean(t2), inf2[-1])
    # the dominant kernel, timed launch by launch with CUDA events on its stream
    kinfos, _ = _timed_solves(solver, max(1, args.steps // 2), stream, kernel_timing=1, **mixed)
    solver.close()
    per_solve = _max_over_ranks(statistics.mean(times), ws)
    per_solve64 = _max_over_ranks(statistics.mean(times64), ws)

    # ---- end to end through the C ABI from host arrays, staged once in pinned
    # (page-locked) host memory so that the copies inside the timed region run
    # at DMA speed
    import dataclasses

    import numpy as np

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(np.empty(0, a.dtype)).dtype,
                        pin_memory=True)
        out = t.numpy()
        out[...] = a
        return out

    inst_pinned = dataclasses.replace(inst, **{
        k: pinned(getattr(inst, k)) for k in ("Q_rowptr", "Q_col", "Q_val", "A_rowptr",
                                              "A_col", "A_val", "c", "b")})
    e2e_times = []
    # what qp_create copies: Q, A, c and b as given (A' is built on the device)
    h2d = (inst.Q_rowptr.nbytes + inst.Q_col.nbytes + inst.Q_val.nbytes
           + inst.A_rowptr.nbytes + inst.A_col.nbytes + inst.A_val.nbytes
           + inst.c.nbytes + inst.b.nbytes)
    d2h = 8 * (inst.n + inst.m)
    e2e_steps = max(1, min(args.steps, 3))
    for s in range(1 + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with QPSolver(inst_pinned, scale=True) as s2:
            s2.solve(**mixed)
            x, y = s2.solution()
        torch.cuda.synchronize()
        if s > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e = _max_over_ranks(statistics.mean(e2e_times), ws)
    largest = None if args.no_largest else largest_qp_record(stream, step)

    if rank != 0:
        return 0
    info = infos[-1]
    peak, peak_kind = _peaks()
    bytes_total = sum(cg_kernel_bytes(inst.nnz_Q, inst.n, i["cg_kernel_spmvs"], 4)
                      for i in kinfos)
    bytes_floor = sum(cg_kernel_bytes(inst.nnz_Q, inst.n, i["cg_kernel_spmvs"], 4, k_v=6)
                      for i in kinfos)
    launches = sum(i["cg_kernel_launches"] for i in kinfos)
    kernel_s = sum(i["cg_kernel_ms"] for i in kinfos) / 1e3
    achieved = bytes_total / kernel_s / 1e9 if kernel_s > 0 else None
    # the capture is of a one-CG-step launch; a launch averages spmvs/launches steps
    traffic = _profiled_traffic()
    steps_per_launch = sum(i["cg_kernel_spmvs"] for i in kinfos) / max(launches, 1)
    if traffic is not None:
        traffic *= steps_per_launch
    gpu_launches = args.steps * mixed_solve_launches(trace_len, 30, 64)
    ceiling = gather_ceiling(inst.nnz_Q, inst.n)
    gathers = (sum(i["cg_kernel_spmvs"] for i in kinfos) * inst.nnz_Q / kernel_s
               if kernel_s > 0 else None)

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record(args.step)
    out = {
        "metric": METRIC, "value": per_solve, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 reductions and scalars)",
        "data": "synthetic",
        "config": dict(WORKLOAD, step=args.step, iterations=info["iterations"],
                       attempts=info["attempts"], cg_steps=info["cg_steps"],
                       restarts=info["restarts"], relkkt_fp64_check=info["check_relkkt"],
                       refine_iterations=info["refine_iterations"],
                       fp64_time_s=per_solve64, fp64_iterations=infos64[-1]["iterations"],
                       fp64_attempts=infos64[-1]["attempts"],
                       speedup_vs_fp64=per_solve64 / per_solve,
                       other_step=("fixed" if args.step == "adaptive" else "adaptive"),
                       other_step_mixed_s=oth["mixed"][0],
                       other_step_mixed_attempts=oth["mixed"][1]["attempts"],
                       other_step_fp64_s=oth["fp64"][0],
                       other_step_fp64_attempts=oth["fp64"][1]["attempts"],
                       rule_shapes_s=statistics.mean(rule_times),
                       tuned_shapes=shapes, tune_s=tune_s,
                       shapes_note="value: row kernels at qp_tune's launch shapes (lanes per "
                                   "row, row layout, waves); rule_shapes_s: the same solve at "
                                   "the mean-row-length rule's shapes, timed before tuning",
                       parallelism=f"replicas x{ws}"),
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "inputs": "pinned host arrays (staged once, before the timed region)",
                "timed": "qp_create + qp_solve + qp_get_solution + qp_destroy"},
        "roofline": {"kernel": "k_cg<float> (persistent CG: Q SpMV + vector phases)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_total / max(launches, 1),
                     "bytes_note": "per CG step (w+4) nnz(Q) + 4(n+1) + 11 n w (w = 4): the "
                                   "matrix stream and textbook CG's vector statements",
                     "frac_fused_floor": (bytes_floor / kernel_s / 1e9 / peak)
                     if kernel_s > 0 else None,
                     "cg_steps_per_launch": steps_per_launch,
                     "traffic_note": "ncu DRAM read+write of a one-CG-step k_cg launch "
                                     "(profiles/k_cg_traffic.json) x CG steps per launch",
                     "gathers_per_s": gathers,
                     "gather_ceiling_per_s": ceiling,
                     "gather_frac": (gathers / ceiling) if gathers and ceiling else None,
                     "gather_note": "p is gathered at one random column per stored entry of "
                                    "Q; the ceiling is qp_gather_rate over nnz(Q) reads of an "
                                    "n-float vector, measured in this run",
                     "avg_launch_us": kernel_s / max(launches, 1) * 1e6,
                     "timing": "CUDA events around every k_cg launch (direct launches) in "
                               "solves run right after the timed region"},
        "cpu_baseline": cpu,
        "gpu_launches": gpu_launches,
        "clocks": clocks.summary(),
        "largest_qp": largest,
    }
    print(json.dumps(out), flush=True)
    return 0


BATCH_WORKLOAD = {
    "workload": "4096 portfolio QPs: n ~ U{20..400}, k = n/10 factors, Q = F F' + diag U[0.01,0.1], "
                "F ~ N(0, 1/k); budget equality, long-only and U{5..20} sector-cap rows; "
                "c = -mu, mu ~ N(0.05, 0.02)",
    "count": 4096, "seed": 0, "tol": 1e-4, "precision": "mixed (FP32 data, products and attempt "
    "vectors; FP64 iterates, averages, block totals and scalars; relKKT on the FP64 data)",
}
BATCH_METRIC = ("time to 1e-4 rel. KKT for 4096 portfolio QPs (batched PDHCG, one launch) "
                "vs plain FP64 GPU PDHCG one instance at a time")
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x FMA x max clock


def batch_flops(insts, results) -> float:
    """Algorithmic FP32 flops of the batch solve: per CG step the two products
    with F (4nk) and the diagonal (n); per iteration A x and A'y (4 nnz(A))."""
    total = 0.0
    for q, r in zip(insts, results):
        total += r["cg_steps"] * (4.0 * q.n * q.k + q.n) + r["iterations"] * 4.0 * len(q.A_col)
    return total


def run_batch_bench(args):
    import numpy as np
    import torch

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2405_16160_b300 import _lib as L
    from paper_2405_16160_b300 import build as B
    from paper_2405_16160_b300 import workloads as W
    from paper_2405_16160_b300.solver import QPBatch, QPSolver

    B.build()
    insts = W.portfolio_batch(BATCH_WORKLOAD["seed"] + rank, BATCH_WORKLOAD["count"])
    tol = BATCH_WORKLOAD["tol"]
    step = L.STEP_ADAPTIVE if args.step == "adaptive" else L.STEP_FIXED
    other = L.STEP_FIXED if step == L.STEP_ADAPTIVE else L.STEP_ADAPTIVE
    stream = torch.cuda.current_stream()
    bt = QPBatch(insts)
    # block sizes per size bin from the autotuner (whole bins, 128 attempts)
    threads = bt.tune(tol=tol, precision=L.PREC_MIXED, step_mode=step, sample_iters=128)
    for _ in range(args.warmup):
        bt.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step)
    with ClockSampler(local) as clocks:
        _barrier(ws)
        torch.cuda.synchronize()
        times, kms = [], []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kms.append(bt.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        _barrier(ws)
    res = bt.results()
    fp64_ms = bt.solve(tol=tol, precision=L.PREC_FP64, step_mode=step)
    res64 = bt.results()
    other_ms = bt.solve(tol=tol, precision=L.PREC_MIXED, step_mode=other)
    res_other = bt.results()
    bt.close()
    # the same instances with long-only written as the bounds x >= 0 (BB x-steps)
    bnds = W.portfolio_batch(BATCH_WORKLOAD["seed"] + rank, BATCH_WORKLOAD["count"], bounds=True)
    with QPBatch(bnds) as bb:
        bb.tune(tol=tol, precision=L.PREC_MIXED, step_mode=step, sample_iters=128)
        bb.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step)
        bounds_ms = statistics.mean(
            bb.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step) for _ in range(2))
        res_b = bb.results()
    obj_diff = max(abs(u["primal_obj"] - v["primal_obj"]) / max(1.0, abs(u["primal_obj"]))
                   for u, v in zip(res, res_b))
    value = _max_over_ranks(statistics.mean(times), ws)
    # plain FP64 GPU PDHCG (the single-QP path), one instance at a time, on a sample
    sample = insts[:16]
    single = []
    for q in sample:
        with QPSolver(q.to_instance()) as s:
            s.solve(tol=tol, step_mode=step)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.solve(tol=tol, step_mode=step)
            torch.cuda.synchronize()
            single.append(time.perf_counter() - t0)
    single_total = statistics.mean(single) * len(insts)
    # end to end from host arrays
    e2e = []
    for i in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with QPBatch(insts) as b2:
            b2.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step)
            b2.results()
            b2.solution()
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(time.perf_counter() - t0)
    h2d = sum(q.F.nbytes + q.qd.nbytes + q.c.nbytes + q.b.nbytes + q.A_rowptr.nbytes
              + q.A_col.nbytes + q.A_val.nbytes for q in insts)
    d2h = sum(8 * (q.n + q.m) for q in insts)
    if rank != 0:
        return 0
    flops = batch_flops(insts, res)
    kernel_s = statistics.mean(kms) / 1e3
    achieved = flops / kernel_s / 1e12
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import pdhcg_oracle as O
        c0, t0 = time.process_time(), time.perf_counter()
        ostep = O.STEP_ADAPTIVE if args.step == "adaptive" else O.STEP_FIXED
        for q in insts[:8]:
            O.solve(O.problem_from_instance(q.to_instance()),
                    O.OracleOptions(tol=tol, step_mode=ostep))
        wall = time.perf_counter() - t0
        cpu = {"value": wall / 8 * len(insts), "unit": "s",
               "cores": round((time.process_time() - c0) / wall, 1), "kind": "oracle",
               "sample": f"oracle solves of the first 8 instances ({wall:.1f} s), scaled to "
                         f"{len(insts)} instances"}
    it = np.array([r["iterations"] for r in res])
    out = {
        "metric": BATCH_METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 iterates and block totals)",
        "data": "synthetic",
        "config": dict(BATCH_WORKLOAD, step=args.step,
                       solved=int(sum(r["termination"] == 0 for r in res)),
                       iterations_mean=float(it.mean()), iterations_max=int(it.max()),
                       attempts_mean=float(np.mean([r["attempts"] for r in res])),
                       other_step_s=other_ms / 1e3,
                       other_step_iterations_mean=float(np.mean(
                           [r["iterations"] for r in res_other])),
                       fp64_batch_s=fp64_ms / 1e3,
                       fp64_solved=int(sum(r["termination"] == 0 for r in res64)),
                       single_qp_fp64_s=single_total,
                       single_qp_fp64_sample="16 instances through qp_solve, one at a time, "
                                             "scaled to 4096",
                       speedup_vs_single_fp64=single_total / value,
                       speedup_vs_fp64_batch=(fp64_ms / 1e3) / value,
                       tuned_threads_largest_bin=threads,
                       bounds_form_s=bounds_ms / 1e3,
                       bounds_form_solved=int(sum(r["termination"] == 0 for r in res_b)),
                       bounds_form_attempts_mean=float(np.mean([r["attempts"] for r in res_b])),
                       bounds_form_objective_max_rel_diff=obj_diff,
                       bounds_form_note="long-only as x >= 0 (Section 4 BB projected-gradient "
                                        "x-steps, m = 1 + sectors); device time of one launch",
                       parallelism=f"replicas x{ws}",
                       l2="per-instance data ~100 MB in total, L2-resident; one launch"),
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"kernel": "k_batch<float> (one block per instance, persistent)",
                     "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_kind": "nominal FP32 (148 SMs x 128 lanes x 2 x 2.032 GHz)",
                     "note": "latency-bound: block barriers and dependent loads per "
                             "iteration, not arithmetic"},
        "cpu_baseline": cpu,
        "gpu_launches": min(4, len(insts)) * args.steps,  # one k_batch launch per size bin
        "clocks": clocks.summary(),
    }
    print(json.dumps(out), flush=True)
    return 0


ZIPF_WORKLOAD = {
    "workload": "largest single QP: n=1e7, m=5e6, Q = diag U[0.5,2] + mirrored N(0,0.1) "
                "(~5 nnz/row, diagonally dominant), A 8 N(0,1) nnz/row with Zipf(1.1) column "
                "popularity through a seeded permutation, c ~ N(0,1), b = A x0 + U[0,1]",
    "n": 10_000_000, "m": 5_000_000, "seed": 0, "tol": 1e-4, "precision": "mixed",
    "scaling": "Section 4: 10 Ruiz steps + Pock-Chambolle on [[Q, A'], [A, 0]]",
    "l2": "inputs larger than L2 (~3.2 GB resident)",
}
ZIPF_METRIC = ("time to 1e-4 rel. KKT on the largest single QP (restarted PDHCG; FP32 "
               "data/iterates, FP64 reductions)")


def run_zipf_bench(args):
    """The largest single QP.  A solve takes about a minute, so each warm-up
    step is a solve capped at 128 attempts (graph capture, caches) and the
    timed region is --steps full solves; the other step rule is timed once."""
    import torch

    ws, rank = _dist()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2405_16160_b300 import _lib as L
    from paper_2405_16160_b300 import build as B
    from paper_2405_16160_b300 import workloads as W
    from paper_2405_16160_b300.solver import QPSolver

    B.build()
    t0 = time.perf_counter()
    inst = W.zipf_dd(ZIPF_WORKLOAD["seed"] + rank, n=ZIPF_WORKLOAD["n"], m=ZIPF_WORKLOAD["m"])
    gen_s = time.perf_counter() - t0
    tol = ZIPF_WORKLOAD["tol"]
    step = L.STEP_ADAPTIVE if args.step == "adaptive" else L.STEP_FIXED
    other = L.STEP_FIXED if step == L.STEP_ADAPTIVE else L.STEP_ADAPTIVE
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    solver = QPSolver(inst, scale=True)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    shapes = solver.tune(reps=5)
    for _ in range(args.warmup):
        solver.solve(tol=tol, precision=L.PREC_MIXED, step_mode=step, max_iter=128)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        _barrier(ws)
        torch.cuda.synchronize()
        infos, times = _timed_solves(solver, args.steps, stream, tol=tol, precision=L.PREC_MIXED,
                                     step_mode=step, time_limit_s=600.0)
        torch.cuda.synchronize()
        _barrier(ws)
    oinfo, otimes = _timed_solves(solver, 1, stream, tol=tol, precision=L.PREC_MIXED,
                                  step_mode=other, time_limit_s=300.0)
    # plain FP64 with the same step rule, allowed to reach the tolerance
    finfo, ftimes = _timed_solves(solver, 1, stream, tol=tol, precision=L.PREC_FP64,
                                  step_mode=step, time_limit_s=600.0)
    kinfos, _ = _timed_solves(solver, 1, stream, tol=tol, precision=L.PREC_MIXED, step_mode=step,
                              kernel_timing=1, max_iter=640)
    solver.close()
    value = _max_over_ranks(statistics.mean(times), ws)
    if rank != 0:
        return 0
    info, oi = infos[-1], oinfo[-1]
    peak, peak_kind = _peaks()
    ki = kinfos[-1]
    kbytes = cg_kernel_bytes(inst.nnz_Q, inst.n, ki["cg_kernel_spmvs"], 4)
    ks = ki["cg_kernel_ms"] / 1e3
    achieved = kbytes / ks / 1e9 if ks > 0 else None
    ceiling = gather_ceiling(inst.nnz_Q, inst.n)
    gathers = ki["cg_kernel_spmvs"] * inst.nnz_Q / ks if ks > 0 else None
    out = {
        "metric": ZIPF_METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 reductions and scalars)",
        "data": "synthetic",
        "config": dict(ZIPF_WORKLOAD, step=args.step, termination=info["termination"],
                       relkkt=info["relkkt"], iterations=info["iterations"],
                       attempts=info["attempts"], cg_steps=info["cg_steps"],
                       restarts=info["restarts"], ms_per_attempt=value * 1e3 / info["attempts"],
                       other_step=("fixed" if args.step == "adaptive" else "adaptive"),
                       other_step_s=otimes[-1], other_step_termination=oi["termination"],
                       other_step_relkkt=oi["relkkt"], other_step_attempts=oi["attempts"],
                       fp64_s=ftimes[-1], fp64_termination=finfo[-1]["termination"],
                       fp64_relkkt=finfo[-1]["relkkt"], fp64_attempts=finfo[-1]["attempts"],
                       speedup_vs_fp64=ftimes[-1] / value,
                       warmup_note="each warm-up solve capped at 128 attempts",
                       generate_s=gen_s, create_s=create_s, tuned_shapes=shapes,
                       parallelism=f"replicas x{ws}"),
        "e2e": None,
        "roofline": {"kernel": "k_cg<float> (persistent CG: Q SpMV + vector phases)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "peak_kind": peak_kind, "gathers_per_s": gathers,
                     "gather_ceiling_per_s": ceiling,
                     "gather_frac": (gathers / ceiling) if gathers and ceiling else None,
                     "timing": "CUDA events around every k_cg launch of a solve capped at "
                               "640 attempts, run after the timed region"},
        "cpu_baseline": None, "gpu_launches": None, "clocks": clocks.summary(),
    }
    print(json.dumps(out), flush=True)
    return 0


WS_WORKLOAD = {
    "workload": "parametric portfolio family: n=2000, k=50 factors, 30 sector caps and the "
                "budget row (m=31), long-only as the variable bounds x >= 0 (Section 4 BB "
                "x-steps); per instance mu ~ N(0.05, 0.02) and F = F0 + 10% Gaussian; network "
                "trained on solver solutions of 20000 instances, judged on 1000 held-out "
                "instances",
    "n": 2000, "train": 20000, "test": 1000, "tol": 1e-4, "hidden": [512, 512],
}
WS_METRIC = ("time to 1e-4 rel. KKT on 1000 held-out portfolio QPs (batched PDHCG): "
             "learned warm start vs cold start")


def run_warmstart_bench(args):
    import numpy as np
    import torch

    ws, rank = _dist()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2405_16160_b300 import _lib as L
    from paper_2405_16160_b300 import build as B
    from paper_2405_16160_b300 import warmstart as WS
    from paper_2405_16160_b300 import workloads as W

    B.build()
    n, tol = WS_WORKLOAD["n"], WS_WORKLOAD["tol"]
    step = L.STEP_ADAPTIVE if args.step == "adaptive" else L.STEP_FIXED
    # training data: solver solutions, generated and solved in chunks
    t0 = time.perf_counter()
    feats, targs, omegas, gen_iters = [], [], [], []
    chunk = 1000
    for s0 in range(1, WS_WORKLOAD["train"] + 1, chunk):
        insts = W.portfolio_family(0, seeds=range(s0, s0 + chunk), n=n, bounds=True)
        res, xs, ys = WS.solve_family(insts, tol=tol, precision=L.PREC_MIXED, step_mode=step)
        keep = [i for i, r in enumerate(res) if r["termination"] == L.TERM_SOLVED]
        feats.append(WS.features([insts[i] for i in keep]))
        targs.append(WS.targets([xs[i] for i in keep], [ys[i] for i in keep]))
        omegas += [res[i]["omega"] for i in keep]
        gen_iters += [res[i]["iterations"] for i in keep]
        del insts
    gen_s = time.perf_counter() - t0
    X, T = np.concatenate(feats), np.concatenate(targs)
    widths = [X.shape[1], *WS_WORKLOAD["hidden"], T.shape[1]]
    net = WS.WarmStartMLP(widths, max_batch=1024)
    net.set_params(WS.he_normal_params(widths, 0))
    t0 = time.perf_counter()
    hist = WS.train(net, X, T, epochs=args.train_epochs, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    model = WS.WarmStartModel(net, n, float(np.median(omegas)))
    test = W.portfolio_family(0, seeds=range(WS_WORKLOAD["train"] + 1,
                                             WS_WORKLOAD["train"] + 1 + WS_WORKLOAD["test"]), n=n,
                              bounds=True)
    cold_t, warm_t = [], []
    cold_ph, warm_ph = {}, {}
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    for rep_i in range(args.warmup + args.steps):
        if rep_i == args.warmup:
            clocks.__enter__()
        timed = rep_i >= args.warmup
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cold, _, _ = WS.solve_family(test, tol=tol, precision=L.PREC_MIXED, step_mode=step,
                                     phases=cold_ph if timed else None)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hot, _, _, n_fb = model.solve(test, tol=tol, precision=L.PREC_MIXED, step_mode=step,
                                      phases=warm_ph if timed else None)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if rep_i >= args.warmup:
            cold_t.append(t1 - t0)
            warm_t.append(t2 - t1)
    clocks.__exit__(None, None, None)
    it_c = float(np.mean([r["iterations"] for r in cold]))
    it_w = float(np.mean([r["iterations"] for r in hot]))
    value = statistics.mean(warm_t)
    if rank != 0:
        return 0
    out = {
        "metric": WS_METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 vectors and reductions)",
        "data": "synthetic",
        "config": dict(WS_WORKLOAD, step=args.step, cold_start_s=statistics.mean(cold_t),
                       speedup_vs_cold=statistics.mean(cold_t) / value,
                       iterations_cold=it_c, iterations_warm=it_w,
                       iteration_ratio=it_w / it_c, fallbacks=n_fb,
                       solved_warm=int(sum(r["termination"] == 0 for r in hot)),
                       omega0=model.omega0, train_loss_first=hist[0], train_loss_last=hist[-1],
                       train_epochs=args.train_epochs, data_generation_s=gen_s,
                       data_generation_iterations_mean=float(np.mean(gen_iters)),
                       training_s=train_s,
                       cold_phases={k: v / args.steps for k, v in cold_ph.items()},
                       warm_phases={k: v / args.steps for k, v in warm_ph.items()},
                       timing="wall clock of create + solve + solution per 1000-instance "
                              "batch, prediction included in the warm arm"),
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": int(sum(
                    q.F.nbytes + q.qd.nbytes + q.c.nbytes + q.b.nbytes + q.A_val.nbytes
                    + q.A_col.nbytes + q.A_rowptr.nbytes + q.lo.nbytes + q.hi.nbytes
                    for q in test)),
                "d2h_bytes_per_step": int(8 * sum(q.n + q.m for q in test))},
        "roofline": None, "cpu_baseline": None, "gpu_launches": None,
        "clocks": clocks.summary(),
    }
    print(json.dumps(out), flush=True)
    net.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shapes", choices=["tuned", "rule"], default="tuned",
                    help="row kernels' launch shapes: qp_tune's (default) or the rule's")
    ap.add_argument("--no-largest", action="store_true",
                    help="skip the largest-QP (n = 1e7) per-attempt record of the default run")
    ap.add_argument("--workload", choices=["sparse_dd", "portfolio_batch", "learned_warm_start",
                                           "zipf_dd"], default="sparse_dd")
    ap.add_argument("--train-epochs", type=int, default=30)
    ap.add_argument("--step", choices=["adaptive", "fixed"], default="adaptive",
                    help="step-size rule (Section 4 adaptive, or eta = 1/(2||A||_2))")
    ap.add_argument("--oracle-solve", action="store_true",
                    help="internal: one full oracle solve of the bench instance, as JSON")
    args = ap.parse_args()
    if args.oracle_solve:
        print(json.dumps(oracle_full_solve(args.step)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "portfolio_batch":
        return run_batch_bench(args)
    if args.workload == "learned_warm_start":
        return run_warmstart_bench(args)
    if args.workload == "zipf_dd":
        return run_zipf_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
