"""The bench's multi-process path on CPU: two gloo ranks under torch.distributed.run.

bench.py runs one independent replica per GPU (the solver has no cross-GPU
exchange) and reports the time of the slowest rank.  These tests check the
host side of that: rank discovery from the launcher's environment, the max
over ranks and the barrier, with world_size 2 on the gloo backend.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_two_ranks(tmp_path, body: str):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, os, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        dist.init_process_group("gloo")
        import bench
        ws, rank = bench._dist()
        out = {{"rank": rank, "ws": ws}}
    """) + textwrap.dedent(body) + textwrap.dedent(f"""
        with open(os.path.join({str(tmp_path)!r}, f"rank{{rank}}.json"), "w") as f:
            json.dump(out, f)
        dist.destroy_process_group()
    """))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", str(script)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env, cwd=ROOT)
    assert p.returncode == 0, p.stdout + p.stderr
    res = []
    for r in range(2):
        with open(tmp_path / f"rank{r}.json") as f:
            res.append(json.load(f))
    return res


def test_max_over_ranks_and_barrier_with_two_gloo_ranks(tmp_path):
    res = _run_two_ranks(tmp_path, """
        # each rank's own time: rank 1 is the slower one
        t = 0.25 if rank == 0 else 0.75
        bench._barrier(ws)
        out["max"] = bench._max_over_ranks(t, ws)
        bench._barrier(ws)
    """)
    assert [r["rank"] for r in res] == [0, 1]
    assert all(r["ws"] == 2 for r in res)
    assert all(r["max"] == 0.75 for r in res)  # whole-job time = the slowest rank's


def test_single_process_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(1.5, 1) == 1.5
    bench._barrier(1)  # a no-op without torch.distributed
