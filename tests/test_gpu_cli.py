"""The command-line solve of a generated workload (paper_2405_16160_b300.solve)."""
import json

import pytest

from paper_2405_16160_b300 import solve as S

pytestmark = pytest.mark.gpu


def test_cli_solves_a_small_workload(capsys):
    assert S.main(["--workload", "sparse_dd", "--n", "20000", "--m", "10000", "--repeat", "2"]) == 0
    lines = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 2 and "create_s" in lines[0] and "create_s" not in lines[1]
    for d in lines:
        assert d["termination"] == 0 and d["relkkt"] <= 1e-4 and d["device_s"] > 0
    assert lines[0]["attempts"] == lines[1]["attempts"]  # repeat solves are identical


def test_cli_iteration_cap():
    import io
    import contextlib
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        S.main(["--workload", "zipf_dd", "--n", "20000", "--m", "10000", "--max-iter", "64",
                "--tol", "1e-12", "--precision", "fp64"])
    d = json.loads(buf.getvalue().splitlines()[-1])
    assert d["attempts"] == 64 and d["termination"] == 1  # QP_TERM_ITERATION_LIMIT
