"""The bench's reference arm (the CPU oracle timed on the same workload) on CPU.

Checks the one-line JSON contract of `bench.py --impl reference` and that under
a two-rank launch only rank 0 does the work and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "spheres8_grid7x14", "--steps", "2", "--warmup", "1"]


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def _check_line(line, n_gpus):
    assert line["impl"] == "reference"
    assert line["metric"] == "LCP solves/s" and line["unit"] == "LCP solves/s"
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["n_gpus"] == n_gpus and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    # the value is one LCP solve's worth of measured, complete oracle solves
    assert cpu["fine_gmres_iterations"] > 0 and cpu["fine_solve_seconds"] > 0
    m = cpu["mvps_per_lcp"]
    t = (1 + m["hi"]) * cpu["fine_solve_seconds"] + m["lo"] * cpu["coarse_solve_seconds"]
    assert abs(line["value"] - 1.0 / t) <= 1e-9 * line["value"]
    assert "complete" in cpu["sample"]
    c1 = cpu["c1_complete_solve"]
    for arm in ("single_core", "all_cores"):
        assert c1[arm]["seconds"] > 0 and c1[arm]["kkt"] < 1e-10
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("spheres8_grid7x14:")


def test_reference_arm_single_rank():
    res = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_two_ranks_rank0_only():
    pytest.importorskip("torch")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", *ARGS[:-4],
           "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1           # rank 1 exits without work or output
    _check_line(lines[0], 2)
