"""CPU checks of bench.py's reference arm (the oracle timed on the host): the
JSON line carries every key of the bench contract, and ranks other than 0
print nothing."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


@pytest.mark.parametrize("workload,side,extra", [("box25-8192", 192, []), ("star7-512", 24, []),
                                                ("box125-512", 16, []), ("star7-512", 20, ["--bc", "periodic"])])
def test_reference_arm_line(workload, side, extra):
    out = run_bench(["--impl", "reference", "--workload", workload, "--side", str(side), "--steps", "2",
                     "--warmup", "1"] + extra)
    line = json.loads(out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "GStencil/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert str(side) in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    out = run_bench(["--impl", "reference", "--side", "64", "--steps", "1", "--warmup", "0"],
                    {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""


def test_workload_options():
    """--bc overrides the workload's boundary; box125-512 is the order-2 3D box."""
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--workload", "star7-512", "--bc", "periodic", "--side", "12"]
        p = bench.workload(bench.parse())
        assert p.bc == "periodic" and p.shape == (12, 12, 12) and p.r == 1
        sys.argv = ["bench.py", "--workload", "box125-512", "--side", "10", "--tsteps", "3"]
        p = bench.workload(bench.parse())
        assert p.bc == "dirichlet" and p.r == 2 and p.kind == "box" and p.coeffs.shape == (5, 5, 5) and p.steps == 3
        sys.argv = ["bench.py"]
        p = bench.workload(bench.parse())
        assert p.bc == "periodic" and p.shape == (8192, 8192) and p.r == 2
    finally:
        sys.argv = old
