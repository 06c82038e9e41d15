"""The reference arm of bench.py (the FP64 oracle on the host cores) prints
one JSON line with the keys the bench contract asks for, on the small
16^3x32 workload; no GPU is involved.  Under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "16c32", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_json_line():
    lines = run_bench()
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["unit"] == "GFLOP/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert "16x16x16x32" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "oracle" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_reports_the_threads_used():
    d = run_bench({"OMP_NUM_THREADS": "2"})[0]
    assert d["cpu_baseline"]["cores"] == 2


def test_reference_arm_other_ranks_print_nothing():
    assert run_bench({"RANK": "1"}) == []


def test_failing_side_leg_is_reported_in_place(capsys):
    """A comparison leg that raises is reported as {"error": ...} in its
    place (and on stderr) instead of costing the run its JSON line; a leg
    that works returns its result unchanged."""
    import bench

    def broken():
        raise RuntimeError("device busy")

    out = bench.guarded("solve", broken)
    assert out == {"error": "RuntimeError: device busy"}
    assert "leg solve failed" in capsys.readouterr().err
    assert bench.guarded("ok", lambda a, b: a + b, 2, 3) == 5
