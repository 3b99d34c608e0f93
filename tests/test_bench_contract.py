"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on the host cores),
on a small grid so that it runs in seconds on the CPU: one line, the keys the benchmark
contract names, and the reference arm's fixed fields."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "2", "--warmup", "1", "--n", "24")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "steps/s" and d["higher_is_better"] is True
    # ms_per_step: wall time of one timed sample (what ran); value: the sample scaled to a full step
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["extrapolated_ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["extrapolated_ms_per_step"]
    assert isinstance(d["config"], dict) and "workload" in d["config"]
    assert d["config"]["cg_forcing"] == 0.0  # the oracle solves every CG system to cg_rtol
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert cb["host"]["nproc"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
