"""The benchmark's JSON line: the keys a reader of the line relies on.

The CPU test runs the reference arm (the oracle) for a few steps; the GPU
test runs the default arm with a short timed region.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=timeout, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_line():
    line = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert BASE_KEYS <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "MLUPS"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


@pytest.mark.gpu
def test_gpu_arm_line():
    line = _run("--steps", "200", "--warmup", "3", "--no-cpu-baseline")
    assert BASE_KEYS <= set(line)
    assert line["value"] > 1000.0 and line["n_gpus"] == 1 and line["gpu_launches"] == 200
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0.0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    e = line["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in line["clocks"] and line["diag"]["status"] == 0
