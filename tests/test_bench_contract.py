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
    line = _run("--steps", "200", "--warmup", "3", "--no-cpu-baseline", "--no-extras")
    assert BASE_KEYS <= set(line)
    regions = line["repeats"]["regions"]
    assert 5 <= regions <= 20
    assert line["value"] > 1000.0 and line["n_gpus"] == 1 and line["gpu_launches"] == 200 * regions
    assert line["repeats"]["mlups_min"] <= line["value"] <= line["repeats"]["mlups_max"]
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0.0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    e = line["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in line["clocks"] and line["diag"]["status"] == 0
    if "issue_roofline" in line:  # present while the committed instruction count matches the build
        i = line["issue_roofline"]
        assert i["bound"] == "issue" and 0.0 < i["frac"] < 1.0 and abs(i["frac"] - i["achieved"] / i["peak"]) < 1e-3


@pytest.mark.gpu
def test_gpu_arm_line_carries_the_16bit_batch_and_serving_results():
    line = _run("--steps", "20", "--warmup", "3", "--no-cpu-baseline", "--serve-requests", "6",
                "--serve-max-steps", "5000")
    for storage in ("fp16", "bf16"):
        e = line[storage]
        assert e["value"] > 1000.0 and 0.0 < e["roofline_frac"] < 1.5 and e["status"] == 0
        assert e["nu_rel_diff_vs_fp32"] < 0.05
    b = line["batch"]
    assert b["value"] > 1000.0 and b["config"]["nodes"] > 0 and b["nu_vs_oracle"]
    assert all(n["rel_err"] < 0.01 for n in b["nu_vs_oracle"])
    sv = line["serving"]
    assert sv["solves_per_s"] > 0 and sv["p99_latency_s"] >= sv["p50_latency_s"] > 0
    assert sv["sequential_fp32"]["solves_per_s"] > 0


def test_committed_counters_are_used_only_for_the_sources_they_were_taken_on(tmp_path, monkeypatch):
    """The roofline's `traffic` and the issue roofline's instruction count come
    from the committed ncu summary only while its hash matches the step
    kernels' sources and nvcc flags."""
    sys.path.insert(0, ROOT)
    import bench
    p = tmp_path / "counters.json"
    key = "k_step3_tma_fp32_1024x2048"
    monkeypatch.setattr(bench, "PROFILE_JSON", str(p))
    p.write_text(json.dumps({key: {"kernel_source_sha256_16": bench.kernel_source_hash(),
                                   "dram_bytes_per_launch": 123, "warp_instructions_per_launch": 456}}))
    assert bench.counters_for(key) == 123
    assert bench.counters_for(key, "warp_instructions_per_launch") == 456
    p.write_text(json.dumps({key: {"kernel_source_sha256_16": "0" * 16, "dram_bytes_per_launch": 123}}))
    assert bench.counters_for(key) is None
    assert bench.counters_for("no_such_kernel") is None

