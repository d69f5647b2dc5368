"""bench.py's JSON line.

The reference arm (the FP64 oracle on host cores, no GPU): one line with the
main arm's metric, unit and direction, the oracle described as the CPU
baseline, and an end-to-end entry without host-device copies.  The main arm
(GPU): a short run carrying every key of the contract.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "1080p encode+decode frames/s"
    assert d["unit"] == "frames/s" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("1080p")


@pytest.mark.gpu
def test_main_arm_json_contract():
    """a short run of the main arm: every key the line must carry"""
    args = ["--steps", "3", "--warmup", "3", "--batch", "4", "--frames", "4", "--e2e-steps", "3",
            "--serve-seconds", "0.5", "--no-scalable", "--no-rd", "--no-taps", "--motion-range", "0",
            "--no-suite", "--cpu-workers", "2"]
    out = subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and r["path_frac"] == r["frac"]
    # counters appear only while they were taken on the current kernel sources
    assert r["traffic"] is None or r["traffic"] > 0
    assert r["binding_roof"] in ("hbm", "alu") and 0 < r["frac_of_binding_roof"]
    ds = r["dominant_stage"]
    assert ds["stage"] in r["stages_ms_per_frame"] and 0 < ds["frac"] < 1.5
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] == 1 and cb["nproc"] >= 1
    assert cb["all_cores"]["cores"] == 2 and cb["all_cores"]["value"] > 0
    pe = d["plain"]["e2e_async"]
    assert pe["value"] > 0 and pe["h2d_bytes_per_step"] > 0 and pe["d2h_bytes_per_step"] > 0
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0 and d["clocks"]["sm_max_mhz"] > 0
