"""Host-side parts of the benchmark's output contract (CPU only): the clock-sample summary that
decides whether a run is kept, and the reference arm's JSON line (the FP64 oracle timed on a
bounded sample of the layered update)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary():
    na, act = "Not Active", "Active"
    lines = [
        f"0, 2070, 2070, 980.1, 0x0000000000000000, {na}, {na}, {na}, {na}",
        f"0, 1995, 2070, 1390.0, 0x0000000000000004, {na}, {na}, {na}, {act}",
        f"0, 2070, 2070, 1200.0, 0x0000000000000000, {na}, {na}, {na}, {na}",
        "0, [N/A], 2070, 0.0, 0x0, x, x, x, x",  # unreadable sample: skipped
        "garbage",
    ]
    out = bench.ClockSampler.parse(lines)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    hot = bench.ClockSampler.parse([f"0, 1500, 2070, 900, 0x8, {na}, {act}, {na}, {na}"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.ClockSampler.parse([]) is None


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["value"] > 0 and d["steps"] == 1
    assert d["config"]["workload"].startswith("layered-faulted 921x301")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
