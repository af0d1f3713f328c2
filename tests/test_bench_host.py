"""Host-side logic of bench.py, on the CPU: the clock-log summary, the
source-hash gate on the reported DRAM traffic, and the JSON line of the
reference arm (the float64 oracle timed on the host cores)."""

import json
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    s.lines.append("0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active")
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    empty = bench.ClockSampler(0)
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_measured_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    # the figure of the committed summary, or None if the kernel changed since it
    v = bench.measured_traffic()
    assert v is None or v > 0
    # a copy of the tree behaves the same; one edited kernel source reports none
    for rel in bench.HDDA_SOURCES + [bench.HDDA_STRUCTS[0], bench.TRAFFIC_PROFILE]:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic() == v
    with open(tmp_path / bench.HDDA_SOURCES[0], "a") as fh:
        fh.write("\n// edit\n")
    assert bench.measured_traffic() is None


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "seg-lambda/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "probes" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD
