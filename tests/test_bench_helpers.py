"""bench.py's host-side helpers: the clock-sample summary and the CPU reference arm's JSON line
(run on the small 64^3 workload).  No GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks()
    c.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1980", "2070", "1390.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2040", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"]]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_without_samples():
    c = bench.Clocks()
    assert c.summary()["reasons"] == ["unavailable"]


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["extrapolated"] is True and d["cpu_baseline"]["iterations_used"] > 0
    # the same config keys and values as the GPU arm prints
    import synth

    class A:
        workload = "c1"
    assert d["config"] == bench.config_of(A, synth.problem("c1"), 1)
