"""Host-side logic of bench.py that needs no GPU: the clock and throttle-reason summary of the
sampled nvidia-smi lines, and the peak bandwidth source."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = object()                       # as if the sampler had run
    return c.summary()


def test_clock_summary_median_and_no_reason(tmp_path):
    rows = ["0, %d, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active" % mhz
            for mhz in (2070, 2055, 2070, 1980, 2070)]
    s = _summary(tmp_path, rows)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == [] and s["samples"] == 5


def test_clock_summary_reports_throttle_reasons(tmp_path):
    rows = ["0, 1800, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1500, 2070, 1400.0, 0x0000000000000048, Active, Not Active, Active, Not Active",
            "malformed line", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _summary(tmp_path, rows)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["samples"] == 2 and s["sm_mhz"] in (1500.0, 1800.0)


def test_clock_summary_without_sampler():
    c = bench.Clocks(0)
    c.path = "/nonexistent/clocks.csv"
    assert c.summary()["sm_mhz"] is None


def test_measured_peaks_source():
    peaks, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peaks == json.load(open(path))
    else:
        assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
    assert peaks["hbm_gbs"] > 1000.0


def test_kernel_source_hash_is_sha1_hex():
    h = bench.kernel_source_sha1()
    assert len(h) == 40 and int(h, 16) >= 0
