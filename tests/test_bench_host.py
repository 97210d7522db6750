"""Host-side pieces of the benchmark (no GPU): the clock summary of sampled
nvidia-smi lines, the whole-job rate, the peak lookup, and the recorded DRAM
traffic being tied to the kernel source it was measured on."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %d, %d, 900.00, 0x0000000000000000, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, cap)


def test_clock_summary_median_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [_line(2070, 2070), _line(2055, 2070, cap="Active"), _line(1980, 2070), "garbage", "0, N/A, 2070"]
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines = [_line(1500, 2070, hw="Active", swt="Active")]
    assert bench.ClockSampler(0).summary()["samples"] == 0
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_whole_job_rate_counts_every_rank():
    # 4 ranks of 1e6 units each, slowest rank 2 ms: 2e9 units/s
    assert bench.whole_job_rate(1e6, 4, 2.0) == 2e9
    assert bench.max_over_ranks(3.5, None, None) == 3.5


def test_peaks_from_measured_file():
    peak, kind = bench._peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == json.load(open(path))["hbm_gbs"]
    else:
        assert kind == "fallback"


def test_traffic_is_tied_to_the_measured_source():
    src = open(os.path.join(ROOT, bench.MEASURED_TRAFFIC["source"]), "rb").read()
    if hashlib.sha256(src).hexdigest() == bench.MEASURED_TRAFFIC["sha256"]:
        assert bench._traffic("interp_top") == bench.MEASURED_TRAFFIC["bytes_per_launch"]["interp_top"]
    else:
        assert bench._traffic("interp_top") is None
    assert bench._traffic("no_such_kernel") is None
