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
    lines = [_line(2070, 2070), _line(2055, 2070, cap="Active"), _line(1980, 2070), "garbage", "0, N/A, 2070"]
    cs.lines = [(1.0 + 0.01 * i, ln) for i, ln in enumerate(lines)]
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines = [(1.0, _line(1500, 2070, hw="Active", swt="Active"))]
    assert bench.ClockSampler(0).summary()["samples"] == 0
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_counts_the_timed_region():
    # samples read 20 ms apart; the timed region covers host times 1.05 .. 1.095:
    # the samples read inside it or within one period after its end (1.06, 1.08,
    # 1.10) are the in-region ones, the rest belong to the padded window
    cs = bench.ClockSampler(0)
    cs.lines = [(1.0 + 0.02 * i, _line(2070 - i, 2070)) for i in range(10)]
    cs.mark(1.05, 1.095)
    s = cs.summary()
    assert s["samples"] == 3 and s["samples_window"] == 10
    assert s["sm_mhz"] == 2066          # median of 2067, 2066, 2065 (read at 1.06, 1.08, 1.10)


def test_algorithmic_bytes_of_the_interpolation_launches():
    N, B = 1 << 24, 32
    assert bench.launch_bytes("interp_top", N, B) == (8 + 6 / 32) * N
    assert bench.launch_bytes("interp_inv_fwd", N, B) == 8 * N
    assert bench.launch_bytes("effdim_classes", N, B) is None
    fams = {"interp_top": (32, 32 * 0.05)}          # 32 launches of 50 us
    r = bench.roofline("interp_top", fams, N, B, 6000.0, "measured")
    assert abs(r["achieved"] - (8 + 6 / 32) * N / 50e-6 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12


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
