"""Host logic of bench.py's per-step timing (no GPU): batch records become
per-step device times charged to radius classes."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_batches_charge_their_steps_by_radius_class():
    # three batches at 1000 MHz (1000 cycles per microsecond): one step of
    # radius 9 taking 4000 cycles, two of radius 3 taking 2000 cycles in all,
    # then four single-voxel steps in 400 cycles
    rec = [[0, 1, 4000, 0], [1, 2, 2000, 0], [3, 4, 400, 1]]
    r2 = np.array([81, 9, 9, 1, 1, 1, 1, 5])   # entries past K are ignored
    s = bench.step_time_stats(rec, r2, 7, span_cycles=10_000, span_ns=10_000)
    assert abs(s["sm_mhz_in_kernel"] - 1000.0) < 1e-9
    c = s["by_radius"]
    assert c["r>8"]["steps"] == 1 and abs(c["r>8"]["p50_us"] - 4.0) < 1e-9
    assert c["2<r<=4"]["steps"] == 2 and abs(c["2<r<=4"]["p99_us"] - 1.0) < 1e-9
    assert c["r=1"]["steps"] == 4 and abs(c["r=1"]["mean_us"] - 0.1) < 1e-9
    assert c["1<r<=2"]["steps"] == 0 and c["4<r<=8"]["steps"] == 0
    assert s["all"]["steps"] == 7
    assert s["batches"] == 3 and s["batches_single_voxel_loop"] == 1
    assert abs(s["traced_fraction_of_kernel"] - 0.64) < 1e-9


def test_records_that_do_not_tile_the_steps_are_rejected():
    r2 = np.ones(8, dtype=np.int64)
    assert bench.step_time_stats([[0, 2, 10, 0], [3, 2, 10, 0]], r2, 4, 1, 1) is None   # gap
    assert bench.step_time_stats([[0, 2, 10, 0]], r2, 3, 1, 1) is None                  # short
    assert bench.step_time_stats([], r2, 0, 1, 1) is None


def test_clock_samples_report_median_and_throttle_reasons():
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clock_samples(text)
    assert c["samples"] == 3 and c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clock_samples("0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active")
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.parse_clock_samples("") is None
