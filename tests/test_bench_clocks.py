"""Clock record of bench.py (no GPU): only samples taken inside the timed
region count, the median SM clock is reported, and throttle reasons that
were active are named."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sampler(lines, start):
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    s.start = start
    return s


def test_only_samples_inside_the_region_count():
    # start-up sample at a low clock before the region, three inside
    lines = ["1005, 2070, 300.1, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
             "2055, 2070, 950.0, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 960.2, Not Active, Not Active, Not Active, Not Active"]
    r = _sampler(lines, 1).summary()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_region_shorter_than_the_sampling_period_uses_the_last_sample():
    lines = ["1980, 2070, 700.0, Not Active, Not Active, Not Active, Not Active"]
    r = _sampler(lines, 1).summary()
    assert r["samples"] == 1 and r["sm_mhz"] == 1980.0


def test_malformed_lines_are_skipped_and_hw_reasons_reported():
    lines = ["garbage", "",
             "1400, 2070, 1400.0, Active, Not Active, Active, Not Active",
             "[N/A], 2070, 1400.0, Not Active, Not Active, Not Active, Not Active"]
    r = _sampler(lines, 0).summary()
    assert r["samples"] == 1
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler([], 0).summary()["samples"] == 0
