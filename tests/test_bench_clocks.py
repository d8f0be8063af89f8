"""The benchmark's clock summary (CPU): median and minimum SM clock, power,
and the throttle reasons that were active in any sample, from nvidia-smi's
CSV lines (index, sm, max sm, power, active mask, hw_slowdown,
hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def summary(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clean_run():
    s = summary(["0, 2070, 2070, 489.8, 0x0, Not Active, Not Active, Not Active, Not Active",
                 "0, 2070, 2070, 501.2, 0x0, Not Active, Not Active, Not Active, Not Active",
                 "0, 2055, 2070, 510.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] == 2070 and s["sm_mhz_min"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["power_w"] == 501.2 and s["reasons"] == [] and s["samples"] == 3


def test_reasons_from_any_sample():
    s = summary(["0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                 "0, 1500, 2070, [N/A], 0x8, Active, Not Active, Active, Not Active",
                 "garbage line"])
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["samples"] == 2 and s["power_w"] == 1390.0 and s["sm_mhz_min"] == 1500


def test_unsampled():
    assert summary([])["reasons"] == ["unsampled"]
