"""The bench's clock record, from nvidia-smi's CSV rows (format=csv,noheader,
nounits; fields: clocks.sm, clocks.max.sm, power.draw, the active-reasons mask,
then hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rows(text):
    return [[x.strip() for x in line.split(",")] for line in text.strip().splitlines()]


def test_clock_summary_median_max_and_reasons():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks()
    c.rows = rows("""
        1980, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
        2010, 2070, 1210.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active
        [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]
        1995, 2070, 1300.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
    """)
    s = c.summary()
    assert s["sm_mhz"] == 1995.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_hardware_slowdown():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks()
    c.rows = rows("""
        1500, 2070, 1400.0, 0x0000000000000048, Active, Not Active, Not Active, Not Active
        1450, 2070, 1398.0, 0x0000000000000068, Not Active, Active, Active, Not Active
    """)
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1475.0


def test_clock_summary_without_samples():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks()
    s = c.summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
