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


def test_qr_roofline_forms(monkeypatch):
    """The bench's roofline of the fine systems' QR: with the tensor-core
    stages, bound by the ALU pipe at the capture's flops per ALU instruction
    x 152 SMs x 2 instructions per clock x the clock (null once the kernel
    sources no longer hash to the capture's), with the FP64 pipe's peak beside
    it; with FP64 stages, bound by the FP64 peak."""
    sys.path.insert(0, ROOT)
    import bench
    fp64 = 152 * 2 * 2 * 2070e6 / 1e12
    r = bench.rqr_roofline(True, True, 2.5, fp64, 2070.0, 6.4e12, 7.7e12, 3000.0, 4600.0)
    assert r["bound"] == "alu"
    if bench.rqr_counters_valid():
        peak = bench.RQR_FLOPS_PER_ALU_INST * 152 * 2 * 2070e6 / 1e12
        assert abs(r["peak"] - peak) < 1e-12 and abs(r["frac"] - 2.5 / peak) < 1e-12
    assert abs(r["vs_fp64_pipe_peak"] - 2.5 / fp64) < 1e-12
    assert abs(r["share_of_step"] - 3000.0 / 4600.0) < 1e-12
    monkeypatch.setattr(bench, "RQR_SRC_SHA256", "0" * 64)
    r = bench.rqr_roofline(True, True, 2.5, fp64, 2070.0, None, 7.7e12, 3000.0, 4600.0)
    assert r["peak"] is None and r["frac"] is None
    r = bench.rqr_roofline(False, True, 0.98, fp64, 2070.0, None, 7.7e12, 7800.0, 10000.0)
    assert r["unit"] == "TFLOP/s (FP64)" and abs(r["frac"] - 0.98 / fp64) < 1e-12
