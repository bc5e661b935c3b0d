"""Host logic of bench.py that needs no GPU: the clock-sample parsing whose
throttle reasons decide whether a run is kept, and the arithmetic of the
instruction-issue roofline."""
import bench


def test_clock_samples_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1010.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "garbage",
    ]
    c = bench.parse_clocks(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    hot = lines[:1] + ["0, 1500, 2070, 1200.0, 0x48, Active, Not Active, Active, Not Active"]
    c = bench.parse_clocks(hot)
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clocks([])["reasons"] == ["no samples"]


def test_issue_roofline_arithmetic():
    """achieved = warp instructions per draw x draws per update x updates per
    step / collision time per step; peak = 4 warp schedulers x the SM count x
    the SM clock."""
    r = bench.issue_roofline(10.0, 1.0e6, 0.25, {"sm_mhz": 2000.0}, 152)
    assert abs(r["peak"] - 4 * 152 * 2.0) < 1e-9                   # Gwarp-inst/s
    assert abs(r["achieved"] - bench.PUSH_WARP_INST_PER_DRAW * 10.0 * 1.0e6 / 0.25e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
