"""The clock record bench.py attaches to its line: nvidia-smi CSV samples
(index, sm, max sm, power, active reasons, hw_slowdown, hw_thermal_slowdown,
sw_thermal_slowdown, sw_power_cap) summarised as median SM clock, maximum
clock and the throttle reasons seen. CPU only: the samples are given."""
import bench


def _summary(lines):
    c = bench.Clocks(0)
    c.lines = list(lines)
    return c.summary()


def test_quiet_samples():
    s = _summary(["0, 2032, 2032, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                  "0, 2032, 2032, 720.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                  "0, 1980, 2032, 730.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"])
    assert s == {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": [], "samples": 3}


def test_throttle_reasons_are_reported():
    s = _summary(["0, 1500, 2032, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
                  "0, 1400, 2032, 1100.0, 0x48, Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1450.0 and s["samples"] == 2


def test_malformed_lines_are_skipped():
    s = _summary(["", "0, [N/A], 2032, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                  "garbage", "0, 2000, 2032, 5.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 1 and s["sm_mhz"] == 2000.0
    assert _summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
