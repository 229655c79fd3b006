"""Host-side pieces of bench.py's line, CPU only:
- the clock record: nvidia-smi CSV samples (index, sm, max sm, power,
  active reasons, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
  sw_power_cap) summarised as median SM clock, maximum clock and the
  throttle reasons seen;
- the roofline's traffic figure, reported only while the scan source is
  the one its DRAM counters were taken on."""
import hashlib
import os

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


def test_traffic_only_for_the_captured_source(monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2106_14038_b300", "csrc", "gs_scan.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    monkeypatch.setattr(bench, "SCAN_TRAFFIC", {"w": (sha[:12], 123), "old": ("0" * 12, 456),
                                                "none": (sha[:12], None)})
    assert bench._scan_traffic("w") == 123
    assert bench._scan_traffic("old") is None
    assert bench._scan_traffic("none") is None
    assert bench._scan_traffic("unknown") is None
