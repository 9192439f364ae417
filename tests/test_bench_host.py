"""Host-side pieces of bench.py on the CPU: the clock record that decides
whether a timed run is kept (median SM clock, maximum, throttle reasons) and
the latency percentiles of the serving report."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx=2070, reasons=("Not Active",) * 4):
    return ["0", str(sm), str(mx), "600.0", "0x0"] + list(reasons)


def test_clock_summary_median_and_reasons():
    c = bench.Clocks(0)
    c.rows = [_row(2070), _row(2070), _row(1980, reasons=("Not Active", "Not Active",
                                                           "Not Active", "Active")),
              _row("[N/A]")]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_flags_thermal_and_hw_slowdown():
    c = bench.Clocks(0)
    c.rows = [_row(1500, reasons=("Active", "Not Active", "Active", "Not Active"))]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    c = bench.Clocks(0)
    assert c.summary() is None


def test_percentiles():
    v = list(range(1, 101))
    assert bench._pct(v, 50) == 50.5
    assert abs(bench._pct(v, 99) - 99.01) < 1e-9
    assert bench._pct([], 50) is None
