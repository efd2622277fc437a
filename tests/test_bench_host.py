"""Host logic of bench.py that needs no GPU: the clock sampler's parsing and windows."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts, sm, reason_cap="Not Active", thermal="Not Active"):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, {thermal}, {reason_cap}"


def test_clock_summary_and_windows():
    s = bench.ClockSampler(0)
    t = 1.7e9
    s.lines = [_line(t + 0.1 * i, 2070 if i != 7 else 1500, "Active" if i == 3 else "Not Active")
               for i in range(20)]
    s.lines.append("garbage line")
    whole = s.summary(t - 0.01, t + 2.0)
    assert whole["samples"] == 20 and whole["sm_mhz"] == 2070 and whole["sm_mhz_min"] == 1500
    assert whole["reasons"] == ["sw_power_cap"] and whole["sm_max_mhz"] == 2070
    part = s.summary(t + 0.25, t + 0.55)  # samples 3, 4, 5
    assert part["samples"] == 3 and part["reasons"] == ["sw_power_cap"]
    assert s.windows_min([(t + 0.65, t + 0.75), (t + 0.05, t + 0.15), (t + 5, t + 6)]) == [1500, 2070, None]
    assert s.summary(t + 5, t + 6) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_thermal_reason_is_reported():
    s = bench.ClockSampler(0)
    t = 1.7e9
    s.lines = [_line(t, 1900, thermal="Active")]
    assert s.summary(t - 1, t + 1)["reasons"] == ["sw_thermal_slowdown"]
