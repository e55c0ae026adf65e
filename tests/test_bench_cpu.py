"""Host-side logic of bench.py without a GPU: the clock-record summary that
decides whether a run is accepted, and the two error measures of the
time-to-solution comparison (Sec. 5.2.1 area rate, Sec. 5.2.2 front
position)."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _summary(lines):
    s = bench.ClockSampler(0)
    s.proc = _DoneProc()
    s.out = list(lines)
    return s.stop()


def test_clock_summary_median_max_and_reasons():
    ok = "0, %d, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, %s"
    lines = [ok % (mhz, "Not Active") for mhz in (2070, 2040, 2070, 1995, 2070)]
    lines.append("garbage line")
    lines.append(ok % (2070, "Active"))                         # power cap seen once: kept and named
    s = _summary(lines)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 6
    assert s["reasons"] == ["sw_power_cap"]
    thermal = "0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = _summary([thermal] * 3)
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_area_rate_error_of_the_exact_law():
    # A(t) = A0 - 2 pi M gamma t (Sec. 5.2.1) has zero error; a 3 % slower
    # shrinkage has 3 %
    ts = np.linspace(0.0, 400.0, 11)
    for M, g in ((1.0, 1.0), (0.5, 2.0)):
        A = 5000.0 - 2 * math.pi * M * g * ts
        assert bench._area_rate_error(ts, A, M, g) == pytest.approx(0.0, abs=1e-12)
        A = 5000.0 - 0.97 * 2 * math.pi * M * g * ts
        assert bench._area_rate_error(ts, A, M, g) == pytest.approx(0.03, rel=1e-9)


def test_front_position_of_a_cubic_profile():
    # the cubic through the four cell centres nearest the 0.5 crossing is
    # exact for a profile that is itself a cubic near the front
    x = np.arange(40) + 0.5
    x0 = 17.3
    prof = np.clip(0.5 + 0.08 * (x - x0) + 0.001 * (x - x0) ** 3, 0.0, 1.0)
    assert bench._front(prof) == pytest.approx(x0, abs=1e-9)
