"""CPU check of bench.py's clock record: the samples that nvidia-smi writes
during the timed region are reduced to the median SM clock under load, the
maximum SM clock and the set of active throttle reasons, which is what decides
whether a timed run stands (hw_slowdown, hw_thermal_slowdown and
sw_thermal_slowdown reject it; sw_power_cap is kept and noted).  nvidia-smi
is replaced by a file of sample lines in its CSV format (no GPU here)."""
from __future__ import annotations

import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    """Stands for the sampling process: already finished."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _stop_with(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _Done(), path
    rec = s.stop()
    assert not os.path.exists(path)  # the sample file is removed
    return rec


def _line(sm, smax, power, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active (bit mask), the four reasons
    return f"0, {sm}, {smax}, {power}, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clean_run_median_and_max():
    rec = _stop_with([_line(2070, 2070, 850.0), _line(2055, 2070, 900.5), _line(2070, 2070, 870.0)])
    assert rec["sm_mhz"] == 2070.0
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == []
    assert rec["samples"] == 3
    assert rec["power_w_max"] == 900.5


def test_idle_samples_do_not_pull_the_median_down():
    # samples at 0 MHz (before the kernels start) are left out of the median
    rec = _stop_with([_line(0, 2070, 90.0), _line(0, 2070, 90.0), _line(1980, 2070, 800.0),
                      _line(1995, 2070, 810.0), _line(2010, 2070, 805.0)])
    assert rec["sm_mhz"] == 1995.0
    assert rec["samples"] == 5


def test_throttle_reasons_are_reported():
    rec = _stop_with([_line(2070, 2070, 900.0, cap="Active"),
                      _line(1800, 2070, 1400.0, hw="Active"),
                      _line(1700, 2070, 1400.0, hwt="Active", swt="Active")])
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                              "sw_thermal_slowdown"]


def test_malformed_lines_are_skipped():
    rec = _stop_with(["", "0, [N/A], 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                      "0, 1500, 2070, [N/A], 0x0, Active, Not Active, Not Active, Not Active",
                      "garbage", _line(2040, 2070, 700.0)])
    assert rec["sm_mhz"] == 2040.0  # numbers count only from lines where all are readable
    assert rec["samples"] == 1
    assert rec["reasons"] == ["hw_slowdown"]  # a throttle reason counts wherever it is read


def test_no_sampler_says_so():
    rec = bench.ClockSampler(0).stop()  # never started
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
