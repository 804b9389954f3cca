"""bench.py's clock record, from synthetic nvidia-smi samples (no GPU).

The JSON line carries the median SM clock under load, the maximum clock and
every throttle reason seen active during the timed region; a run that saw
hw_slowdown, hw_thermal_slowdown or sw_thermal_slowdown is rejected by the
reader of the line, so those must not be lost or invented.
"""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def summary_of(text):
    s = bench.ClockSampler(0)
    f = tempfile.NamedTemporaryFile("w", suffix=".csv", delete=False)
    f.write(text)
    f.close()
    s.f = f
    return s.summary()


NA = "Not Active"


def row(sm, mx, hw=NA, hwt=NA, swt=NA, cap=NA):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {hwt}, {swt}, {cap}\n"


def test_median_max_and_no_reasons():
    d = summary_of(row(2070, 2070) + row(1995, 2070) + row(2070, 2070))
    assert d == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_reasons_are_kept_and_named():
    d = summary_of(row(2070, 2070) + row(1800, 2070, cap="Active") + row(1500, 2070, hwt="Active"))
    assert d["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and d["sm_mhz"] == 1800.0


def test_malformed_lines_are_skipped_and_empty_is_unavailable():
    d = summary_of("garbage\n" + row("[N/A]", 2070) + row(2000, 2070))
    assert d["samples"] == 1 and d["sm_mhz"] == 2000.0
    assert summary_of("")["reasons"] == ["unavailable"]
