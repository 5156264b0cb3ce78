"""Host logic of bench.py that decides what a measurement reports: the clock summary
(median SM clock and the throttle reasons seen during the timed region) and the
recorded ncu traffic, reported only while the kernel's sources are those it was taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line", "0, [N/A], 2070, 0, 0x0, a, b, c, d"]
    s = _sampler(lines).summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    lines = ["0, 1500, 2070, 1000, 0x48, Active, Active, Not Active, Not Active"]
    assert _sampler(lines).summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = _sampler([]).summary()
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_recorded_traffic_only_for_the_captured_sources(monkeypatch):
    rec = dict(bench.NCU_TRAFFIC["relax"])
    good = bench.sources_sha256(rec["sources"])
    monkeypatch.setitem(bench.NCU_TRAFFIC, "relax", dict(rec, sha256=good))
    assert bench.recorded_traffic("relax") == rec["bytes"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, "relax", dict(rec, sha256="0" * 64))
    assert bench.recorded_traffic("relax") is None
    assert bench.recorded_traffic("no_such_kind") is None

