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



def test_sampled_steps_are_the_middles_of_equal_strata():
    idx = bench.sampled_steps(200, 20)
    assert idx == [5 + 10 * j for j in range(20)]
    assert bench.sampled_steps(200, 500) == list(range(200))  # all steps when K >= the run
    for k in (1, 3, 7, 64, 199):
        s = bench.sampled_steps(200, k)
        assert len(s) == k and len(set(s)) == k and s == sorted(s)
        assert all(int(j * 200 / k) <= s[j] < int((j + 1) * 200 / k) + 1 for j in range(k))


def test_reference_evaluations_follow_the_timed_steps():
    assert len(bench.EVALS_PER_STEP_256) == 200
    idx = bench.sampled_steps(200, 20)
    assert bench.reference_evals(idx) == sum(bench.EVALS_PER_STEP_256[i] for i in idx) / 20


def test_oracle_step_model_sums_its_pieces():
    m = bench.OracleStepModel.__new__(bench.OracleStepModel)
    m.times = {"deposit": [2.0], "forward": [1.0], "source": [1.5], "evaluation": [10.0, 12.0], "update": [0.5],
               "phi_forces": [4.0], "interpolate": [1.0]}
    # 2 + 1 + 1.5 + E 11 + (E - 1) 0.5 + 4 + 3 x 1 at E = 3
    assert m.step_seconds(3.0) == 2.0 + 1.0 + 1.5 + 33.0 + 1.0 + 4.0 + 3.0
