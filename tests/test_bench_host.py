"""Host-side pieces of bench.py that decide whether a bench line is valid:
the clock sampler's summary of nvidia-smi rows (median SM clock, maximum,
throttle reasons seen), the layout cycle of the timed steps, and the FP64
peak from unit counts."""
import pytest

import bench


def _summary(rows):
    s = bench.ClockSampler(0)
    s.rows = rows
    return s.stop()          # no process was started: only the rows are summarised


def test_clock_summary_median_max_and_no_reasons():
    rows = [["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["2055", "2070", "950.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["1980", "2070", "990.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    c = _summary(rows)
    assert c["sm_mhz"] == 2055 and c["sm_max_mhz"] == 2070 and c["reasons"] == [] and c["samples"] == 3


def test_clock_summary_reports_each_throttle_reason_seen():
    rows = [["1800", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["1500", "2070", "1400", "0x8", "Active", "Not Active", "Active", "Not Active"],
            ["garbage"], []]
    c = _summary(rows)
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert c["samples"] == 2 and c["sm_mhz"] == 1650


def test_clock_summary_without_samples():
    c = _summary([])
    assert c["sm_mhz"] is None and c["sm_max_mhz"] is None and c["samples"] == 0


def test_timed_steps_cycle_every_layout_and_both_parities():
    n = 16384
    seen = {bench.step_layout(s, n) for s in range(8)}
    assert {(t, u) for t, u, _ in seen} == {(t, u) for t in "NT" for u in "LU"}
    assert {m for _, _, m in seen} == {n, n - 1}
    assert len(seen) == 8


def test_fp64_peak_from_unit_counts():
    assert bench.fp64_peak_tflops(2070.0) == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert bench.fp64_peak_tflops(None) == bench.fp64_peak_tflops(2070.0)
