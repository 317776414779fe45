"""Host logic of bench.py (no GPU): the clock record that decides whether a
run is kept (throttle reasons, clocks), the counter record that is used only
while it matches the evaluator's source, and the kernel-source hash."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_no_reason(bench):
    c = bench.ClockSampler(0)
    c.lines = [line(2070, 2070), line(1980, 2070), line(2070, 2070)]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == [] and s["samples"] == 3


def test_clock_summary_names_every_active_reason(bench):
    c = bench.ClockSampler(0)
    c.lines = [line(1500, 2070, hw="Active"), line(1600, 2070, cap="Active"),
               line(1700, 2070, hwt="Active", swt="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                                      "sw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines(bench):
    c = bench.ClockSampler(0)
    c.lines = ["", "garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
               line(2000, 2070)]
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2000.0


def test_clock_summary_without_samples_says_so(bench):
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unsampled"]


def test_counter_record_only_for_the_current_kernel_source(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"dram_bytes_per_launch": 123, "warp_instructions": 456, "kernel_source_sha": bench.kernel_source_sha()}
    (prof / "eval_kernel_traffic.json").write_text(json.dumps(rec))
    # the hash is taken over the real sources; only the record's folder moves
    real_sha = bench.kernel_source_sha()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: real_sha)
    assert bench.recorded_traffic() == 123
    rec["kernel_source_sha"] = "0" * 16
    (prof / "eval_kernel_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic() is None and bench.recorded_counters() == {}


def test_kernel_source_hash_covers_only_what_the_evaluator_compiles_from(bench):
    h = bench.kernel_source_sha()
    assert len(h) == 16 and int(h, 16) >= 0
    assert bench.kernel_source_sha() == h


def test_measured_peaks_fallback(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_nearest_rank_quantiles(bench):
    """p99 by the nearest-rank rule: the ceil(0.99 n)-th smallest value, so
    with 20 samples it is the largest and with 200 the second largest."""
    v = list(range(1, 21))
    assert bench.nearest_rank(v, 0.99) == 20 and bench.nearest_rank(v, 0.5) == 10
    w = list(range(200, 0, -1))
    assert bench.nearest_rank(w, 0.99) == 198 and bench.nearest_rank(w, 0.5) == 100
    assert bench.nearest_rank([7.0], 0.99) == 7.0
