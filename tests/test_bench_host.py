"""Host-side logic of the benchmark (no GPU): the clock sampler's window, the
traffic figure's source digest and the replica throughput of one rank."""
import datetime
import time

import pytest

import bench


def _line(ts, sm, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ts, ", ".join([stamp, "0", str(sm), "2070", "900.5", "0x0", *reasons])


def test_clock_sampler_keeps_the_samples_of_the_timed_window():
    c = bench.ClockSampler(0)
    t0 = time.time()
    c.lines = [_line(t0 - 1.0, 1000), _line(t0 + 0.01, 2070), _line(t0 + 0.03, 2050), _line(t0 + 1.0, 900)]
    c.mark(t0, t0 + 0.04)
    out = c.summary()
    assert out["samples"] == 2
    assert out["sm_mhz"] == pytest.approx(2060.0)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_clock_sampler_reports_throttle_reasons_inside_the_window():
    c = bench.ClockSampler(0)
    t0 = time.time()
    c.lines = [_line(t0 + 0.01, 1800, ("Not Active", "Not Active", "Active", "Active"))]
    c.mark(t0, t0 + 0.02)
    out = c.summary()
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_sampler_falls_back_to_the_sampled_span():
    c = bench.ClockSampler(0)
    t0 = time.time()
    c.lines = [_line(t0 - 5.0, 2070)]
    c.mark(t0, t0 + 0.01)
    out = c.summary()
    assert out["samples"] == 1 and "window" in out


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on():
    key = ("kset", "paper", 22)
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC[key] = {"bytes": 123, "digest": bench.kernel_digest()}
        assert bench.traffic_for(*key) == 123
        bench.TRAFFIC[key] = {"bytes": 123, "digest": "0" * 16}
        assert bench.traffic_for(*key) is None
        assert bench.traffic_for("tpl", "paper", 22) is None
    finally:
        bench.TRAFFIC.clear()
        bench.TRAFFIC.update(saved)


def test_single_rank_throughput_is_units_over_seconds():
    assert bench.replica_throughput(1000.0, 0.5) == pytest.approx(2000.0)
