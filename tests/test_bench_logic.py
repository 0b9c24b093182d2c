"""CPU checks of bench.py's host-side reductions: the equal-p99 selection of
the served/plain sweep and the windowed clock summary (no GPU, no
nvidia-smi: the sampler's rows are fed by hand)."""
import bench


def point(value, p99, dropped=0, completed=1000, hz=256.0):
    return {"value": value, "p99_ms": p99, "p50_ms": p99 / 2, "dropped": dropped, "completed": completed,
            "offered_hz": hz}


def test_equal_p99_takes_the_fastest_point_within_the_bound():
    pts = [point(1.0, 0.4), point(3.0, 0.9), point(5.0, 1.5), point(9.0, 80.0)]
    r = bench.equal_p99(pts, 1.0)
    assert r["value"] == 3.0 and r["p99_ms"] == 0.9
    assert bench.equal_p99(pts, 33.0)["value"] == 5.0
    assert bench.equal_p99(pts, 0.1) is None


def test_equal_p99_never_counts_a_point_that_dropped_frames():
    pts = [point(2.0, 0.5), point(7.0, 0.6, dropped=50, completed=950)]
    assert bench.equal_p99(pts, 1.0)["value"] == 2.0
    # one drop in 2000 is within the 0.1 % allowance
    pts = [point(2.0, 0.5), point(7.0, 0.6, dropped=1, completed=1999)]
    assert bench.equal_p99(pts, 1.0)["value"] == 7.0


def test_clock_summary_reports_median_reasons_and_windows():
    c = bench.ClockSampler(0)
    row = "0, {sm}, 2070, 900, 0x0, Not Active, Not Active, {sw}, Not Active"
    c.lines = [(1.0, row.format(sm=2070, sw="Not Active")), (2.0, row.format(sm=1900, sw="Not Active")),
               (3.0, row.format(sm=2070, sw="Active")), (4.0, "garbage")]
    c.windows = {"a": [1.5, 3.5], "b": [5.0, 6.0]}
    s = c._summary(c.lines)
    assert s["samples"] == 3 and s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_thermal_slowdown"]
    inside = [r for r in c.lines if 1.5 <= r[0] <= 3.5]
    w = c._summary(inside)
    assert w["samples"] == 2 and w["sm_mhz"] == (1900 + 2070) / 2
