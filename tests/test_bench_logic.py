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


def test_patch_sector_bytes_counts_distinct_sectors():
    """Two refined matches on level 0 whose left patches share their sectors
    and whose right strips are far apart: the byte count is 2 x 352, the
    sector count 11 rows x (2 shared left + 3 right) sectors."""
    import numpy as np
    from types import SimpleNamespace as NS

    class Pyr:
        def __init__(self, base, pitch):
            self.data = [base] + [0] * 15
            self.pitch = [pitch] + [0] * 15

    fr = NS(camera="pinhole", pyr_left=[None], pyr_right=[None],
            left=NS(x=np.array([100.0, 101.0], np.float32), y=np.array([50.0, 50.0], np.float32),
                    oct=np.array([0, 0], np.int8)),
            right=NS(x=np.array([60.0, 300.0], np.float32)))
    out = {"sad_shift": np.array([0, 1], np.int32), "best_r": np.array([0, 1], np.int32)}
    pb = NS(frames=[fr], outputs=lambda f: out,
            pyramid=lambda f, side: Pyr(1 << 20 if side == "L" else 1 << 24, 1024))
    b, s = bench.patch_sector_bytes(pb)
    assert b == 2 * bench.PATCH_BYTES
    # left rows: columns 95..105 and 96..106 lie in sector 2 (bytes 64..95) and
    # sector 3 (96..127): two sectors per row, shared by both patches
    # right rows: columns 50..70 (sectors 1, 2) and 290..310 (sector 9): 3 per row
    assert s == 32 * 11 * (2 + 3)
    # 128-byte lines: left rows (bytes 95..105 and 96..106) share line 0;
    # right rows 50..70 lie in line 0 of the right buffer, 290..310 in line 2
    b, s = bench.patch_sector_bytes(pb, 128)
    assert b == 2 * bench.PATCH_BYTES
    assert s == 128 * 11 * (1 + 2)
