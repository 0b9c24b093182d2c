"""Pins of the oracle's search of the last frame's points (next row f2): the
motion rule, the projection, and the whole search against a brute force over
all keypoints written here from the stated predicates (numpy, float32 where
the method computes in float32); plus hand cases for the octave window, the
radius of the last octave, the absent ratio test and invalid octaves."""
import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes

P = dict(scenes.DEFAULT_PARAMS)
NL = P["nlevels"]


def scale_table():
    sc = [np.float32(1.0)]
    for _ in range(1, NL):
        sc.append(np.float32(sc[-1] * np.float32(P["scale_factor"])))
    return np.array(sc, np.float32)


def hamming(a, b):
    return int(np.unpackbits(np.bitwise_xor(a, b)).sum())


def brute_force(kps, u_right, taken, desc, level, proj, motion, bounds):
    """The f2 search, every keypoint of the grid (membership by the pinned a7
    cell rule) against every point in view."""
    sc = scale_table()
    M, N = len(level), kps.n
    in_grid = [orc.grid_cell(float(kps.x[k]), float(kps.y[k]), *bounds)[0] for k in range(N)]
    mp_kp = np.full(M, -1, np.int32)
    d1 = np.full(M, -1, np.int32)
    d2 = np.full(M, -1, np.int32)
    claims = {}
    for m in range(M):
        lv = int(level[m])
        if lv < 0:
            continue
        u, v, ur = np.float32(proj[m, 0]), np.float32(proj[m, 1]), np.float32(proj[m, 2])
        r = np.float32(np.float32(P["th_last"]) * sc[lv])
        lo, hi = {1: (lv, NL - 1), -1: (0, lv), 0: (lv - 1, lv + 1)}[motion]
        cands = []
        for k in range(N):
            if not in_grid[k]:
                continue
            o = int(kps.oct[k])
            if o < lo or o > hi:
                continue
            if not (abs(np.float32(kps.x[k] - u)) < r and abs(np.float32(kps.y[k] - v)) < r):
                continue
            if taken is not None and taken[k]:
                continue
            if u_right is not None and u_right[k] > 0 and abs(np.float32(ur - u_right[k])) > r:
                continue
            cands.append((hamming(desc[m], kps.desc[k]), k))
        if not cands:
            continue
        cands.sort()
        d1[m] = cands[0][0]
        d2[m] = cands[1][0] if len(cands) > 1 else 256
        if d1[m] <= P["th_search"]:
            k = cands[0][1]
            mp_kp[m] = k
            claims.setdefault(k, []).append((int(d1[m]), m))
    kp_mp = np.full(N, -1, np.int32)
    for k, c in claims.items():
        kp_mp[k] = min(c)[1]
    for m in range(M):
        if mp_kp[m] >= 0 and kp_mp[mp_kp[m]] != m:
            mp_kp[m] = -1
    return dict(mp_kp=mp_kp, mp_d1=d1, mp_d2=d2, kp_mp=kp_mp)


def test_motion_rule():
    fr = scenes.single_pinhole(2)
    b = fr.cam.b
    for mode, want in (("forward", 1), ("backward", -1), ("none", 0)):
        assert orc.motion(fr.pose, scenes.last_frame(fr, 1, mode).pose, b) == want
    # exactly one baseline along the axis is not "moved" (strict), a bit more is
    R = fr.pose.R.reshape(3, 3).astype(np.float64)
    O = fr.pose.O.astype(np.float64)
    for d, want in ((0.5 * b, 0), (-0.5 * b, 0), (2 * b, 1), (-2 * b, -1)):
        last = scenes.make_pose(R, O - d * R[2])
        assert orc.motion(fr.pose, last, b) == want, d


@pytest.mark.parametrize("mode", ["forward", "backward", "none"])
def test_pinhole_search_equals_brute_force(mode):
    fr = scenes.pinhole_frame(11, n_left=500, n_map=700)
    st = orc.stereo_frame(P, fr)
    last = scenes.last_frame(fr, 12, mode)
    out = orc.search_last_frame(P, fr, last, st["u_right"])
    motion = orc.motion(fr.pose, last.pose, fr.cam.b)
    c = fr.cam
    ref = brute_force(fr.left, st["u_right"], fr.taken_l, last.desc, out["level"], out["proj"], motion,
                      (c.min_x, c.max_x, c.min_y, c.max_y))
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k
    assert (out["mp_kp"] >= 0).sum() > 100


def test_fisheye_search_equals_brute_force():
    fr = scenes.fisheye_frame(13, n_left=600, n_map=900)
    last = scenes.last_frame(fr, 14, "forward")
    out = orc.search_last_frame(P, fr, last)
    motion = orc.motion(fr.pose, last.pose, fr.rig.b)
    assert motion == 1
    for s, kps, tk, c in (("l", fr.left, fr.taken_l, fr.rig.left), ("r", fr.right, fr.taken_r, fr.rig.right)):
        ref = brute_force(kps, None, tk, last.desc, out["level_" + s], out["proj_" + s], motion,
                          (c.min_x, c.max_x, c.min_y, c.max_y))
        for k in ref:
            assert np.array_equal(out[f"{k}_{s}"], ref[k]), (s, k)
    assert (out["mp_kp_l"] >= 0).sum() > 50 and (out["mp_kp_r"] >= 0).sum() > 20


def test_projection_and_view():
    """In view = in front and inside the image, whatever the distance and the
    normal; the projection equals the local-map search's where both apply;
    the level is the last octave; invalid octaves and skipped points stay out."""
    fr = scenes.pinhole_frame(15, n_left=300, n_map=800)
    last = scenes.last_frame(fr, 16, "none")
    out = orc.search_last_frame(P, fr, last, None)
    loc = orc.search_frame(P, fr, None)
    both = (out["level"] >= 0) & (loc["level"] >= 0)
    assert both.sum() > 300
    assert np.array_equal(out["proj"][both, :3].view(np.uint32), loc["proj"][both, :3].view(np.uint32))
    assert np.all(out["proj"][:, 3] == 0.0)
    R = fr.pose.R.reshape(3, 3).astype(np.float64)
    Pc = last.pos[:, :3].astype(np.float64) @ R.T + fr.pose.t.astype(np.float64)
    for m in range(last.n):
        valid_oct = 0 <= last.oct[m] < NL
        if last.skip[m] or not valid_oct or Pc[m, 2] <= 1e-6:
            assert out["level"][m] == -1 and out["mp_kp"][m] == -1
            continue
        u = fr.cam.fx * Pc[m, 0] / Pc[m, 2] + fr.cam.cx
        v = fr.cam.fy * Pc[m, 1] / Pc[m, 2] + fr.cam.cy
        inside = 0.01 < u < fr.cam.max_x - 0.01 and 0.01 < v < fr.cam.max_y - 0.01
        outside = u < -0.01 or u > fr.cam.max_x + 0.01 or v < -0.01 or v > fr.cam.max_y + 0.01
        if inside:
            assert out["level"][m] == last.oct[m]
            assert abs(out["proj"][m, 0] - u) < 1e-2 and abs(out["proj"][m, 1] - v) < 1e-2
        elif outside:
            assert out["level"][m] == -1


def _hand(level, ks, motion, desc_pts=None, taken=None):
    """One point at (100, 100) with octave `level` against keypoints ks =
    [(x, y, octave, distance)]."""
    rng = np.random.default_rng(0)
    pd = rng.integers(0, 256, (1, 32), dtype=np.uint8) if desc_pts is None else desc_pts
    x = np.array([k[0] for k in ks], np.float32)
    y = np.array([k[1] for k in ks], np.float32)
    o = np.array([k[2] for k in ks], np.int8)
    d = np.zeros((len(ks), 32), np.uint8)
    for i, k in enumerate(ks):
        bits = np.unpackbits(pd[0].copy())
        bits[:k[3]] ^= 1
        d[i] = np.packbits(bits)
    kps = scenes.Keypoints(x=x, y=y, oct=o, desc=d)
    proj = np.array([[100.0, 100.0, -1.0, 0.0]], np.float32)
    return orc.search_last_camera(P, (0.0, 752.0, 0.0, 480.0), kps, None, taken, pd,
                                  np.array([level], np.int8), proj, motion)


def test_octave_window_by_motion():
    ks = [(100.0, 100.0, 1, 40), (100.5, 100.0, 2, 30), (101.0, 100.0, 3, 20), (99.0, 100.0, 5, 10)]
    # forward: octaves >= 2 -> the octave-5 keypoint (d 10)
    assert _hand(2, ks, 1)["mp_kp"][0] == 3
    # backward: octaves <= 2 -> octave 2 (d 30)
    assert _hand(2, ks, -1)["mp_kp"][0] == 1
    # neither: octaves 1..3 -> octave 3 (d 20)
    assert _hand(2, ks, 0)["mp_kp"][0] == 2


def test_radius_of_the_last_octave_and_no_ratio():
    sc3 = scale_table()[3]
    r = float(np.float32(np.float32(P["th_last"]) * sc3))
    inside = [(100.0 + 0.99 * r, 100.0, 3, 12)]
    outside = [(100.0 + 1.01 * r, 100.0, 3, 12)]
    assert _hand(3, inside, 0)["mp_kp"][0] == 0
    assert _hand(3, outside, 0)["mp_kp"][0] == -1
    # two candidates at the same distance: the smaller index wins, no ratio test
    out = _hand(3, [(101.0, 100.0, 3, 50), (100.0, 101.0, 3, 50)], 0)
    assert out["mp_kp"][0] == 0 and out["mp_d1"][0] == 50 and out["mp_d2"][0] == 50
    # above the threshold nothing is accepted, but d1 is reported
    out = _hand(3, [(101.0, 100.0, 3, 101)], 0)
    assert out["mp_kp"][0] == -1 and out["mp_d1"][0] == 101 and out["mp_d2"][0] == 256
    # taken keypoints are skipped
    out = _hand(3, [(101.0, 100.0, 3, 5), (100.0, 101.0, 3, 9)], 0, taken=np.array([1, 0], np.uint8))
    assert out["mp_kp"][0] == 1
