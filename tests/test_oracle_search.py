"""Pins of the CPU oracle's search-by-projection steps (a7-a10): hand cases on
the frustum and grid boundaries, double-precision geometry, the predicted
level against log(), the grid gather against a linear scan, and the conflict
rule on hand-built claims."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes

f32 = np.float32


def bitcount(a, b):
    return int(np.unpackbits(np.bitwise_xor(a, b)).sum())


def identity_pose(O=(0.0, 0.0, 0.0)):
    O = np.array(O, np.float32)
    return scenes.Pose(R=np.eye(3, dtype=np.float32).reshape(9), t=(-O).astype(np.float32), O=O)


# --------------------------------------------------------------------------
# a7: grid cell
# --------------------------------------------------------------------------
def test_grid_cell_rounding_and_bounds():
    # W = 64, H = 48: one pixel per cell, cell = round(coordinate)
    assert orc.grid_cell(0.0, 0.0, 0, 64, 0, 48) == (True, 0, 0)
    assert orc.grid_cell(10.5, 3.49, 0, 64, 0, 48) == (True, 11, 3)   # half away from zero
    assert orc.grid_cell(63.49, 47.49, 0, 64, 0, 48) == (True, 63, 47)
    assert orc.grid_cell(63.5, 1.0, 0, 64, 0, 48)[0] is False          # rounds to 64
    assert orc.grid_cell(-0.49, 1.0, 0, 64, 0, 48) == (True, 0, 1)
    assert orc.grid_cell(-0.5, 1.0, 0, 64, 0, 48)[0] is False          # rounds to -1
    # 752 x 480: cell width 11.75 px, height 10 px
    ok, cx, cy = orc.grid_cell(100.0, 100.0, 0, 752, 0, 480)
    assert ok and cx == round(100 / 11.75) and cy == 10


# --------------------------------------------------------------------------
# a8: projection, frustum, predicted level
# --------------------------------------------------------------------------
def cam64():
    return scenes.pinhole_camera(752, 480)


def test_projection_on_axis_is_principal_point(params):
    cam = cam64()
    ok, out, lv = orc.project_pinhole(params, cam, identity_pose(), [0, 0, 4.0], [0, 0, 1], 1.0, 5.0)
    assert ok and out[0] == f32(cam.cx) and out[1] == f32(cam.cy)
    assert out[2] == f32(f32(cam.cx) - f32(f32(cam.bf) * f32(0.25)))
    assert out[3] == 1.0


def test_projection_behind_or_at_camera_plane_is_out(params):
    cam = cam64()
    for z in (-1.0, -1e-6, 0.0):
        ok, _, _ = orc.project_pinhole(params, cam, identity_pose(), [0, 0, z], [0, 0, -1], 0.1, 5.0)
        assert not ok


def test_projection_image_bounds_inclusive(params):
    cam = scenes.PinholeCamera(fx=1.0, fy=1.0, cx=0.0, cy=0.0, b=0.1, bf=0.1, width=100, height=50,
                               min_x=0.0, max_x=100.0, min_y=0.0, max_y=50.0)
    P = [100.0, 50.0, 1.0]              # u = W, v = H exactly
    n = np.array(P) / np.linalg.norm(P)
    d = float(np.linalg.norm(P))
    assert orc.project_pinhole(params, cam, identity_pose(), P, n, d, d)[0]
    for Q in ([float(np.nextafter(f32(100.0), f32(200.0))), 50.0, 1.0],
              [100.0, float(np.nextafter(f32(50.0), f32(100.0))), 1.0],
              [float(np.nextafter(f32(0.0), f32(-1.0))), 10.0, 1.0]):
        assert not orc.project_pinhole(params, cam, identity_pose(), Q, n, d, d)[0]


def test_distance_window_boundaries(params):
    cam = cam64()
    P = [0.0, 0.0, 2.0]                 # dist = 2 exactly from O = 0
    n = [0.0, 0.0, 1.0]
    # dist == 0.8 * dmin exactly: in; dmin one ulp larger: out
    dmin = f32(2.5)                     # 0.8f * 2.5f == 2.0f
    assert f32(0.8) * dmin == f32(2.0)
    assert orc.project_pinhole(params, cam, identity_pose(), P, n, dmin, 3.0)[0]
    assert not orc.project_pinhole(params, cam, identity_pose(), P, n,
                                   float(np.nextafter(dmin, f32(9))), 3.0)[0]
    # dist > 1.2 * dmax: out
    assert not orc.project_pinhole(params, cam, identity_pose(), P, n, 1.0, 1.6)[0]
    assert orc.project_pinhole(params, cam, identity_pose(), P, n, 1.0, 1.7)[0]


def test_viewing_cosine_boundary(params):
    cam = cam64()
    P = [0.0, 0.0, 2.0]
    ok, out, _ = orc.project_pinhole(params, cam, identity_pose(), P, [0.866, 0.0, 0.5], 1.0, 2.0)
    assert ok and out[3] == 0.5
    lo = float(np.nextafter(f32(0.5), f32(0)))
    assert not orc.project_pinhole(params, cam, identity_pose(), P, [0.866, 0.0, lo], 1.0, 2.0)[0]


def test_projection_matches_double_precision(params):
    cam = cam64()
    rng = np.random.default_rng(7)
    for _ in range(300):
        R = scenes.random_rotation(rng, 30.0)
        O = rng.normal(0, 1, 3)
        pose = scenes.make_pose(R, O)
        Pc = np.array([rng.uniform(-3, 3), rng.uniform(-2, 2), rng.uniform(2, 9)])
        Pw = R.T @ (Pc - (-R @ O))
        n = (Pw - O) / np.linalg.norm(Pw - O)
        d = float(np.linalg.norm(Pw - O))
        ok, out, lv = orc.project_pinhole(params, cam, pose, Pw, n, d / 2, d)
        Rf, tf = pose.R.reshape(3, 3).astype(np.float64), pose.t.astype(np.float64)
        pc = Rf @ Pw.astype(np.float32).astype(np.float64) + tf
        u = cam.fx * pc[0] / pc[2] + cam.cx
        v = cam.fy * pc[1] / pc[2] + cam.cy
        inside = 0 <= u <= 752 and 0 <= v <= 480
        if abs(u) < 1e-3 or abs(u - 752) < 1e-3 or abs(v) < 1e-3 or abs(v - 480) < 1e-3:
            continue
        assert ok == inside
        if ok:
            assert abs(out[0] - u) < 2e-3 and abs(out[1] - v) < 2e-3
            assert abs(out[2] - (u - cam.bf / pc[2])) < 2e-3
            assert abs(out[3] - 1.0) < 1e-5


def test_predicted_level_is_ceil_log_ratio(params):
    cam = cam64()
    rng = np.random.default_rng(8)
    checked = 0
    for ratio in rng.uniform(0.3, 6.0, 2000):
        x = math.log(ratio) / math.log(1.2)
        if abs(x - round(x)) < 1e-4:
            continue
        expect = min(max(math.ceil(x), 0), 7)
        dist = 2.0
        dmax = float(f32(ratio * dist))
        if dist > 1.2 * dmax or dist < 0.8 * (dmax / 3.6):
            continue
        ok, _, lv = orc.project_pinhole(params, cam, identity_pose(), [0, 0, dist], [0, 0, 1],
                                        dmax / 3.6, dmax)
        assert ok and lv == expect, (ratio, lv, expect)
        checked += 1
    assert checked > 1000


def test_kb8_closed_forms(params):
    cam = scenes.KB8Camera(fx=190.0, fy=190.0, cx=256.0, cy=256.0, k=np.zeros(4, np.float32),
                           width=512, height=512, min_x=0.0, max_x=512.0, min_y=0.0, max_y=512.0)
    R, t, O = np.eye(3).reshape(9), np.zeros(3), np.zeros(3)
    ok, out, _ = orc.project_kb8(params, cam, R, t, O, [0, 0, 3.0], [0, 0, 1], 1.0, 3.0)
    assert ok and out[0] == 256.0 and out[1] == 256.0
    # equidistant model: a ray 45 degrees off axis lands fx*pi/4 from the centre
    ok, out, _ = orc.project_kb8(params, cam, R, t, O, [2.0, 0, 2.0], [0.7071, 0, 0.7071], 1.0, 3.0)
    assert ok and abs(out[0] - (256 + 190 * math.pi / 4)) < 1e-3 and out[1] == 256.0
    # a point in the image plane (90 degrees) is still projected: radius fx*pi/2
    ok, out, _ = orc.project_kb8(params, cam, R, t, O, [0, 1.0, 1e-30], [0, 1, 0], 0.5, 1.0)
    assert not ok or abs(out[1] - (256 + 190 * math.pi / 2)) < 1e-3


def test_kb8_matches_double_precision(params):
    rng = np.random.default_rng(9)
    rig = scenes.fisheye_rig(3)
    cam = rig.left
    for _ in range(300):
        P = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.3, 5)])
        n = P / np.linalg.norm(P)
        d = float(np.linalg.norm(P))
        ok, out, _ = orc.project_kb8(params, cam, np.eye(3).reshape(9), np.zeros(3), np.zeros(3),
                                     P, n, d / 2, d)
        uv = scenes.kb8_project64(cam, P.astype(np.float32).astype(np.float64)[None, :])[0]
        inside = 0 <= uv[0] <= 512 and 0 <= uv[1] <= 512
        if min(abs(uv[0]), abs(uv[0] - 512), abs(uv[1]), abs(uv[1] - 512)) < 1e-2:
            continue
        assert ok == inside
        if ok:
            assert np.max(np.abs(out[:2] - uv)) < 5e-3


# --------------------------------------------------------------------------
# a9: grid gather equals a linear scan over every keypoint
# --------------------------------------------------------------------------
def linear_scan_search(params, bounds, kps, u_right, taken, mp_desc, level, proj):
    sc = 1.2 ** np.arange(8)
    min_x, max_x, min_y, max_y = bounds
    M = len(level)
    d1 = np.full(M, -1)
    d2 = np.full(M, -1)
    pick = np.full(M, -1)
    for m in range(M):
        lv = int(level[m])
        if lv < 0:
            continue
        u, v, ur, vc = (float(a) for a in proj[m])
        r = float(f32(f32(f32(2.5 if vc > f32(0.998) else 4.0) * f32(params["search_th"]))
                      * scenes.level_scales32()[lv]))
        c = []
        for k in range(kps.n):
            ok, _, _ = orc.grid_cell(float(kps.x[k]), float(kps.y[k]), *bounds)
            if not ok:
                continue
            if not (lv - 1 <= kps.oct[k] <= lv):
                continue
            if not (abs(float(f32(kps.x[k] - f32(u)))) < r and abs(float(f32(kps.y[k] - f32(v)))) < r):
                continue
            if taken is not None and taken[k]:
                continue
            if u_right is not None and u_right[k] > 0 and abs(float(f32(f32(ur) - u_right[k]))) > r:
                continue
            c.append((bitcount(mp_desc[m], kps.desc[k]), k))
        c.sort()
        if not c:
            continue
        d1[m] = c[0][0]
        d2[m] = c[1][0] if len(c) > 1 else 256
        o1 = kps.oct[c[0][1]]
        o2 = kps.oct[c[1][1]] if len(c) > 1 else -1
        if d1[m] <= params["th_search"] and not (o1 == o2 and f32(d1[m]) > f32(0.8) * f32(d2[m])):
            pick[m] = c[0][1]
    return d1, d2, pick


def resolve(pick, d1, nk):
    owner = {}
    for m in range(len(pick)):
        k = pick[m]
        if k >= 0 and (k not in owner or (d1[m], m) < owner[k]):
            owner[k] = (int(d1[m]), m)
    mp_kp = np.array([k if k >= 0 and owner[k][1] == m else -1 for m, k in enumerate(pick)])
    kp_mp = np.array([owner[k][1] if k in owner else -1 for k in range(nk)])
    return mp_kp, kp_mp


@pytest.mark.parametrize("seed", range(3))
def test_search_grid_equals_linear_scan(params, seed):
    f = scenes.pinhole_frame(seed, W=300, H=200, n_left=400, n_map=500)
    st = orc.stereo_frame(params, f)
    out = orc.search_frame(params, f, st)
    bounds = (f.cam.min_x, f.cam.max_x, f.cam.min_y, f.cam.max_y)
    d1, d2, pick = linear_scan_search(params, bounds, f.left, st["u_right"], f.taken_l, f.map.desc,
                                      out["level"], out["proj"])
    assert np.array_equal(out["mp_d1"], d1)
    assert np.array_equal(out["mp_d2"], np.where(d1 < 0, -1, d2))
    mp_kp, kp_mp = resolve(pick, d1, f.left.n)
    assert np.array_equal(out["mp_kp"], mp_kp)
    assert np.array_equal(out["kp_mp"], kp_mp)
    assert (out["mp_kp"] >= 0).sum() > 20


def test_search_wider_radius_th2(params):
    p = dict(params, search_th=2.0)
    f = scenes.pinhole_frame(11, W=300, H=200, n_left=400, n_map=400)
    out = orc.search_frame(p, f, None)
    bounds = (f.cam.min_x, f.cam.max_x, f.cam.min_y, f.cam.max_y)
    d1, _, pick = linear_scan_search(p, bounds, f.left, None, f.taken_l, f.map.desc,
                                     out["level"], out["proj"])
    assert np.array_equal(out["mp_d1"], d1)
    assert np.array_equal(out["mp_kp"], resolve(pick, d1, f.left.n)[0])


# --------------------------------------------------------------------------
# a9 ratio rule and a10 conflict rule on hand-built claims
# --------------------------------------------------------------------------
def _hand_frame(descs_kp, descs_mp, octs, kp_xy):
    k = scenes.Keypoints(x=np.array([p[0] for p in kp_xy], np.float32),
                         y=np.array([p[1] for p in kp_xy], np.float32),
                         oct=np.array(octs, np.int8), desc=np.array(descs_kp, np.uint8))
    return k, np.array(descs_mp, np.uint8)


def test_ratio_and_conflict_rules(params):
    rng = np.random.default_rng(12)
    base = rng.integers(0, 256, (4, 32), dtype=np.uint8)

    def with_dist(a, d):
        b = np.unpackbits(a.copy())
        b[:d] ^= 1
        return np.packbits(b)

    bounds = (0.0, 640.0, 0.0, 480.0)
    # map points 0, 1, 2 all project onto (100, 100) at level 0
    proj = np.array([[100, 100, -1, 0.9]] * 3 + [[300, 300, -1, 0.9]] * 2, np.float32)
    level = np.array([0, 0, 0, 0, 0], np.int8)
    kps, mp = _hand_frame(
        descs_kp=[base[0], with_dist(base[1], 60), base[2], base[3]],
        descs_mp=[with_dist(base[0], 30), with_dist(base[0], 20), with_dist(base[0], 20),
                  with_dist(base[2], 50), with_dist(base[2], 50)],
        octs=[0, 0, 0, 0],
        kp_xy=[(100.5, 100.0), (101.0, 101.0), (300.0, 300.5), (301.0, 300.0)])
    # kp 3 is a near-duplicate of kp 2 in descriptor space for map points 3, 4
    kps.desc[3] = with_dist(base[2], 3)
    out = orc.search_camera(params, bounds, kps, None, None, mp, level, proj)
    # map points 0-2 claim kp 0 with d = 30, 20, 20: the smallest (d, m) = (20, 1) wins
    assert list(out["mp_d1"][:3]) == [30, 20, 20]
    assert list(out["mp_kp"][:3]) == [-1, 0, -1]
    assert out["kp_mp"][0] == 1
    # map points 3, 4: best kp 2 (d 50) vs second kp 3 (d 50 +- 3); same octave
    # and d1 > 0.8 d2, so the ratio test rejects both
    assert list(out["mp_kp"][3:]) == [-1, -1]
    assert out["kp_mp"][2] == -1 and out["kp_mp"][3] == -1
    # different octaves: the ratio test does not apply (default reading) ...
    kps.oct[3] = 1
    level[3:] = 1
    out = orc.search_camera(params, bounds, kps, None, None, mp, level, proj)
    assert out["mp_kp"][3] in (2, 3) and out["mp_kp"][4] == -1
    # ... unless ratio_any_octave is set
    out = orc.search_camera(dict(params, ratio_any_octave=1), bounds, kps, None, None, mp, level, proj)
    assert list(out["mp_kp"][3:]) == [-1, -1]


def test_taken_and_stereo_consistency_filters(params):
    bounds = (0.0, 640.0, 0.0, 480.0)
    d = np.random.default_rng(13).integers(0, 256, (1, 32), dtype=np.uint8)
    kps = scenes.Keypoints(x=np.array([100.0], np.float32), y=np.array([100.0], np.float32),
                           oct=np.array([0], np.int8), desc=d.copy())
    proj = np.array([[100.0, 100.0, 90.0, 0.9]], np.float32)
    level = np.array([0], np.int8)
    assert orc.search_camera(params, bounds, kps, None, None, d, level, proj)["mp_kp"][0] == 0
    assert orc.search_camera(params, bounds, kps, None, np.array([1], np.uint8), d, level,
                             proj)["mp_kp"][0] == -1
    # stereo check: |uR - u_right| must be <= radius (4 px at level 0, cos 0.9)
    for ur, ok in ((94.0, True), (86.0, True), (85.9, False), (-1.0, True), (0.0, True)):
        got = orc.search_camera(params, bounds, kps, np.array([ur], np.float32), None, d, level, proj)
        assert (got["mp_kp"][0] == 0) == ok, ur


def test_search_generated_scene_hits_ground_truth(params):
    f = scenes.single_pinhole(0)
    st, out = orc.track_frame(params, f)
    assoc = f.truth["map_kp"]
    hit = out["mp_kp"][:len(assoc)]
    matched = hit >= 0
    assert matched.sum() > 200
    assert np.mean(hit[matched] == assoc[matched]) > 0.95
