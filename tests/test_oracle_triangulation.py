"""Pins of the oracle's fisheye triangulation (next row f1): the series sine
and cosine against the library functions, the Kannala-Brandt unprojection
against rays projected in double precision, the two-ray triangulation against
known points, its rejections, and the generator's true points of a fisheye
frame.  The paper only says that stereo matches give depth (section II-B);
the unprojection, the midpoint of the common perpendicular and the
thresholds are readings, each a parameter."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes

P = dict(scenes.DEFAULT_PARAMS)


def kb_project64(cam, ray):
    """Kannala-Brandt projection of a direction, double precision."""
    x, y, z = (float(c) for c in ray)
    rho = math.hypot(x, y)
    if rho == 0.0:
        return cam.cx, cam.cy
    th = math.atan2(rho, z)
    k = [float(c) for c in cam.k]
    thd = th * (1 + k[0] * th ** 2 + k[1] * th ** 4 + k[2] * th ** 6 + k[3] * th ** 8)
    return cam.fx * thd * x / rho + cam.cx, cam.fy * thd * y / rho + cam.cy


def angle(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
    return math.acos(max(-1.0, min(1.0, c)))


def camera(fx=190.0, fy=205.0, k=(0.01, -0.008, 0.004, -0.002)):
    return scenes.KB8Camera(fx=fx, fy=fy, cx=256.0, cy=250.0, k=np.array(k, np.float32), width=512,
                            height=512, min_x=0.0, max_x=512.0, min_y=0.0, max_y=512.0)


def rig(b=0.1, deg=3.0, seed=0):
    rng = np.random.default_rng(seed)
    R = scenes.axis_angle(np.array([0.3, -0.8, 0.5]) / np.linalg.norm([0.3, -0.8, 0.5]), math.radians(deg))
    t = -R @ np.array([b, 0.0, 0.0])
    return R, t


@pytest.mark.parametrize("t", list(np.linspace(0.0, 2.0, 41)))
def test_series_sine_cosine(t):
    t = float(np.float32(t))
    assert abs(orc.sin_series(t) - math.sin(t)) <= 2.5e-7
    assert abs(orc.cos_series(t) - math.cos(t)) <= 2.5e-7


def test_unprojection_recovers_the_projected_ray():
    cam = camera()
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(400):
        th = rng.uniform(0.0, 1.45)
        ph = rng.uniform(-math.pi, math.pi)
        ray = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        u, v = kb_project64(cam, ray)
        ok, r = orc.unproject_kb8(cam, P["kb_iters"], float(np.float32(u)), float(np.float32(v)))
        assert ok
        worst = max(worst, angle(r, ray))
    # a float32 pixel position is good to ~3e-5 px, i.e. ~2e-7 rad at f = 190
    assert worst < 2e-6


def test_unprojection_rejects_pixels_past_the_lens_maximum():
    # theta * (1 + k1 t + ... + k4 t^4) peaks below theta_d for this pixel
    cam = camera(fx=190.0, fy=190.0, k=(0.0067, 0.0019, -0.0042, -0.0091))
    ok, _ = orc.unproject_kb8(cam, 10, 433.3, 103.8)
    assert not ok
    ok, _ = orc.unproject_kb8(cam, 10, 300.0, 200.0)
    assert ok


def test_unprojection_special_cases():
    cam = camera()
    ok, r = orc.unproject_kb8(cam, 10, cam.cx, cam.cy)
    assert ok and list(r) == [0.0, 0.0, 1.0]
    # strong distortion still converges in the fixed number of steps
    cam2 = camera(k=(0.05, 0.01, -0.005, 0.001))
    ray = np.array([math.sin(1.2), 0.0, math.cos(1.2)])
    u, v = kb_project64(cam2, ray)
    ok, r = orc.unproject_kb8(cam2, 10, u, v)
    assert ok and angle(r, ray) < 2e-6
    # with fx != fy the vertical offset uses fy
    ray = np.array([0.0, math.sin(0.7), math.cos(0.7)])
    u, v = kb_project64(cam, ray)
    ok, r = orc.unproject_kb8(cam, 10, u, v)
    assert ok and angle(r, ray) < 2e-6


def test_triangulation_recovers_known_points():
    R, t = rig()
    rng = np.random.default_rng(2)
    for _ in range(300):
        z = rng.uniform(0.3, 15.0)
        Pl = np.array([rng.uniform(-1, 1) * z, rng.uniform(-1, 1) * z, z])
        Pr = R @ Pl + t
        rl = (Pl / np.linalg.norm(Pl)).astype(np.float32)
        rr = (Pr / np.linalg.norm(Pr)).astype(np.float32)
        ok, X = orc.triangulate(rl, rr, R.astype(np.float32), t.astype(np.float32), P["min_depth"])
        assert ok
        # a float32 ray is good to ~1e-7 rad; depth error grows as z^2 / baseline
        tol = 2e-6 * np.linalg.norm(Pl) * (1.0 + np.linalg.norm(Pl) / 0.1)
        assert np.linalg.norm(X - Pl) <= tol, (Pl, X)


def test_triangulation_rejections():
    R, t = rig()
    Rf, tf = R.astype(np.float32), t.astype(np.float32)
    # parallel and nearly parallel rays
    d = np.array([0.1, 0.2, 1.0])
    d /= np.linalg.norm(d)
    assert not orc.triangulate(d, R @ d, Rf, tf, 1e-4)[0]
    # rays meeting 1e5 m away, in front of both cameras: 1e-6 rad apart
    Pl = np.array([0.0, 0.0, 1e5])
    Pr = R @ Pl + t
    assert not orc.triangulate(Pl / 1e5, Pr / np.linalg.norm(Pr), Rf, tf, 1e-4)[0]
    # a point behind both cameras: the rays meet at negative parameters
    Pl = np.array([0.2, -0.1, -3.0])
    Pr = R @ Pl + t
    assert not orc.triangulate(-Pl / np.linalg.norm(Pl), -Pr / np.linalg.norm(Pr), Rf, tf, 1e-4)[0]
    # depth at or below the threshold, rays in front
    for z, keep in ((5e-5, False), (2e-3, True)):
        Pl = np.array([-0.05, 0.0, z])
        Pr = R @ Pl + t
        ok, X = orc.triangulate(Pl / np.linalg.norm(Pl), Pr / np.linalg.norm(Pr), Rf, tf, 1e-4)
        assert ok == keep, (z, X)


def test_fisheye_frame_true_matches_give_true_points():
    fr = scenes.fisheye_frame(3)
    st = orc.stereo_frame(P, fr)
    true_r = fr.truth["true_r"]
    Pl = fr.truth["P_left"]
    # the generator's own double-precision unprojection has no solution for
    # pixels past the lens model's maximum; keep the points it placed exactly
    uv = scenes.kb8_project64(fr.rig.left, Pl)
    exact = np.hypot(uv[:, 0] - fr.left.x, uv[:, 1] - fr.left.y) < 1e-3
    good = np.nonzero((st["r_idx"] >= 0) & (st["r_idx"] == true_r) & exact)[0]
    assert len(good) > 200
    kept = 0
    for i in good:
        if Pl[i, 2] <= 1e-3:
            assert st["fdepth"][i] < 0 or st["fdepth"][i] > 1e-4
            continue
        kept += 1
        assert st["xyz"][i, 3] == 1.0
        assert st["fdepth"][i] == st["xyz"][i, 2]
        err = np.linalg.norm(st["xyz"][i, :3] - Pl[i])
        assert err <= 1e-3 * np.linalg.norm(Pl[i]) * (1 + np.linalg.norm(Pl[i]) / 0.1), (i, err)
    assert kept > 150
    # keypoints without an accepted match have no point
    none = st["r_idx"] < 0
    assert np.all(st["fdepth"][none] == -1.0) and np.all(st["xyz"][none] == 0.0)
