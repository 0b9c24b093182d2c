"""Pins of the oracle's pose optimization (next row f4; the paper's tracking
refines the pose with the map points found in the frame, section II-D, and
FastTrack switches the step off, section IV-F).

What fixes the result independently of the oracle's code:
* the exponential map of a twist against scipy's matrix exponential of the
  4x4 se(3) matrix;
* the Jacobian against central differences of the projection under
  expm(d^) T (mono and stereo rows);
* exact observations of a known pose: the optimization returns that pose
  from a perturbed start, with every observation an inlier; with planted
  gross outliers it still returns the pose and flags exactly the outliers;
* without the Huber weights and outliers, one round of Gauss-Newton is the
  weighted least-squares solution scipy.optimize.least_squares finds;
* with the Huber weights, the result is a stationary point of the robust
  cost written out here (sum of chi2 below the threshold, 2 sqrt(th chi2) -
  th above it): its gradient vanishes;
* a rigid change of the world frame changes the result by the same change;
* fewer than three observations leave the pose as given.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes

scipy_linalg = pytest.importorskip("scipy.linalg")
scipy_optimize = pytest.importorskip("scipy.optimize")

P = dict(scenes.DEFAULT_PARAMS)


def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def twist(d):
    X = np.zeros((4, 4))
    X[:3, :3] = hat(d[:3])
    X[:3, 3] = d[3:]
    return X


def exp_pose(d, R, t):
    """expm(d^) (R, t) by scipy's matrix exponential."""
    E = scipy_linalg.expm(twist(np.asarray(d, np.float64)))
    return E[:3, :3] @ R, E[:3, :3] @ t + E[:3, 3]


def project(cam, R, t, Pw, stereo):
    Pc = R @ Pw + t
    u = cam.fx * Pc[0] / Pc[2] + cam.cx
    v = cam.fy * Pc[1] / Pc[2] + cam.cy
    return np.array([u, v, u - cam.bf / Pc[2]]) if stereo else np.array([u, v])


def synthetic(seed, n=200, stereo_frac=0.5, noise=0.0, outlier_frac=0.0):
    """A known pose, world points in front of it, their observations as
    float32 keypoints (octaves 0-3), u_right for a share of them."""
    rng = np.random.default_rng(seed)
    cam = scenes.pinhole_camera()
    R = scenes.random_rotation(rng, 20.0)
    O = rng.normal(0.0, 1.0, 3)
    t = -R @ O
    u = rng.uniform(20, cam.width - 20, n)
    v = rng.uniform(20, cam.height - 20, n)
    z = rng.uniform(1.0, 10.0, n)
    Pc = np.stack([(u - cam.cx) / cam.fx * z, (v - cam.cy) / cam.fy * z, z], axis=1)
    Pw = (Pc - t) @ R                                   # R^T (Pc - t)
    pos = np.concatenate([Pw, np.ones((n, 1))], axis=1).astype(np.float32)
    Pw32 = pos[:, :3].astype(np.float64)
    obs = np.array([project(cam, R, t, Pw32[i], True) for i in range(n)])
    obs[:, :2] += rng.normal(0.0, noise, (n, 2)) if noise else 0.0
    octs = rng.integers(0, 4, n).astype(np.int8)
    out = np.zeros(n, bool)
    if outlier_frac:
        out = rng.random(n) < outlier_frac
        ang = rng.uniform(0, 2 * np.pi, out.sum())
        obs[out, 0] += 40.0 * np.cos(ang)
        obs[out, 1] += 40.0 * np.sin(ang)
    stereo = rng.random(n) < stereo_frac
    ur = np.where(stereo, obs[:, 2], -1.0).astype(np.float32)
    kps = scenes.Keypoints(x=obs[:, 0].astype(np.float32), y=obs[:, 1].astype(np.float32), oct=octs,
                           desc=np.zeros((n, 32), np.uint8))
    return cam, R, t, O, pos, kps, ur, out


def perturbed(R, O, rng, deg=0.5, m=0.02):
    Re, Oe = scenes.perturb_pose(rng, R, O)
    return scenes.make_pose(Re, Oe)


def test_exp_map_equals_matrix_exponential():
    rng = np.random.default_rng(1)
    for theta in (1e-7, 1e-4, 0.005, 0.0099, 0.0101, 0.3, 1.5, 3.0):
        for _ in range(5):
            w = rng.normal(size=3)
            w *= theta / np.linalg.norm(w)
            d = np.concatenate([w, rng.normal(size=3)])
            Rd, V = orc.se3_exp(d)
            E = scipy_linalg.expm(twist(d))
            assert np.max(np.abs(Rd - E[:3, :3])) < 1e-12, theta
            assert np.max(np.abs(V @ d[3:] - E[:3, 3])) < 1e-12, theta


@pytest.mark.parametrize("stereo", [False, True])
def test_jacobian_equals_central_differences(stereo):
    cam, R, t, _, pos, kps, ur, _ = synthetic(2, n=20)
    h = 1e-6
    for i in range(20):
        Pw = pos[i, :3].astype(np.float64)
        obs = [float(kps.x[i]), float(kps.y[i]), float(ur[i]) if stereo else 0.0]
        ok, e, J = orc.pose_residual(cam, R, t, pos[i, :3], obs, stereo)
        assert ok
        rows = 3 if stereo else 2
        pred = np.array(obs[:rows]) - e[:rows]
        assert np.allclose(pred, project(cam, R, t, Pw, stereo), atol=1e-9)
        for c in range(6):
            d = np.zeros(6)
            d[c] = h
            Rp, tp = exp_pose(d, R, t)
            Rm, tm = exp_pose(-d, R, t)
            fd = (project(cam, Rp, tp, Pw, stereo) - project(cam, Rm, tm, Pw, stereo)) / (2 * h)
            assert np.allclose(J[:rows, c], fd, rtol=1e-5, atol=1e-4), (i, c, J[:rows, c], fd)
        if not stereo:
            assert np.all(J[2] == 0.0)


def run(cam, pose0, pos, kps, ur, params=None, mp_kp=None):
    p = dict(P)
    p.update(params or {})
    n = len(pos)
    mk = np.arange(n, dtype=np.int32) if mp_kp is None else mp_kp
    return orc.optimize_pose(p, cam, pose0, kps, ur, pos, mk)


def test_exact_observations_return_the_pose():
    cam, R, t, O, pos, kps, ur, _ = synthetic(3)
    rng = np.random.default_rng(3)
    for deg, m in ((0.5, 0.02), (3.0, 0.2)):
        Re = scenes.axis_angle(rng.normal(size=3) / 1.7, math.radians(deg)) @ R
        pose0 = scenes.make_pose(Re, O + rng.normal(size=3) / np.sqrt(3) * m)
        r = run(cam, pose0, pos, kps, ur)
        # observations are float32: the pose is exact to their rounding
        assert np.max(np.abs(r["R"] - R)) < 2e-6 and np.max(np.abs(r["t"] - t)) < 2e-5, (deg, m)
        assert np.all(r["inlier"] == 1) and r["n_inliers"] == len(pos)
        assert r["rounds"] == P["po_rounds"]


def test_planted_outliers_are_flagged_and_ignored():
    cam, R, t, O, pos, kps, ur, out = synthetic(4, n=300, outlier_frac=0.2)
    rng = np.random.default_rng(4)
    r = run(cam, perturbed(R, O, rng), pos, kps, ur)
    assert out.sum() > 40
    assert np.array_equal(r["inlier"] == 0, out)
    assert np.max(np.abs(r["R"] - R)) < 2e-6 and np.max(np.abs(r["t"] - t)) < 2e-5


def weighted_residuals(cam, R, t, pos, kps, ur):
    sc = scenes.level_scales32()
    res = []
    for i in range(len(pos)):
        stereo = ur[i] >= 0
        obs = np.array([kps.x[i], kps.y[i]] + ([ur[i]] if stereo else []), np.float64)
        e = obs - project(cam, R, t, pos[i, :3].astype(np.float64), stereo)
        res.append(e / float(sc[kps.oct[i]]))
    return res


def test_one_round_without_huber_is_the_least_squares_solution():
    cam, R, t, O, pos, kps, ur, _ = synthetic(5, noise=0.7)
    rng = np.random.default_rng(5)
    pose0 = perturbed(R, O, rng)
    R0, t0 = pose0.R.reshape(3, 3).astype(np.float64), pose0.t.astype(np.float64)
    r = run(cam, pose0, pos, kps, ur, dict(po_rounds=1, po_iters=20, po_huber=0))

    def f(d):
        Rd, td = exp_pose(d, R0, t0)
        return np.concatenate(weighted_residuals(cam, Rd, td, pos, kps, ur))

    sol = scipy_optimize.least_squares(f, np.zeros(6), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    Rs, ts = exp_pose(sol.x, R0, t0)
    assert np.max(np.abs(r["R"] - Rs)) < 1e-9 and np.max(np.abs(r["t"] - ts)) < 1e-8
    assert np.max(np.abs(r["R"] - R)) > 1e-6            # the noise moved it off the true pose


def test_huber_result_is_a_stationary_point_of_the_robust_cost():
    cam, R, t, O, pos, kps, ur, out = synthetic(6, noise=0.5, outlier_frac=0.1)
    rng = np.random.default_rng(6)
    r = run(cam, perturbed(R, O, rng), pos, kps, ur, dict(po_rounds=1, po_iters=30))
    th = np.where(ur >= 0, P["po_chi2_stereo"], P["po_chi2_mono"])

    def cost(d):
        Rd, td = exp_pose(d, r["R"], r["t"])
        c2 = np.array([float(e @ e) for e in weighted_residuals(cam, Rd, td, pos, kps, ur)])
        return float(np.sum(np.where(c2 <= th, c2, 2.0 * np.sqrt(th * c2) - th)))

    h = 1e-7
    grad = np.array([(cost(h * np.eye(6)[c]) - cost(-h * np.eye(6)[c])) / (2 * h) for c in range(6)])
    base = np.array([(cost(1e-3 * np.eye(6)[c]) - cost(0 * np.eye(6)[c])) / 1e-3 for c in range(6)])
    assert np.max(np.abs(grad)) < 1e-4 * max(1.0, np.max(np.abs(base))), (grad, base)
    assert out.sum() > 10


def test_change_of_world_frame():
    cam, R, t, O, pos, kps, ur, _ = synthetic(7, noise=0.5, outlier_frac=0.1)
    rng = np.random.default_rng(7)
    pose0 = perturbed(R, O, rng)
    r = run(cam, pose0, pos, kps, ur)
    # world' = G world: points P' = Rg P + tg, pose T' = T G^-1
    Rg = scenes.random_rotation(rng, 40.0)
    tg = rng.normal(size=3)
    pos2 = pos.copy()
    pos2[:, :3] = (pos[:, :3].astype(np.float64) @ Rg.T + tg).astype(np.float32)
    R0, t0 = pose0.R.reshape(3, 3).astype(np.float64), pose0.t.astype(np.float64)
    pose2 = scenes.Pose(R=(R0 @ Rg.T).astype(np.float32).reshape(9), t=(t0 - R0 @ Rg.T @ tg).astype(np.float32),
                        O=np.zeros(3, np.float32))
    r2 = run(cam, pose2, pos2, kps, ur)
    # the float32 inputs of the two problems differ by rounding only
    assert np.max(np.abs(r2["R"] - r["R"] @ Rg.T)) < 2e-5
    assert np.max(np.abs(r2["t"] - (r["t"] - r["R"] @ Rg.T @ tg))) < 2e-4
    assert np.array_equal(r2["inlier"], r["inlier"])


def test_degenerate_inputs():
    cam, R, t, O, pos, kps, ur, _ = synthetic(8, n=10)
    rng = np.random.default_rng(8)
    pose0 = perturbed(R, O, rng)
    # two matches: no round runs, the pose is returned as given
    mk = np.full(10, -1, np.int32)
    mk[:2] = [0, 1]
    r = run(cam, pose0, pos, kps, ur, mp_kp=mk)
    assert r["rounds"] == 0 and r["n_inliers"] == 2
    assert np.array_equal(r["R"], pose0.R.reshape(3, 3).astype(np.float64))
    assert np.array_equal(r["t"], pose0.t.astype(np.float64))
    assert np.array_equal(r["inlier"], np.where(mk >= 0, 1, -1).astype(np.int8))
    # a point behind the camera is an outlier; unmatched points stay -1
    pos_b = pos.copy()
    pos_b[0, :3] = (2 * O - pos[0, :3].astype(np.float64)).astype(np.float32)
    mk = np.arange(10, dtype=np.int32)
    mk[9] = -1
    r = run(cam, pose0, pos_b, kps, ur, mp_kp=mk)
    assert r["inlier"][0] == 0 and r["inlier"][9] == -1 and r["n_inliers"] == 8


def test_generated_frame_moves_toward_the_true_pose():
    fr = scenes.single_pinhole(0)
    st, se = orc.track_frame(P, fr)
    r = orc.optimize_pose(P, fr.cam, fr.pose, fr.left, st["u_right"], fr.map.pos, se["mp_kp"])
    Rt, tt = fr.pose_true.R.reshape(3, 3).astype(np.float64), fr.pose_true.t.astype(np.float64)
    e0 = np.max(np.abs(fr.pose.R.reshape(3, 3) - Rt)), np.max(np.abs(fr.pose.t - tt))
    e1 = np.max(np.abs(r["R"] - Rt)), np.max(np.abs(r["t"] - tt))
    assert e1[0] < e0[0] / 20 and e1[1] < e0[1] / 20
    assert r["n_inliers"] > 0.9 * (se["mp_kp"] >= 0).sum()


def test_gauss_newton_converges_quadratically():
    """Exact observations, a rotation error of 0.5 degrees: one Gauss-Newton
    step leaves an error of the order of its square (~1e-4), two steps
    leave float32 rounding only.  A step taken along the wrong direction
    (say, the update applied on the wrong side of the pose) does not."""
    cam, R, t, O, pos, kps, ur, _ = synthetic(9)
    rng = np.random.default_rng(9)
    Re = scenes.axis_angle(rng.normal(size=3) / 1.7, math.radians(0.5)) @ R
    pose0 = scenes.make_pose(Re, O)
    e0 = np.max(np.abs(Re - R))
    r1 = run(cam, pose0, pos, kps, ur, dict(po_rounds=1, po_iters=1))
    r2 = run(cam, pose0, pos, kps, ur, dict(po_rounds=1, po_iters=2))
    e1 = np.max(np.abs(r1["R"] - R))
    e2 = np.max(np.abs(r2["R"] - R))
    assert e0 > 5e-3 and e1 < 4 * e0 ** 2 and e2 < 2e-6, (e0, e1, e2)


def test_thresholds_by_observation_kind():
    """Exact observations plus two planted ones at the true pose: a stereo
    observation with chi2 = 7.0 (below the three-residual threshold 7.815,
    above the two-residual one 5.991) stays an inlier; a mono observation
    with chi2 = 6.5 is an outlier; chi2 = 5.0 mono stays in."""
    cam, R, t, O, pos, kps, ur, _ = synthetic(10, n=120)
    sc = scenes.level_scales32()
    x, y = kps.x.copy(), kps.y.copy()
    urp = ur.copy()
    st = np.nonzero(urp >= 0)[0][0]
    mo = np.nonzero(urp < 0)[0][:2]
    urp[st] += np.float32(math.sqrt(7.0) * float(sc[kps.oct[st]]))
    x[mo[0]] += np.float32(math.sqrt(6.5) * float(sc[kps.oct[mo[0]]]))
    y[mo[1]] += np.float32(math.sqrt(5.0) * float(sc[kps.oct[mo[1]]]))
    k2 = scenes.Keypoints(x=x, y=y, oct=kps.oct, desc=kps.desc)
    r = run(cam, scenes.make_pose(R, O), pos, k2, urp)
    assert r["inlier"][st] == 1 and abs(r["chi2"][st] - 7.0) < 0.2
    assert r["inlier"][mo[0]] == 0 and abs(r["chi2"][mo[0]] - 6.5) < 0.2
    assert r["inlier"][mo[1]] == 1 and abs(r["chi2"][mo[1]] - 5.0) < 0.5
