"""Pins of the oracle's right fisheye camera in the search by projection
(a8 for the right camera; paper §II-D, §IV-E run the search for both cameras
of a fisheye rig).

The right camera's pose is T_rw = T_rl T_lw and its centre O_right is the
caller's.  These tests hold the oracle's right-camera outputs against what
the geometry fixes, computed here in double precision from the rig's
definition (a point in the left camera, P_l = R_lw P + t_lw, is
P_r = R_rl P_l + t_rl in the right camera; distance and viewing angle are
measured from the right centre), on a rig whose relative rotation is far
from the identity (15 degrees), so that a transposed R_rl, a dropped t_rl or
the left centre used for the right camera all move the result:

* the right projection (u, v), the viewing cosine and the predicted level of
  every map point in view, in the local-map search;
* the right projection of the last frame's points (f2, same composition);
* on a generated frame, right-camera map points land on the right keypoints
  the generator planted for them.
"""
import math

import numpy as np

import oracle as orc
from paper_2509_10757_gb300 import scenes

P = dict(scenes.DEFAULT_PARAMS)
NL = P["nlevels"]


def rotated_rig(seed: int, deg: float = 15.0) -> scenes.FisheyeRig:
    """A fisheye rig with a 15-degree relative rotation (right <- left) about
    a tilted axis, baseline 0.10 m along the left camera's x."""
    base = scenes.fisheye_rig(seed)
    axis = np.array([0.25, 1.0, 0.15])
    R_rl = scenes.axis_angle(axis / np.linalg.norm(axis), math.radians(deg))
    t_rl = -R_rl @ np.array([base.b, 0.0, 0.0])
    return scenes.FisheyeRig(left=base.left, right=base.right, R_rl=R_rl.astype(np.float32).reshape(9),
                             t_rl=t_rl.astype(np.float32), b=base.b, lap_l0=base.lap_l0, lap_l1=base.lap_l1,
                             lap_r0=base.lap_r0, lap_r1=base.lap_r1)


def right_geometry64(rig, pose, O_right, pos, nrm):
    """Double-precision right-camera geometry of map points: camera-frame
    point, pixel, distance to the right centre and viewing cosine."""
    Rlw = pose.R.reshape(3, 3).astype(np.float64)
    tlw = pose.t.astype(np.float64)
    Rrl = rig.R_rl.reshape(3, 3).astype(np.float64)
    trl = rig.t_rl.astype(np.float64)
    Pw = pos[:, :3].astype(np.float64)
    Pr = (Pw @ Rlw.T + tlw) @ Rrl.T + trl
    uv = scenes.kb8_project64(rig.right, Pr)
    PO = Pw - O_right.astype(np.float64)
    dist = np.linalg.norm(PO, axis=1)
    vc = np.sum(PO * nrm[:, :3].astype(np.float64), axis=1) / dist
    return Pr, uv, dist, vc


def away_from_boundaries(cam, Pr, uv, dist, vc, dmin, dmax, ratio):
    """Points whose in-view decision and level no rounding can flip."""
    W, H = cam.max_x, cam.max_y
    e = 0.05
    ok = Pr[:, 2] > 1e-3
    ok &= (np.abs(uv[:, 0]) > e) & (np.abs(uv[:, 0] - W) > e) & (np.abs(uv[:, 1]) > e) & (np.abs(uv[:, 1] - H) > e)
    ok &= (np.abs(dist - 0.8 * dmin) > 1e-4 * dist) & (np.abs(dist - 1.2 * dmax) > 1e-4 * dist)
    ok &= np.abs(vc - 0.5) > 1e-4
    lg = np.log(np.maximum(ratio, 1e-30)) / math.log(1.2)
    ok &= (np.abs(lg - np.rint(lg)) > 1e-3) | (ratio <= 1.0 - 1e-4)
    return ok


def expected_level(ratio):
    lv = np.zeros(len(ratio), np.int64)
    for i, r in enumerate(ratio):
        l = 0
        while l < NL - 1 and 1.2 ** l < r:
            l += 1
        lv[i] = l
    return lv


def test_right_camera_projection_level_and_view_cosine():
    rig = rotated_rig(5)
    fr = scenes.fisheye_frame(31, n_left=400, n_map=3000, rig=rig)
    out = orc.search_frame(P, fr, None)
    m = fr.map
    Pr, uv, dist, vc = right_geometry64(rig, fr.pose, fr.O_right, m.pos, m.nrm)
    dmin = m.pos[:, 3].astype(np.float64)
    dmax = m.nrm[:, 3].astype(np.float64)
    ratio = dmax / dist
    inside = ((Pr[:, 2] > 0) & (uv[:, 0] >= 0) & (uv[:, 0] <= rig.right.max_x) & (uv[:, 1] >= 0)
              & (uv[:, 1] <= rig.right.max_y))
    view = inside & (dist >= 0.8 * dmin) & (dist <= 1.2 * dmax) & (vc >= 0.5) & (m.skip == 0)
    sure = away_from_boundaries(rig.right, Pr, uv, dist, vc, dmin, dmax, ratio)
    got = out["level_r"] >= 0
    assert np.array_equal(got[sure], view[sure])
    both = sure & view
    assert both.sum() > 300, "too few right-camera points in view to pin anything"
    pr = out["proj_r"]
    assert np.max(np.abs(pr[both, 0] - uv[both, 0])) < 5e-3
    assert np.max(np.abs(pr[both, 1] - uv[both, 1])) < 5e-3
    assert np.all(pr[both, 2] == -1.0)
    # the viewing cosine is measured from the right camera's centre
    assert np.max(np.abs(pr[both, 3] - vc[both])) < 2e-5
    assert np.array_equal(out["level_r"][both].astype(np.int64), expected_level(ratio[both]))
    # the right centre is not the left one: the two cosines differ on this rig
    PO_l = m.pos[:, :3].astype(np.float64) - fr.pose.O.astype(np.float64)
    vc_l = np.sum(PO_l * m.nrm[:, :3], axis=1) / np.linalg.norm(PO_l, axis=1)
    assert np.max(np.abs(vc_l[both] - vc[both])) > 1e-3


def test_right_camera_projection_of_last_frame_points():
    rig = rotated_rig(6)
    fr = scenes.fisheye_frame(32, n_left=400, n_map=3000, rig=rig)
    last = scenes.last_frame(fr, 33, "none")
    out = orc.search_last_frame(P, fr, last)
    Pr, uv, _, _ = right_geometry64(rig, fr.pose, fr.O_right, last.pos, np.zeros_like(last.pos) + 1.0)
    valid = (last.oct >= 0) & (last.oct < NL) & (last.skip == 0)
    inside = ((Pr[:, 2] > 0) & (uv[:, 0] >= 0) & (uv[:, 0] <= rig.right.max_x) & (uv[:, 1] >= 0)
              & (uv[:, 1] <= rig.right.max_y)) & valid
    e = 0.05
    sure = (Pr[:, 2] > 1e-3) & (np.abs(uv[:, 0]) > e) & (np.abs(uv[:, 0] - rig.right.max_x) > e) \
        & (np.abs(uv[:, 1]) > e) & (np.abs(uv[:, 1] - rig.right.max_y) > e)
    got = out["level_r"] >= 0
    assert np.array_equal(got[sure], inside[sure])
    both = sure & inside
    assert both.sum() > 300
    pr = out["proj_r"]
    assert np.max(np.abs(pr[both, :2] - uv[both])) < 5e-3
    assert np.array_equal(out["level_r"][both], last.oct[both])


def test_right_camera_map_points_hit_their_planted_right_keypoints():
    """Map points placed behind left keypoints that have a right partner are
    found by the right camera's search at that partner."""
    rig = rotated_rig(7)
    fr = scenes.fisheye_frame(34, n_left=1500, n_map=6000, rig=rig, taken_frac=0.0)
    out = orc.search_frame(P, fr, None)
    assoc = fr.truth["map_kp"]
    true_r = fr.truth["true_r"]
    partner = true_r[assoc]
    has = partner >= 0
    hit = out["mp_kp_r"][: len(assoc)]
    found = has & (hit >= 0)
    assert found.sum() > 200, found.sum()
    assert np.mean(hit[found] == partner[found]) > 0.95
    # and the left camera likewise finds the keypoint itself
    hit_l = out["mp_kp_l"][: len(assoc)]
    fl = hit_l >= 0
    assert np.mean(hit_l[fl] == assoc[fl]) > 0.95
