"""The mirror invariant of stereo matching (a2-a4, a6), a pin of the oracle.

Mirror both images left to right, swap the left and right cameras, and map
every keypoint x -> W-1-x.  A left keypoint at x_l with its partner at x_r
becomes a right keypoint at W-1-x_l, its partner a left keypoint at W-1-x_r,
and the disparity x_l - x_r is unchanged.  Searching the mirrored pair is a
second, independent run of the method on the same geometry, so:

* Hamming stage (pinhole a2 and fisheye a6): on inputs where every distance
  that can be accepted is the unique minimum of its row and of its column
  (tie-free), the accepted pairs of the mirrored problem are the original
  pairs, swapped, with the same distances.
* SAD stage (a3), on a zero-noise scene whose right image is the left one
  shifted by a whole number of pixels: the best shift k* is the same in both
  runs, so the integer disparity x_l - (x_r + k*) is unchanged; where the
  right keypoint sits exactly on the true match, the mirrored SAD vector is
  the original one reversed, element for element.
* Parabola (a4) on those pairs: the sub-pixel offset changes sign exactly
  (the numerator S- - S+ swaps, the denominator does not change), so the two
  refined disparities lie symmetrically about the integer one.

The keypoints of the SAD part sit on octave 0, where level and image
coordinates coincide (the mirror of a coarser level's pixel grid is not that
grid).
"""
import numpy as np

import oracle as orc
from paper_2509_10757_gb300 import scenes

P = dict(scenes.DEFAULT_PARAMS)
POPC = np.array([bin(i).count("1") for i in range(256)], np.int64)


def hamming_matrix(a, b):
    return POPC[np.bitwise_xor(a[:, None, :], b[None, :, :])].sum(axis=2)


def mirrored(k: scenes.Keypoints, W: int) -> scenes.Keypoints:
    return scenes.Keypoints(x=(np.float32(W - 1) - k.x).astype(np.float32), y=k.y.copy(), oct=k.oct.copy(),
                            desc=k.desc.copy())


def accepted_pairs(best, dist):
    return {(i, int(j), int(d)) for i, (j, d) in enumerate(zip(best, dist)) if j >= 0}


def test_pinhole_hamming_pairs_are_mirror_consistent():
    fr = scenes.pinhole_frame(41, n_left=500, n_map=10)
    W = fr.cam.width
    D = hamming_matrix(fr.left.desc, fr.right.desc)
    # tie-free: any distance that can pass the threshold is alone in its row and column
    low = D < P["th_stereo"]
    assert low.sum(axis=1).max() <= 1 and low.sum(axis=0).max() <= 1
    best, dist = orc.stereo_best(P, fr.cam, fr.left, fr.right)
    mbest, mdist = orc.stereo_best(P, fr.cam, mirrored(fr.right, W), mirrored(fr.left, W))
    orig = accepted_pairs(best, dist)
    mirr = {(int(j), i, int(d)) for i, j, d in accepted_pairs(mbest, mdist)}
    assert len(orig) > 250
    assert orig == mirr


def test_fisheye_overlap_pairs_are_mirror_consistent():
    fr = scenes.fisheye_frame(42, n_left=800, n_map=10)
    rig = fr.rig
    W = rig.left.width
    w1 = float(W - 1)
    flat = scenes.FisheyeRig(left=None, right=None, R_rl=rig.R_rl, t_rl=rig.t_rl, b=rig.b,
                             lap_l0=rig.lap_l0, lap_l1=rig.lap_l1, lap_r0=rig.lap_r0, lap_r1=rig.lap_r1)
    # mirrored rig: the right overlap range, mirrored, becomes the left one and vice versa
    mrig = scenes.FisheyeRig(left=None, right=None, R_rl=rig.R_rl, t_rl=rig.t_rl, b=rig.b,
                             lap_l0=w1 - rig.lap_r1, lap_l1=w1 - rig.lap_r0, lap_r0=w1 - rig.lap_l1,
                             lap_r1=w1 - rig.lap_l0)
    lo = (fr.left.x >= rig.lap_l0) & (fr.left.x <= rig.lap_l1)
    ro = (fr.right.x >= rig.lap_r0) & (fr.right.x <= rig.lap_r1)
    D = hamming_matrix(fr.left.desc[lo], fr.right.desc[ro])
    # tie-free for the ratio test: a distance below 60 is alone in its row and
    # column and every other one is at least 86, so 0.7 * d2 > d1 both ways
    low = D < 60
    assert low.sum(axis=1).max() <= 1 and low.sum(axis=0).max() <= 1
    assert D[~low].min() >= 86
    st = orc.stereo_fisheye(P, flat, fr.left, fr.right)
    ms = orc.stereo_fisheye(P, mrig, mirrored(fr.right, W), mirrored(fr.left, W))
    orig = accepted_pairs(st["r_idx"], st["d1"])
    mirr = {(int(j), i, int(d)) for i, j, d in accepted_pairs(ms["r_idx"], ms["d1"])}
    assert len(orig) > 200
    assert orig == mirr


def shifted_scene(seed: int, W=320, H=160, d=17, n=160):
    """Zero-noise stereo pair: right(x, y) = left(x + d, y); octave-0
    keypoints on whole pixels, each right keypoint offset from the true match
    by e in [-2, 2] (e = 0 for the first 60)."""
    rng = np.random.default_rng(seed)
    left = scenes.band_limited_noise(rng, H, W)
    right = left.copy()
    right[:, : W - d] = left[:, d:]
    right[:, W - d:] = scenes.band_limited_noise(rng, H, d)
    xl = rng.choice(np.arange(d + 16, W - 16), n, replace=False).astype(np.float32)
    y = rng.integers(12, H - 12, n).astype(np.float32)
    e = rng.integers(-2, 3, n)
    e[:60] = 0
    xr = (xl - d + e).astype(np.float32)
    desc = scenes.random_desc(rng, n)
    oct0 = np.zeros(n, np.int8)
    L = scenes.Keypoints(x=xl, y=y, oct=oct0, desc=desc)
    R = scenes.Keypoints(x=xr, y=y.copy(), oct=oct0.copy(), desc=scenes.flip_bits(rng, desc, 0.05))
    cam = scenes.pinhole_camera(W, H)
    return left, right, L, R, e, cam


def test_sad_and_parabola_under_the_mirror():
    d = 17
    left, right, L, R, e, cam = shifted_scene(43, d=d)
    W = cam.width
    pl, pr = scenes.build_pyramid(left), scenes.build_pyramid(right)
    ml, mr = scenes.build_pyramid(np.ascontiguousarray(right[:, ::-1])), \
        scenes.build_pyramid(np.ascontiguousarray(left[:, ::-1]))
    st = orc.stereo_pinhole(P, cam, L, R, pl, pr)
    ms = orc.stereo_pinhole(P, cam, mirrored(R, W), mirrored(L, W), ml, mr)
    n = L.n
    # every keypoint is matched to its partner in both runs (distinct random descriptors)
    assert np.array_equal(st["best_r"], np.arange(n))
    assert np.array_equal(ms["best_r"], np.arange(n))
    assert np.array_equal(st["dist"], ms["dist"])
    # the best shift undoes the offset in both runs; the integer disparity is d in both
    assert np.array_equal(st["sad_shift"], -e)
    assert np.array_equal(ms["sad_shift"], -e)
    assert np.all(st["sad_best"] == 0) and np.all(ms["sad_best"] == 0)
    xl = L.x.astype(np.int64)
    xr = R.x.astype(np.int64)
    assert np.all(xl - (xr + st["sad_shift"]) == d)
    xl_m = (W - 1) - xr
    xr_m = (W - 1) - xl
    assert np.all(xl_m - (xr_m + ms["sad_shift"]) == d)
    Lw = P["sad_L"]
    checked = 0
    for i in np.nonzero(e == 0)[0]:
        v = int(L.y[i])
        s = orc.sad_vector(P, pl, pr, 0, int(xl[i]), v, int(xr[i]))
        sm = orc.sad_vector(P, ml, mr, 0, int(xl_m[i]), v, int(xr_m[i]))
        assert s is not None and sm is not None
        assert np.array_equal(sm, s[::-1]), i
        ok, ur, disp, delta = orc.subpixel(s, Lw, 0, int(xr[i]), 1.0, float(L.x[i]), cam.bf, cam.fx)
        okm, urm, dispm, deltam = orc.subpixel(sm, Lw, 0, int(xr_m[i]), 1.0, float(xl_m[i]), cam.bf, cam.fx)
        assert ok and okm
        assert deltam == -delta
        assert abs((xl[i] - ur) + (xl_m[i] - urm) - 2 * d) < 1e-4
        checked += 1
    assert checked >= 60
