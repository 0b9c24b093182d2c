"""Pins of the oracle's keypoint detection and description (next row f3;
the paper's ORB extraction finds keypoints on every pyramid level,
describes them and filters them, section II-A).

What fixes each step independently of the oracle's code:
* FAST: hand-built circles (a bright dot, 9 contiguous pixels just above and
  at the threshold, 8 pixels, an arc across the circle's start); the score
  equals the largest threshold at which a segment test written here (runs
  on the doubled circle) still passes, on random patches;
* non-maximum suppression and filtering: a brute force over a small image
  (corner map, neighbour rule, ordering and caps written here with numpy);
* smoothing: scipy's correlation with the 5x5 binomial kernel (nearest
  border), rounded half up;
* orientation: exact 90-degree rotation of the patch turns (c, s) into
  (-s, c) bit for bit; an off-centre bright spot points the orientation at
  it;
* descriptor: the bits recomputed here from the definition (float32 numpy,
  rounding half away from zero) on the scipy-smoothed image; and the exact
  invariance: the 90-degree rotated image gives the same 256 bits;
* end to end: keypoints extracted from both images of a generated stereo
  pair are matched by the oracle's stereo matching with disparities close
  to the generator's planes.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes

ndimage = pytest.importorskip("scipy.ndimage")

P = dict(scenes.DEFAULT_PARAMS)
CIRCLE = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
          (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]


def segment_test(img, x, y, t):
    """9 contiguous circle pixels all > I + t or all < I - t (runs on the
    circle listed twice)."""
    c = int(img[y, x])
    vals = [int(img[y + dy, x + dx]) for dx, dy in CIRCLE]
    for pred in (lambda v: v > c + t, lambda v: v < c - t):
        run = best = 0
        for v in vals + vals:
            run = run + 1 if pred(v) else 0
            best = max(best, run)
        if best >= 9:
            return True
    return False


def blank(v=100, n=15):
    return np.full((n, n), v, np.uint8)


def test_fast_hand_cases():
    img = blank()
    img[7, 7] = 200                                  # a bright dot: every circle pixel is darker by 100
    assert orc.fast_score(img, 7, 7, 20) == 99
    assert orc.fast_score(img, 7, 7, 99) == 99 and orc.fast_score(img, 7, 7, 100) == -1
    for n, start, ok in ((9, 0, True), (8, 0, False), (9, 12, True), (9, 5, True)):
        img = blank()
        for k in range(n):
            dx, dy = CIRCLE[(start + k) % 16]
            img[7 + dy, 7 + dx] = 121                # brighter by exactly t + 1
        s = orc.fast_score(img, 7, 7, 20)
        assert (s >= 0) == ok, (n, start)
        if ok:
            assert s == 20
        img2 = img.copy()
        img2[img2 == 121] = 120                      # brighter by exactly t: not a corner
        assert orc.fast_score(img2, 7, 7, 20) == -1


def test_fast_score_is_the_largest_passing_threshold():
    rng = np.random.default_rng(1)
    n = 0
    for _ in range(300):
        img = rng.integers(0, 256, (7, 7)).astype(np.uint8)
        if rng.random() < 0.5:                       # make corners likely
            img[3, 3] = rng.choice([5, 250])
        s = orc.fast_score(img, 3, 3, 0)
        passing = [t for t in range(0, 256) if segment_test(img, 3, 3, t)]
        assert s == (max(passing) if passing else -1)
        for t in (10, 40):
            assert (orc.fast_score(img, 3, 3, t) >= 0) == segment_test(img, 3, 3, t)
        n += s >= 0
    assert n > 50


def test_smoothing_is_the_binomial_filter():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, (40, 53)).astype(np.uint8)
    b = np.array([1, 4, 6, 4, 1])
    k = np.outer(b, b)
    acc = ndimage.correlate(img.astype(np.int64), k, mode="nearest")
    assert np.array_equal(orc.smooth_level(img), ((acc + 128) // 256).astype(np.uint8))


def rot90_about(img, x, y, r):
    """Patch of half size r around (x, y) rotated so that image point
    (x + u, y + v) moves to (x - v, y + u); returns the new image (same
    centre)."""
    out = img.copy()
    patch = img[y - r:y + r + 1, x - r:x + r + 1]
    # new[v', u'] = old at (u, v) with (u', v') = (-v, u)  =>  new[v', u'] = old[-u', v']
    out[y - r:y + r + 1, x - r:x + r + 1] = np.rot90(patch, k=-1)
    return out


def test_orientation_rotates_exactly_with_the_patch():
    rng = np.random.default_rng(3)
    img = scenes.band_limited_noise(rng, 80, 80)
    x = y = 40
    cs = orc.orientation(img, x, y)
    r = orc.orientation(rot90_about(img, x, y, 30), x, y)
    assert r[0] == -cs[1] and r[1] == cs[0]
    # a bright spot at 30 degrees from the centre
    img = np.full((60, 60), 50, np.uint8)
    ang = np.radians(30.0)
    img[int(round(30 + 9 * np.sin(ang))), int(round(30 + 9 * np.cos(ang)))] = 250
    c, s = orc.orientation(img, 30, 30)
    assert abs(np.degrees(np.arctan2(s, c)) - 30.0) < 4.0
    assert np.array_equal(orc.orientation(np.full((40, 40), 9, np.uint8), 20, 20), [1.0, 0.0])
    # the disk u^2 + v^2 <= 15^2: a lone pixel at (0, 15) or (-9, -12) counts,
    # one at (11, 11) (distance 15.6) does not
    for (u, v, want) in ((0, 15, [0.0, 1.0]), (-9, -12, [-0.6, -0.8]), (11, 11, [1.0, 0.0])):
        img = np.zeros((40, 40), np.uint8)
        img[20 + v, 20 + u] = 200
        assert np.allclose(orc.orientation(img, 20, 20), want, atol=1e-7), (u, v)


def round_half_away(v):
    v = np.float32(v)
    return int(np.sign(v) * np.floor(np.abs(v) + np.float32(0.5)))


def test_descriptor_bits_from_the_definition():
    rng = np.random.default_rng(4)
    img = scenes.band_limited_noise(rng, 90, 90)
    pat = scenes.orb_pattern()
    b = np.array([1, 4, 6, 4, 1])
    sm = ((ndimage.correlate(img.astype(np.int64), np.outer(b, b), mode="nearest") + 128) // 256).astype(np.uint8)
    for (x, y) in ((45, 45), (30, 60), (60, 28)):
        cs = orc.orientation(img, x, y)
        c, s = np.float32(cs[0]), np.float32(cs[1])
        bits = []
        for i in range(256):
            v = []
            for q in range(2):
                px, py = np.float32(pat[i, 2 * q]), np.float32(pat[i, 2 * q + 1])
                u = round_half_away(np.float32(c * px) - np.float32(s * py))
                w = round_half_away(np.float32(s * px) + np.float32(c * py))
                v.append(int(sm[y + w, x + u]))
            bits.append(v[0] < v[1])
        ref = np.packbits(np.array(bits, np.uint8), bitorder="little")
        assert np.array_equal(orc.describe(orc.smooth_level(img), x, y, cs, pat), ref)


def test_descriptor_invariant_under_exact_rotation():
    rng = np.random.default_rng(5)
    img = scenes.band_limited_noise(rng, 100, 100)
    pat = scenes.orb_pattern()
    x = y = 50
    rot = rot90_about(img, x, y, 40)
    d0 = orc.describe(orc.smooth_level(img), x, y, orc.orientation(img, x, y), pat)
    d1 = orc.describe(orc.smooth_level(rot), x, y, orc.orientation(rot, x, y), pat)
    assert np.array_equal(d0, d1)
    # and a plain image rotation changes the unsteered tests (the steering matters)
    d2 = orc.describe(orc.smooth_level(rot), x, y, np.array([1.0, 0.0], np.float32), pat)
    d3 = orc.describe(orc.smooth_level(img), x, y, np.array([1.0, 0.0], np.float32), pat)
    assert not np.array_equal(d2, d3)


def brute_force_level(img, t, edge, cap):
    h, w = img.shape
    sco = np.full((h, w), -1, np.int64)
    for y in range(edge, h - edge):
        for x in range(edge, w - edge):
            if segment_test(img, x, y, t):
                sco[y, x] = max(tt for tt in range(t, 256) if segment_test(img, x, y, tt))
    kept = []
    for y in range(edge, h - edge):
        for x in range(edge, w - edge):
            if sco[y, x] < 0:
                continue
            ok = True
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dx or dy) and sco[y + dy, x + dx] >= 0:
                        q = sco[y + dy, x + dx]
                        earlier = (y + dy, x + dx) < (y, x)
                        if q > sco[y, x] or (q == sco[y, x] and earlier):
                            ok = False
            if ok:
                kept.append((-int(sco[y, x]), y, x))
    kept.sort()
    return kept[:cap], len(kept)


def test_detection_suppression_and_filtering_brute_force():
    rng = np.random.default_rng(6)
    img = scenes.band_limited_noise(rng, 64, 72, sigma=1.2)
    levels = [img]
    p = dict(P, nlevels=1)
    pat = scenes.orb_pattern()
    for cap in (5, 40, 10000):
        ref, n_all = brute_force_level(img, 20, 19, cap)
        out = orc.extract_orb(p, levels, 20, 19, [cap], pat)
        n = len(ref)
        assert out["n_level"][0] == n and out["n_level"][1] == n
        assert np.array_equal(out["score"][:n], [-s for s, _, _ in ref])
        assert np.array_equal(out["x"][:n], [float(x) for _, _, x in ref])
        assert np.array_equal(out["y"][:n], [float(y) for _, y, _ in ref])
        if cap > n:
            assert np.all(out["x"][n:cap] == -1e9) and np.all(out["score"][n:cap] == -1)
            assert np.all(out["desc"][n:cap] == 0)
    assert n_all > 40


def test_levels_scale_and_slots():
    imgs = scenes.stereo_images(7, scenes.pinhole_camera(320, 240))
    caps = scenes.orb_level_caps(500)
    out = orc.extract_orb(P, imgs.pyr_left, 20, 19, caps, scenes.orb_pattern())
    sc = scenes.level_scales32()
    off = 0
    for l, cap in enumerate(caps):
        n = out["n_level"][l]
        sl = slice(off, off + n)
        assert np.all(out["oct"][sl] == l)
        # level-0 coordinates are level pixels times the FP32 scale
        xl = out["x"][sl] / sc[l]
        assert np.all(np.abs(xl - np.rint(xl)) < 1e-3)
        assert np.all(out["x"][sl] == (np.rint(xl).astype(np.float32) * sc[l]).astype(np.float32))
        off += cap
    assert out["n_level"][-1] == sum(out["n_level"][:-1])


def test_extracted_stereo_pair_matches_the_planted_disparities():
    cam = scenes.pinhole_camera()
    imgs = scenes.stereo_images(8, cam)
    caps = scenes.orb_level_caps(1200)
    pat = scenes.orb_pattern()
    L = orc.extract_orb(P, imgs.pyr_left, 20, 19, caps, pat)
    R = orc.extract_orb(P, imgs.pyr_right, 20, 19, caps, pat)
    kl = scenes.Keypoints(x=L["x"], y=L["y"], oct=L["oct"], desc=L["desc"])
    kr = scenes.Keypoints(x=R["x"], y=R["y"], oct=R["oct"], desc=R["desc"])
    st = orc.stereo_pinhole(P, cam, kl, kr, imgs.pyr_left, imgs.pyr_right)
    ok = st["u_right"] >= 0
    assert ok.sum() > 300
    x, y = L["x"][ok], L["y"][ok]
    lab = imgs.label[np.clip(np.rint(y).astype(int), 0, cam.height - 1), np.clip(np.rint(x).astype(int), 0,
                                                                                   cam.width - 1)]
    disp_true = cam.fx * cam.b / imgs.depth[lab]
    err = np.abs((x - st["u_right"][ok]) - disp_true)
    assert np.median(err) < 1.0 and np.mean(err < 2.0) > 0.8
