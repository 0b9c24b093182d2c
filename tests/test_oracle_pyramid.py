"""Pins of the oracle's image pyramid (next row f3, its pyramid part): level
sizes against round(W / 1.2^l), constant and linear images (bilinear
resampling reproduces a linear image up to the final rounding), the identity
at scale 1, hand-worked clamping at the borders, and the generator's own
double-precision resampling (equal but for values at a rounding tie)."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes


@pytest.mark.parametrize("W,H", [(752, 480), (640, 480), (1280, 720), (512, 512), (1920, 1080), (37, 23)])
def test_level_sizes(W, H):
    ws, hs = orc.pyramid_sizes(W, H, 8, 1.2)
    for l in range(8):
        assert ws[l] == int(math.floor(W / 1.2 ** l + 0.5)) and hs[l] == int(math.floor(H / 1.2 ** l + 0.5)), l


def test_constant_image():
    img = np.full((480, 752), 137, np.uint8)
    for lvl in orc.build_pyramid(img)[1:]:
        assert np.all(lvl == 137)


def test_linear_image_is_reproduced():
    W, H = 752, 480
    x = np.arange(W)[None, :]
    y = np.arange(H)[:, None]
    a, b, c = 0.21, 0.13, 9.0
    img = np.rint(a * x + b * y + c).astype(np.uint8)   # exact linear values below 255
    ws, hs = orc.pyramid_sizes(W, H)
    for l in range(1, 8):
        out = orc.resample_level(img, ws[l], hs[l]).astype(np.float64)
        xs = np.clip((np.arange(ws[l]) + 0.5) * W / ws[l] - 0.5, 0, W - 1)[None, :]
        ys = np.clip((np.arange(hs[l]) + 0.5) * H / hs[l] - 0.5, 0, H - 1)[:, None]
        # the source holds the line rounded to integers (|error| <= 0.5); the
        # resampled value adds its own rounding (<= 0.5) and FP32 noise
        assert np.max(np.abs(out - (a * xs + b * ys + c))) <= 1.0 + 1e-3, l


def test_identity_at_scale_one():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (31, 45), dtype=np.uint8)
    assert np.array_equal(orc.resample_level(img, 45, 31), img)


def test_border_clamping_by_hand():
    # 2 x 2 source upsampled to 3 x 3: xs = (x + 0.5) * 2/3 - 0.5 = -1/6, 1/2, 7/6
    img = np.array([[0, 90], [30, 210]], np.uint8)
    out = orc.resample_level(img, 3, 3)
    # x: clamped to 0 (weights 1, 0), half way, then 1 + 1/6 -> x0 = 1, x1 = 1
    top = [0.0, 45.0, 90.0]
    bot = [30.0, 120.0, 210.0]
    want = np.array([top, [(t + b) / 2 for t, b in zip(top, bot)], bot])
    assert np.array_equal(out, np.rint(want).astype(np.uint8))


def test_agrees_with_the_generator_resampling():
    fr = scenes.single_pinhole(4)
    pyr = orc.build_pyramid(fr.pyr_left[0])
    for l in range(1, 8):
        d = pyr[l].astype(int) - fr.pyr_left[l].astype(int)
        assert np.all(np.abs(d) <= 1), l
        assert np.mean(d != 0) < 0.005, l


def _round_f32(q):
    """The float32 nearest to the exact rational q >= 0, ties to even."""
    from fractions import Fraction
    if q == 0:
        return np.float32(0)
    e = math.floor(math.log2(q))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    ulp = Fraction(2) ** (e - 23)
    m = q / ulp
    lo = math.floor(m)
    r = m - lo
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return np.float32(float(lo * ulp))


def test_products_are_rounded_before_the_sum():
    # One pixel of a seeded 752x480 image (level 5, row 9, column 225) whose
    # value is an exact tie, 177.5, when top (1-fy) and bottom fy are each
    # rounded to FP32 before their sum (178 after rounding half to even); a
    # fused multiply-add of the first product into the sum gives 177.49998
    # (177).  Exact rational arithmetic decides both, and the oracle (built
    # without contraction) must give 178.
    from fractions import Fraction
    f32 = np.float32
    rng = np.random.default_rng(752)
    img = rng.integers(0, 256, size=(480, 752), dtype=np.uint8)
    ws, hs = orc.pyramid_sizes(752, 480, 8, 1.2)
    w, h, y, x = ws[5], hs[5], 9, 225
    sx, sy = f32(752) / f32(w), f32(480) / f32(h)
    xs = min(max((f32(x) + f32(0.5)) * sx - f32(0.5), f32(0)), f32(751))
    ys = min(max((f32(y) + f32(0.5)) * sy - f32(0.5), f32(0)), f32(479))
    x0, y0 = int(np.floor(xs)), int(np.floor(ys))
    fx, fy = f32(xs - f32(x0)), f32(ys - f32(y0))
    gx, gy = f32(1) - fx, f32(1) - fy
    top = f32(f32(f32(img[y0, x0]) * gx) + f32(f32(img[y0, x0 + 1]) * fx))
    bot = f32(f32(f32(img[y0 + 1, x0]) * gx) + f32(f32(img[y0 + 1, x0 + 1]) * fx))
    F = lambda v: Fraction(float(v))
    separate = _round_f32(F(_round_f32(F(top) * F(gy))) + F(_round_f32(F(bot) * F(fy))))
    fused = _round_f32(F(top) * F(gy) + F(_round_f32(F(bot) * F(fy))))
    assert separate == f32(177.5) and fused < f32(177.5)
    assert orc.resample_level(img, w, h)[y, x] == 178
