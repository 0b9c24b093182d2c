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
