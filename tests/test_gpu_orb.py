"""GPU parity of keypoint detection and description (next row f3) through
the C ABI: ft_extract_orb against the CPU oracle, bit for bit on every
output (coordinates, octaves, scores, orientation cosines and sines,
descriptors, per-level counts), and the extraction feeding ft_track_batch
on the device with no host round trip."""
import ctypes as C

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes
from tests.gpu_common import assert_search_equal, assert_stereo_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P = dict(scenes.DEFAULT_PARAMS)
KEYS = ("x", "y", "oct", "score", "cs", "desc", "n_level")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2509_10757_gb300 import build
    build.build()
    from paper_2509_10757_gb300 import _lib as L
    return L


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_2509_10757_gb300.batch import Context
    c = Context(arena_bytes=1 << 30, max_frames=64)
    yield c
    c.close()


def device_pyramid(lib, levels):
    """An ft_pyramid over device copies of the levels (16-byte aligned rows)."""
    from paper_2509_10757_gb300.batch import pad_rows
    keep = []
    s = lib.ft_pyramid()
    s.nlevels = len(levels)
    for l, img in enumerate(levels):
        t = torch.from_numpy(pad_rows(img)).cuda()
        keep.append(t)
        s.data[l] = t.data_ptr()
        s.height[l], s.width[l] = img.shape
        s.pitch[l] = t.shape[1]
    return s, keep


def extract(ctx, lib, pyramids, caps, pattern, fast_th=20, edge=19):
    from paper_2509_10757_gb300.batch import OrbOutputs, run_extract
    oo = OrbOutputs(len(pyramids), caps, pattern, fast_th, edge)
    structs, keep = zip(*[device_pyramid(lib, lv) for lv in pyramids])
    run_extract(ctx, list(structs), oo)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    return oo.download_all()


def assert_orb_equal(got, ref, where):
    for k in KEYS:
        a, b = got[k], ref[k]
        if a.dtype == np.float32:
            a, b = a.view(np.uint32), b.view(np.uint32)
        bad = np.nonzero(np.any((a != b).reshape(len(a), -1), axis=1))[0]
        assert len(bad) == 0, f"{where}{k}: {len(bad)} differ, first {bad[:5].tolist()}"


def low_contrast_pyramid(seed, W, H, amp):
    rng = np.random.default_rng(seed)
    img = scenes.band_limited_noise(rng, H, W, sigma=2.0).astype(np.float64)
    img = np.clip(np.rint(128 + (img - 128) * amp), 0, 255).astype(np.uint8)
    return scenes.build_pyramid(img)


@pytest.mark.parametrize("shape,n_feat", [((752, 480), 1200), ((640, 480), 500), ((1280, 720), 3000),
                                          ((333, 217), 800), ((160, 120), 300)])
def test_extraction_matches_the_oracle(ctx, lib, shape, n_feat):
    W, H = shape
    imgs = scenes.stereo_images(31 + W, scenes.pinhole_camera(W, H))
    caps = scenes.orb_level_caps(n_feat)
    pat = scenes.orb_pattern()
    got = extract(ctx, lib, [imgs.pyr_left, imgs.pyr_right], caps, pat)
    for i, lv in enumerate((imgs.pyr_left, imgs.pyr_right)):
        ref = orc.extract_orb(P, lv, 20, 19, caps, pat)
        assert_orb_equal(got[i], ref, f"{shape} image {i}: ")
        assert ref["n_level"][-1] > 0


def test_fewer_corners_than_slots_and_odd_caps(ctx, lib):
    pyrs = [low_contrast_pyramid(40 + i, 752, 480, a) for i, a in enumerate((0.25, 0.35, 0.0))]
    caps = [4096, 0, 700, 3, 1, 0, 250, 4096]
    pat = scenes.orb_pattern(7)
    got = extract(ctx, lib, pyrs, caps, pat)
    for i, lv in enumerate(pyrs):
        ref = orc.extract_orb(P, lv, 20, 19, caps, pat)
        assert_orb_equal(got[i], ref, f"image {i}: ")
    assert got[2]["n_level"][-1] == 0                       # a flat image: padding only
    assert np.all(got[2]["x"] == -1e9) and np.all(got[2]["desc"] == 0)


@pytest.mark.parametrize("fast_th,edge", [(10, 19), (40, 19), (20, 31)])
def test_parameter_variants(ctx, lib, fast_th, edge):
    imgs = scenes.stereo_images(50, scenes.pinhole_camera())
    caps = scenes.orb_level_caps(1500)
    pat = scenes.orb_pattern(11)
    got = extract(ctx, lib, [imgs.pyr_left], caps, pat, fast_th, edge)
    assert_orb_equal(got[0], orc.extract_orb(P, imgs.pyr_left, fast_th, edge, caps, pat), f"t={fast_th} e={edge}: ")


def test_batch_of_images(ctx, lib):
    cam = scenes.pinhole_camera()
    pyrs = []
    for s in range(12):
        imgs = scenes.stereo_images(60 + s, cam)
        pyrs += [imgs.pyr_left, imgs.pyr_right]
    caps = scenes.orb_level_caps(1200)
    pat = scenes.orb_pattern()
    got = extract(ctx, lib, pyrs, caps, pat)
    for i, lv in enumerate(pyrs):
        assert_orb_equal(got[i], orc.extract_orb(P, lv, 20, 19, caps, pat), f"image {i}: ")


def test_extraction_feeds_tracking_on_the_device(ctx, lib):
    """ft_extract_orb then ft_track_batch on the same stream, the batch's
    keypoints pointing at the extraction outputs: stereo and search results
    equal the oracle's on the oracle's extraction."""
    from paper_2509_10757_gb300.batch import OrbOutputs, PackedBatch, run_batch, run_extract
    cam = scenes.pinhole_camera()
    caps = scenes.orb_level_caps(1200)
    pat = scenes.orb_pattern()
    frames, structs, keep = [], [], []
    for s in range(4):
        imgs = scenes.stereo_images(70 + s, cam)
        L_ = orc.extract_orb(P, imgs.pyr_left, 20, 19, caps, pat)
        R_ = orc.extract_orb(P, imgs.pyr_right, 20, 19, caps, pat)
        kl = scenes.Keypoints(x=L_["x"], y=L_["y"], oct=L_["oct"], desc=L_["desc"])
        kr = scenes.Keypoints(x=R_["x"], y=R_["y"], oct=R_["oct"], desc=R_["desc"])
        frames.append(scenes.frame_with_keypoints(80 + s, cam, imgs, kl, kr))
    pb = PackedBatch(frames)
    pb.upload()
    pb.clear_outputs()
    oo = OrbOutputs(2 * len(frames), caps, pat)
    pyr_structs = []
    for f in range(len(frames)):
        pyr_structs += [pb.pyramid(f, "L"), pb.pyramid(f, "R")]
    # the keypoint inputs the batch uploaded are zeroed on the device: the
    # tracking must read the extraction's outputs
    for f in range(len(frames)):
        for key in ("lx", "ly", "loct", "ldesc", "rx", "ry", "roct", "rdesc"):
            _, off, dt, shape = pb.lin.items[pb.lin.index[(f, key)]]
            pb.dev_in[off:off + int(np.prod(shape)) * dt.itemsize].zero_()
    run_extract(ctx, pyr_structs, oo)
    for f in range(len(frames)):
        pb.jobs[f].left = oo.keypoints(2 * f)
        pb.jobs[f].right = oo.keypoints(2 * f + 1)
    run_batch(ctx, pb)
    pb.download()
    assert ctx.sync_status() == 0
    for f, fr in enumerate(frames):
        out = pb.outputs(f)
        st, se = orc.track_frame(P, fr)
        assert_stereo_equal(out, st, f"frame {f}: ")
        assert_search_equal(out, se, "l", None, f"frame {f}: ")
        assert (st["u_right"] >= 0).sum() > 200 and (se["mp_kp"] >= 0).sum() > 100


def test_host_checks(ctx, lib):
    from paper_2509_10757_gb300.batch import OrbOutputs, stream_handle
    imgs = scenes.stereo_images(90, scenes.pinhole_camera(320, 240))
    s, keep = device_pyramid(lib, imgs.pyr_left)
    caps = scenes.orb_level_caps(300)
    pat = scenes.orb_pattern()
    oo = OrbOutputs(1, caps, pat)
    arr = (lib.ft_pyramid * 1)(s)

    def call(params=None):
        return ctx.lib.ft_extract_orb(ctx.ptr, stream_handle(), None, 1, arr, C.byref(params or oo.params), oo.outs)

    bad = np.array(pat)
    bad[5, 2] = 14
    p = lib.ft_orb_params.from_buffer_copy(oo.params)
    p.pattern = bad.ctypes.data
    assert call(p) == lib.FT_EINVAL and "pattern" in lib.last_error()
    for field, v in (("edge", 18), ("fast_th", 0), ("fast_th", 255)):
        p = lib.ft_orb_params.from_buffer_copy(oo.params)
        setattr(p, field, v)
        assert call(p) == lib.FT_EINVAL, field
    p = lib.ft_orb_params.from_buffer_copy(oo.params)
    p.max_kp[0] = 4097
    assert call(p) == lib.FT_EINVAL
    saved = oo.outs[0].desc
    oo.outs[0].desc = saved + 4
    assert call() == lib.FT_EALIGN
    oo.outs[0].desc = saved
    assert call() == lib.FT_OK
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
