"""GPU parity: libfasttrack.so (through its C ABI) against the CPU oracle,
element by element, on seeded synthetic frames.  Sizes span several work
items with ragged tails (15 stereo strips of 32 rows at 480 rows, search
tiles of 512 map points with a partial last tile, fisheye tiles of 256 left
keypoints with a partial last tile)."""
import ctypes as C
import dataclasses

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes
from tests.gpu_common import (assert_fisheye_equal, assert_search_equal, assert_stereo_equal)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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
    c = Context(arena_bytes=1 << 30, max_frames=256)
    yield c
    c.close()


def _params(lib, overrides=None):
    return lib.default_params(overrides)


def _oracle_params(overrides=None):
    p = dict(scenes.DEFAULT_PARAMS)
    p.update(overrides or {})
    return p


def check_frame(pb, f, params=None, what=""):
    fr = pb.frames[f]
    out = pb.outputs(f)
    st, se = orc.track_frame(_oracle_params(params), fr)
    where = f"{what} frame {f} ({fr.camera}): "
    if fr.camera == "pinhole":
        assert_stereo_equal(out, st, where)
        assert_search_equal(out, se, "l", None, where)
    else:
        assert_fisheye_equal(out, st, where)
        assert_search_equal(out, se, "l", "l", where)
        assert_search_equal(out, se, "r", "r", where)
    return out, st, se


def run_per_frame(ctx, frames, params=None, lib=None):
    from paper_2509_10757_gb300.batch import PackedBatch, run_search, run_stereo
    pb = PackedBatch(frames)
    pb.upload()
    pb.clear_outputs()
    p = lib.default_params(params) if lib is not None else None
    for f in range(len(frames)):
        run_stereo(ctx, pb, f, p)
        run_search(ctx, pb, f, p)
    pb.download()
    assert ctx.sync_status() == 0
    return pb


def run_fused(ctx, frames, params=None, lib=None, stage=False):
    from paper_2509_10757_gb300.batch import PackedBatch, run_batch
    pb = PackedBatch(frames)
    if not stage:
        pb.upload()
    pb.clear_outputs()
    p = lib.default_params(params) if lib is not None else None
    run_batch(ctx, pb, p, stage=stage)
    if stage:
        torch.cuda.synchronize()
    else:
        pb.download()
    assert ctx.sync_status() == 0
    return pb


# ---------------------------------------------------------------- single frames
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pinhole_frame_per_call(ctx, lib, seed):
    pb = run_per_frame(ctx, [scenes.single_pinhole(seed)], lib=lib)
    out, st, _ = check_frame(pb, 0, what="per-call")
    assert (st["u_right"] >= 0).sum() > 300 and (out["mp_kp_l"] >= 0).sum() > 100


@pytest.mark.parametrize("seed", [0, 1])
def test_fisheye_frame_per_call(ctx, lib, seed):
    pb = run_per_frame(ctx, [scenes.fisheye_frame(seed)], lib=lib)
    out, st, _ = check_frame(pb, 0, what="per-call")
    assert (st["r_idx"] >= 0).sum() > 300


def test_search_without_stereo_check(ctx, lib):
    from paper_2509_10757_gb300.batch import PackedBatch, run_search
    fr = scenes.single_pinhole(5)
    pb = PackedBatch([fr])
    pb.upload()
    pb.clear_outputs()
    run_search(ctx, pb, 0, u_right=False)
    pb.download()
    se = orc.search_frame(_oracle_params(), fr, None)
    assert_search_equal(pb.outputs(0), se, "l")


# ---------------------------------------------------------------- fused batch
def test_batch_mixed_shapes_matches_oracle(ctx, lib):
    frames = [scenes.served_stream_frame(0, s) for s in range(8)]
    assert {f.camera for f in frames} == {"pinhole", "fisheye"}
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="batch")


def test_batch_equals_per_call(ctx, lib):
    frames = [scenes.single_pinhole(3), scenes.fisheye_frame(3), scenes.single_pinhole(4)]
    a = run_per_frame(ctx, frames)
    b = run_fused(ctx, frames)
    assert np.array_equal(a.host_out.numpy(), b.host_out.numpy())


def test_batch_64_frames_full_size(ctx, lib):
    frames = scenes.pinhole_batch(seed=0, n_frames=64)
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="64-frame batch")


def test_fisheye_batch_full_size(ctx, lib):
    frames = scenes.fisheye_batch(seed=0, n_frames=8)
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="fisheye batch")


def test_fisheye_rotated_rig_local_map_and_last_frame(ctx, lib):
    """A rig whose right camera is rotated 15 degrees from the left one: the
    right camera's pose (T_rl T_lw) and centre matter to every right-camera
    projection, distance and viewing angle, in the local-map search and in
    the last-frame search."""
    from paper_2509_10757_gb300.batch import PackedBatch, run_batch
    from tests.test_oracle_fisheye_rig import rotated_rig
    frames = [scenes.fisheye_frame(60 + i, n_left=1500, n_map=6000, rig=rotated_rig(5 + i)) for i in range(4)]
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        out, _, se = check_frame(pb, f, what="rotated rig")
        assert (se["mp_kp_r"] >= 0).sum() > 200
    lasts = [scenes.last_frame(fr, 70 + i, mo) for i, (fr, mo) in
             enumerate(zip(frames, ["forward", "backward", "none", "none"]))]
    pb = PackedBatch(frames, lasts=lasts)
    pb.upload()
    pb.clear_outputs()
    run_batch(ctx, pb)
    pb.download()
    assert ctx.sync_status() == 0
    for f, fr in enumerate(frames):
        st = orc.stereo_frame(_oracle_params(), fr)
        assert_fisheye_equal(pb.outputs(f), st, f"rotated rig frame {f}: ")
        ref = _check_last(pb, f, st, f"rotated rig last-frame {f}: ")
        assert (ref["mp_kp_r"] >= 0).sum() > 50


def test_stress_frames(ctx, lib):
    frames = scenes.stress_batch(seed=0, n_frames=2, n_map=100_000)
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="1080p stress")


def test_search_keypoints_on_chip_boundary(ctx, lib):
    # the search keeps up to 1536 keypoints of a camera in shared memory (and
    # the grid's 16-bit cell starts too up to 1407 keypoints) and reads larger
    # frames from device memory: both sides of each boundary, fused (right
    # coordinates from the stereo step) and per call
    frames = [scenes.pinhole_frame(40 + n, 752, 480, n, 0.2, 0.05, 3000) for n in (1407, 1408, 1536, 1537)]
    frames.append(scenes.fisheye_frame(43, 1536, n_map=3000))
    frames.append(scenes.fisheye_frame(44, 1537, n_map=3000))
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="on-chip boundary, fused")
    pb = run_per_frame(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="on-chip boundary, per call")


def test_fisheye_triangulation_outputs_are_optional(ctx, lib):
    # depth without xyz, and neither (matching only): the other outputs stay
    # untouched and the matches are the same
    from paper_2509_10757_gb300.batch import PackedBatch, rig_struct, stream_handle
    fr = scenes.fisheye_frame(9)
    st = orc.stereo_frame(_oracle_params(), fr)
    pb = PackedBatch([fr])
    pb.upload()
    rig = rig_struct(fr.rig)
    kl, kr = pb.keypoints(0, "l"), pb.keypoints(0, "r")
    for keep_depth in (True, False):
        pb.clear_outputs(0x5a)
        out = pb.fisheye_out(0)
        out.xyz = None
        if not keep_depth:
            out.depth = None
        lib.check(ctx.lib.ft_stereo_match_fisheye(ctx.ptr, stream_handle(), None, C.byref(rig), C.byref(kl),
                                                  C.byref(kr), C.byref(out)), "ft_stereo_match_fisheye")
        pb.download()
        assert ctx.sync_status() == 0
        got = pb.outputs(0)
        for k in ("r_idx", "d1", "d2"):
            assert np.array_equal(got[k], st[k])
        assert np.all(got["xyz"].view(np.uint8) == 0x5a)
        if keep_depth:
            assert np.array_equal(got["fdepth"].view(np.uint32), st["fdepth"].view(np.uint32))
        else:
            assert np.all(got["fdepth"].view(np.uint8) == 0x5a)
    assert (st["fdepth"] > 0).sum() > 300


@pytest.mark.parametrize("overrides", [{"search_th": 2.0}, {"ratio_any_octave": 1}, {"kb_iters": 3, "min_depth": 2.0},
                                       {"th_stereo": 40, "th_search": 60}])
def test_parameter_variants(ctx, lib, overrides):
    frames = [scenes.single_pinhole(6), scenes.fisheye_frame(6)]
    pb = run_fused(ctx, frames, overrides, lib)
    for f in range(len(frames)):
        check_frame(pb, f, overrides, what=str(overrides))


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_randomized_batches(ctx, lib, seed):
    # seeded random ragged batches: pinhole images from 64x48 to 1280x720
    # (multiples of 16), 0-3000 left keypoints with 0-50 % distractors, 0-6000
    # map points, descriptor flip rates up to 15 %, a quarter fisheye frames
    # with 20-90 % overlap, and one parameter set per batch; every frame
    # equals the oracle's result for it alone
    rng = np.random.default_rng(900 + seed)
    frames = []
    for _ in range(10):
        if rng.random() < 0.25:
            frames.append(scenes.fisheye_frame(int(rng.integers(1 << 30)), n_left=int(rng.integers(0, 2500)),
                                               overlap_frac=float(rng.uniform(0.2, 0.9)),
                                               flip_p=float(rng.uniform(0, 0.15)), n_map=int(rng.integers(0, 6000))))
        else:
            W, H = int(rng.integers(4, 81)) * 16, int(rng.integers(3, 46)) * 16
            frames.append(scenes.pinhole_frame(int(rng.integers(1 << 30)), W=W, H=H,
                                               n_left=int(rng.integers(0, 3000)),
                                               distractor_frac=float(rng.uniform(0, 0.5)),
                                               flip_p=float(rng.uniform(0, 0.15)), n_map=int(rng.integers(0, 6000))))
    overrides = [{}, {"search_th": 2.0}, {"ratio_any_octave": 1}, {"th_stereo": 50, "th_search": 80}][seed]
    out = run_fused(ctx, frames, params=overrides, lib=lib)
    for f in range(len(frames)):
        check_frame(out, f, params=overrides, what=f"random batch {seed}")


def _shrink(fr, nl=None, nr=None, m=None):
    fr = dataclasses.replace(fr)
    def cut(k, n):
        return scenes.Keypoints(k.x[:n].copy(), k.y[:n].copy(), k.oct[:n].copy(), k.desc[:n].copy())
    if nl is not None:
        fr.left = cut(fr.left, nl)
        fr.taken_l = fr.taken_l[:nl].copy()
    if nr is not None:
        fr.right = cut(fr.right, nr)
        if fr.taken_r is not None:
            fr.taken_r = fr.taken_r[:nr].copy()
    if m is not None:
        fr.map = scenes.LocalMap(fr.map.pos[:m].copy(), fr.map.nrm[:m].copy(),
                                 fr.map.desc[:m].copy(), fr.map.skip[:m].copy())
    return fr


def test_empty_and_single_inputs(ctx, lib):
    p, q = scenes.single_pinhole(7), scenes.fisheye_frame(7)
    frames = [_shrink(p, nl=0), _shrink(p, nr=0), _shrink(p, m=0), _shrink(p, nl=1, nr=1, m=1),
              _shrink(q, nl=0), _shrink(q, nr=0), _shrink(q, m=0), _shrink(q, nl=1, nr=1, m=1)]
    pb = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(pb, f, what="edge")
    pb2 = run_per_frame(ctx, frames)
    assert np.array_equal(pb.host_out.numpy(), pb2.host_out.numpy())


def test_all_equal_descriptors_break_ties_by_index(ctx, lib):
    p, q = scenes.single_pinhole(8), scenes.fisheye_frame(8)
    for fr in (p, q):
        d = fr.left.desc[0].copy()
        fr.left.desc[:] = d
        fr.right.desc[:] = d
        fr.map.desc[:] = d
    pb = run_fused(ctx, [p, q])
    check_frame(pb, 0, what="ties")
    check_frame(pb, 1, what="ties")


def test_keypoints_on_image_borders(ctx, lib):
    fr = scenes.single_pinhole(9)
    W, H = fr.cam.width, fr.cam.height
    n = fr.left.n
    xs = np.array([0, W - 1, 0, W - 1, 5, W - 6, 0.5, W - 0.5], np.float32)
    ys = np.array([0, 0, H - 1, H - 1, 5, H - 6, H - 0.5, 0.49], np.float32)
    k = len(xs)
    fr.left.x[:k], fr.left.y[:k] = xs, ys
    fr.right.x[:k], fr.right.y[:k] = xs - 3, ys
    fr.right.desc[:k] = fr.left.desc[:k]
    fr.right.oct[:k] = fr.left.oct[:k]
    assert n > k
    pb = run_fused(ctx, [fr])
    check_frame(pb, 0, what="borders")


def test_keypoints_at_huge_coordinates_are_not_refined(ctx, lib):
    """Keypoints whose x is 3e9 or +inf (with right partners of the same
    descriptor at the same place) are matched by the Hamming step but have no
    SAD window inside the level images: their level coordinates saturate at
    INT_MAX on the device, and the window test must reject them rather than
    let the addition of the window half-widths wrap around.  They lie outside
    the search grid, so every other result is the oracle's on the frame
    without them."""
    fr = scenes.single_pinhole(19)
    st, se = orc.track_frame(_oracle_params(), fr)
    rng = np.random.default_rng(19)
    xs = np.array([3e9, np.inf, 3e9], np.float32)
    ys = np.array([100.0, 200.0, 300.0], np.float32)
    octs = np.array([0, 0, 3], np.int8)
    desc = scenes.random_desc(rng, len(xs))
    nl, nr = fr.left.n, fr.right.n
    big = dataclasses.replace(
        fr,
        left=scenes.Keypoints(x=np.concatenate([fr.left.x, xs]), y=np.concatenate([fr.left.y, ys]),
                              oct=np.concatenate([fr.left.oct, octs]), desc=np.concatenate([fr.left.desc, desc])),
        right=scenes.Keypoints(x=np.concatenate([fr.right.x, xs]), y=np.concatenate([fr.right.y, ys]),
                               oct=np.concatenate([fr.right.oct, octs]),
                               desc=np.concatenate([fr.right.desc, desc])),
        taken_l=np.concatenate([fr.taken_l, np.zeros(len(xs), np.uint8)]))
    pb = run_fused(ctx, [big])
    out = pb.outputs(0)
    base = {k: (v[:nl] if k in ("best_r", "dist", "sad_shift", "sad_best", "u_right", "depth", "kp_mp_l")
                else v) for k, v in out.items()}
    assert_stereo_equal(base, st, "huge coordinates (other keypoints): ")
    assert_search_equal(base, se, "l", None, "huge coordinates (map points): ")
    assert np.array_equal(out["best_r"][nl:], nr + np.arange(len(xs)))
    assert np.all(out["dist"][nl:] == 0)
    assert np.all(out["sad_shift"][nl:] == lib.FT_NO_SHIFT)
    assert np.all(out["sad_best"][nl:] == -1)
    assert np.all(out["u_right"][nl:] == -1.0) and np.all(out["depth"][nl:] == -1.0)
    assert np.all(out["kp_mp_l"][nl:] == -1)


def test_dense_rows_fall_back_to_scan(ctx, lib):
    # thousands of right keypoints on a few rows overflow the shared-memory stage
    fr = scenes.single_pinhole(10)
    rng = np.random.default_rng(10)
    m = fr.right.n
    fr.right.y[:] = np.float32(200.0) + rng.integers(0, 4, m).astype(np.float32)
    fr.left.y[: fr.left.n // 2] = np.float32(201.0)
    pb = run_fused(ctx, [fr])
    check_frame(pb, 0, what="dense rows")


# ---------------------------------------------------------------- launch shapes, graphs, host staging
@pytest.mark.parametrize("tune", [(1, 256, 512, 256, 1, 1), (7, 1024, 256, 512, 0, -1), (200, 512, 512, 4096, 1, -1),
                                  (32, 512, 128, 2048, 1, 1), (32, 256, 128, 2048, 0, 0)])
def test_tuning_variants_same_results(ctx, lib, tune):
    # strip heights, tiles, both search staging modes (records on chip or in
    # L2) and the search in two halves around the stereo step or in one pass
    from paper_2509_10757_gb300.batch import PackedBatch
    frames = [scenes.single_pinhole(11), scenes.fisheye_frame(11)]
    pb = PackedBatch(frames)
    t = lib.ft_tuning(strip_rows=tune[0], search_tile=tune[1], fisheye_tile=tune[2],
                      resolve_tile=tune[3], ctas_per_sm=1, search_stage=tune[4], split_search=tune[5])
    b = pb.batch()
    lib.check(lib.ft_set_tuning(ctx.ptr, C.byref(b), C.byref(t)), "ft_set_tuning")
    try:
        out = run_fused(ctx, frames)
    finally:
        d = lib.ft_tuning(strip_rows=32, search_tile=512, fisheye_tile=256, resolve_tile=2048,
                          ctas_per_sm=0)
        lib.ft_set_tuning(ctx.ptr, C.byref(b), C.byref(d))
    for f in range(len(frames)):
        check_frame(out, f, what=f"tuning {tune}")


def test_graph_replay_and_host_staging(lib):
    from paper_2509_10757_gb300.batch import Context
    frames = [scenes.single_pinhole(12), scenes.fisheye_frame(12), scenes.single_pinhole(13)]
    g = Context(arena_bytes=256 << 20, max_frames=16, use_graphs=True)
    try:
        a = run_fused(g, frames)
        b = run_fused(g, frames)                 # replay of the cached graph
        c = run_fused(g, frames, stage=True)     # host -> device -> host in the call
    finally:
        g.close()
    for f in range(len(frames)):
        check_frame(a, f, what="graph")
    assert np.array_equal(a.host_out.numpy(), b.host_out.numpy())
    assert np.array_equal(a.host_out.numpy(), c.host_out.numpy())


def test_autotune_and_table_roundtrip(ctx, lib, tmp_path):
    from paper_2509_10757_gb300.batch import PackedBatch, stream_handle
    frames = scenes.pinhole_batch(seed=1, n_frames=4)
    pb = PackedBatch(frames)
    pb.upload()
    best = lib.ft_tuning()
    b = pb.batch()
    lib.check(lib.ft_autotune(ctx.ptr, stream_handle(), None, C.byref(b), 1, C.byref(best)), "autotune")
    assert best.strip_rows in (16, 32, 64) and best.search_tile in (256, 512, 1024)
    path = str(tmp_path / "tuning.txt").encode()
    lib.check(lib.ft_save_tuning(ctx.ptr, path), "save")
    lib.check(lib.ft_load_tuning(ctx.ptr, path), "load")
    got = lib.ft_tuning()
    lib.check(lib.ft_get_tuning(ctx.ptr, C.byref(b), C.byref(got)), "get")
    assert (got.strip_rows, got.search_tile, got.fisheye_tile, got.search_stage, got.split_search) == \
        (best.strip_rows, best.search_tile, best.fisheye_tile, best.search_stage, best.split_search)
    assert best.split_search in (1, -1)
    out = run_fused(ctx, frames)
    for f in range(len(frames)):
        check_frame(out, f, what="tuned")


def test_autotune_stream_sets_every_context(ctx, lib):
    # the stream autotuner times candidates as launches taken in turn by
    # three contexts; each keeps the winner, results are the oracle's, and it
    # refuses a context given twice, fewer than two, or batches of different
    # buckets
    import torch as _t
    from paper_2509_10757_gb300.batch import Context, PackedBatch, autotune_stream, run_batch, stream_handle
    frames = scenes.pinhole_batch(seed=2, n_frames=4)
    pbs = [PackedBatch(frames) for _ in range(3)]
    for p in pbs:
        p.upload()
    extra = [Context(arena_bytes=1 << 28, max_frames=8) for _ in range(2)]
    ctxs = [ctx] + extra
    try:
        streams = [_t.cuda.Stream() for _ in range(3)]
        best = autotune_stream(ctxs, streams, pbs, iters=1)
        assert best.strip_rows in (16, 32, 64) and best.search_tile in (256, 512, 1024)
        assert 1 <= best.ctas_per_sm <= 3
        ba = pbs[0].batch()
        for c in ctxs:
            got = lib.ft_tuning()
            lib.check(lib.ft_get_tuning(c.ptr, C.byref(ba), C.byref(got)), "get")
            assert (got.strip_rows, got.search_tile, got.fisheye_tile, got.ctas_per_sm) == \
                (best.strip_rows, best.search_tile, best.fisheye_tile, best.ctas_per_sm)

        def call(cs, ps):
            n = len(cs)
            keep = [p.batch() for p in ps]
            return lib.ft_autotune_stream((C.c_void_p * n)(*[c.ptr for c in cs]),
                                          (C.c_void_p * n)(*[stream_handle(st).value for st in streams[:n]]), n,
                                          None, (C.POINTER(lib.ft_batch) * n)(*[C.pointer(b) for b in keep]), 1,
                                          None)
        assert call([ctx, ctx], pbs[:2]) == lib.FT_EINVAL
        assert call([ctx], pbs[:1]) == lib.FT_EINVAL
        other = PackedBatch(scenes.pinhole_batch(seed=3, n_frames=9))
        other.upload()
        assert call([ctx, extra[0]], [pbs[0], other]) == lib.FT_EINVAL
        _t.cuda.synchronize()
        for c, p in zip(ctxs, pbs):
            p.clear_outputs()
            run_batch(c, p)
            p.download()
            assert c.sync_status() == 0
            for f in range(len(frames)):
                check_frame(p, f, what="stream-tuned")
    finally:
        for c in extra:
            c.close()


def test_two_contexts_overlapping_launches(ctx, lib):
    # the headline form: two contexts on two streams launch alternately with
    # no synchronisation between them, so their persistent kernels overlap;
    # each context's results stay the oracle's
    import torch as _t
    from paper_2509_10757_gb300.batch import Context, PackedBatch, run_batch
    fa = scenes.pinhole_batch(seed=6, n_frames=6)
    fb = scenes.pinhole_batch(seed=7, n_frames=6)
    pa, pb2 = PackedBatch(fa), PackedBatch(fb)
    pa.upload()
    pb2.upload()
    pa.clear_outputs()
    pb2.clear_outputs()
    ctx2 = Context(arena_bytes=1 << 28, max_frames=8, use_graphs=True)
    try:
        s1, s2 = _t.cuda.Stream(), _t.cuda.Stream()
        for i in range(12):
            c, p, st = (ctx, pa, s1) if i % 2 == 0 else (ctx2, pb2, s2)
            with _t.cuda.stream(st):
                run_batch(c, p, stream=st)
        _t.cuda.synchronize()
        assert ctx.sync_status() == 0 and ctx2.sync_status() == 0
        for p, frames in ((pa, fa), (pb2, fb)):
            p.download()
            for f in range(len(frames)):
                check_frame(p, f, what="overlapped")
    finally:
        ctx2.close()


def test_measure_popcount(lib):
    # the popcount roofline's denominator: a plausible rate (between a tenth
    # and twice 16 popcounts per SM per clock at 2 GHz) and a refused NULL
    v = C.c_double(0.0)
    lib.check(lib.load().ft_measure_popcount(None, C.byref(v)), "ft_measure_popcount")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.1 * sms * 16 * 2e9 < v.value < 2.0 * sms * 16 * 2e9
    assert lib.load().ft_measure_popcount(None, None) == lib.FT_EINVAL


# ---------------------------------------------------------------- failures reported, never trapped
def test_bounded_wait_reports_timeout_and_context_recovers(lib):
    from paper_2509_10757_gb300.batch import Context
    frames = [scenes.single_pinhole(14)]
    c = Context(arena_bytes=128 << 20, max_frames=4)
    try:
        lib.check(lib.ft_set_debug(c.ptr, 1, 20_000_000), "debug")   # withhold stereo-ready, 20 ms bound
        from paper_2509_10757_gb300.batch import PackedBatch, run_batch
        pb = PackedBatch(frames)
        pb.upload()
        run_batch(c, pb)
        assert c.sync_status() == lib.FT_ETIMEOUT
        lib.check(lib.ft_set_debug(c.ptr, 0, 0), "debug")
        out = run_fused(c, frames)
        check_frame(out, 0, what="after timeout")
    finally:
        c.close()


def test_host_checks_reject_bad_arguments(ctx, lib):
    from paper_2509_10757_gb300.batch import PackedBatch, stream_handle
    fr = scenes.single_pinhole(15)
    pb = PackedBatch([fr])
    st, out = pb.stereo_frame(0), pb.stereo_out(0)
    from paper_2509_10757_gb300.batch import pinhole_struct
    cam = pinhole_struct(fr.cam)
    call = lambda: lib.ft_stereo_match_pinhole(ctx.ptr, stream_handle(), None, C.byref(cam),
                                               C.byref(st), C.byref(out))
    st.left.desc += 1
    assert call() == lib.FT_EALIGN
    st.left.desc -= 1
    st.left.n = -3
    assert call() == lib.FT_EINVAL
    st.left.n = fr.left.n
    out.depth = None
    assert call() == lib.FT_EINVAL
    out.depth = pb.pout(0, "depth")
    st.pyr_left.data[3] = None
    assert call() == lib.FT_EINVAL
    assert "level 3" in lib.last_error()
    st.pyr_left.data[3] = pb.pin_(0, "pyrL3")
    pitch = st.pyr_left.pitch[2]
    for bad in (pitch + 1, pitch + 4):               # rows must be 16-byte aligned
        st.pyr_left.pitch[2] = bad
        assert call() == lib.FT_EALIGN
    st.pyr_left.pitch[2] = pitch
    assert call() == lib.FT_OK
    assert ctx.sync_status() == 0
    # 8 frames of 4000 keypoints need about 1.9 MB of grid scratch; the
    # smallest arena leaves 1 MB
    big = scenes.pinhole_batch(seed=2, n_frames=8, nl_range=(4000, 4000), m_range=(100, 100))
    from paper_2509_10757_gb300.batch import Context
    small = Context(arena_bytes=1, max_frames=8)
    try:
        pbb = PackedBatch(big)
        b = pbb.batch()
        assert lib.ft_track_batch(small.ptr, stream_handle(), None, C.byref(b)) == lib.FT_ENOMEM
    finally:
        small.close()


# ---------------------------------------------------------------- search of the last frame (f2)
def _check_last(pb, f, st, what):
    fr, last = pb.frames[f], pb.lasts[f]
    ref = orc.search_last_frame(_oracle_params(), fr, last, st["u_right"] if fr.camera == "pinhole" else None)
    out = pb.outputs(f)
    got = {k[3:]: v for k, v in out.items() if k.startswith("lf_")}
    if fr.camera == "pinhole":
        assert_search_equal(got, ref, "l", None, what)
    else:
        assert_search_equal(got, ref, "l", "l", what)
        assert_search_equal(got, ref, "r", "r", what)
    return ref


@pytest.mark.parametrize("motion", ["forward", "backward", "none"])
def test_last_frame_search_per_call(ctx, lib, motion):
    from paper_2509_10757_gb300.batch import PackedBatch, run_search_last, run_stereo
    frames = [scenes.single_pinhole(30), scenes.fisheye_frame(31)]
    lasts = [scenes.last_frame(fr, 32 + i, motion) for i, fr in enumerate(frames)]
    pb = PackedBatch(frames, lasts=lasts)
    pb.upload()
    pb.clear_outputs()
    for f in range(len(frames)):
        run_stereo(ctx, pb, f)
        run_search_last(ctx, pb, f)
    pb.download()
    assert ctx.sync_status() == 0
    for f, fr in enumerate(frames):
        st = orc.stereo_frame(_oracle_params(), fr)
        ref = _check_last(pb, f, st, f"last-frame {motion} frame {f}: ")
        key = "mp_kp" if fr.camera == "pinhole" else "mp_kp_l"
        assert (ref[key] >= 0).sum() > 100


def test_last_frame_search_batched_with_local_map_frames(ctx, lib):
    # a batch mixing frames that search their local map with frames that
    # search their last frame's points (stereo first in both)
    frames = scenes.pinhole_batch(seed=3, n_frames=6) + [scenes.fisheye_frame(33), scenes.fisheye_frame(34)]
    motions = ["forward", None, "backward", "none", None, "forward", "backward", None]
    lasts = [None if mo is None else scenes.last_frame(fr, 40 + i, mo)
             for i, (fr, mo) in enumerate(zip(frames, motions))]
    from paper_2509_10757_gb300.batch import PackedBatch, run_batch
    pb = PackedBatch(frames, lasts=lasts)
    pb.upload()
    pb.clear_outputs()
    run_batch(ctx, pb)
    pb.download()
    assert ctx.sync_status() == 0
    for f, fr in enumerate(frames):
        st = orc.stereo_frame(_oracle_params(), fr)
        if fr.camera == "pinhole":
            assert_stereo_equal(pb.outputs(f), st, f"frame {f}: ")
        else:
            assert_fisheye_equal(pb.outputs(f), st, f"frame {f}: ")
        if lasts[f] is None:
            check_frame(pb, f, what="mixed batch")
        else:
            _check_last(pb, f, st, f"mixed batch frame {f}: ")


def test_last_frame_search_edge_cases(ctx, lib):
    from paper_2509_10757_gb300.batch import PackedBatch, run_search_last, run_stereo
    fr = scenes.single_pinhole(35)
    empty = scenes.last_frame(fr, 36, "none", n=0)
    bad = scenes.last_frame(fr, 37, "forward", n=50)
    bad.oct[:] = np.int8(-1)
    bad.oct[::7] = np.int8(8)
    for last in (empty, bad):
        pb = PackedBatch([fr], lasts=[last])
        pb.upload()
        pb.clear_outputs()
        run_stereo(ctx, pb, 0)
        run_search_last(ctx, pb, 0)
        pb.download()
        assert ctx.sync_status() == 0
        st = orc.stereo_frame(_oracle_params(), fr)
        ref = _check_last(pb, 0, st, "edge: ")
        assert np.all(ref["level"] == -1)


# ---------------------------------------------------------------- device-built pyramids (f3)
def _with_oracle_pyramids(fr):
    return dataclasses.replace(fr, pyr_left=orc.build_pyramid(fr.pyr_left[0]),
                               pyr_right=orc.build_pyramid(fr.pyr_right[0]))


def test_device_pyramids_in_the_batch(ctx, lib):
    # pinhole frames that upload only level 0 of their images: the launch
    # builds levels 1.. first; levels and results equal the oracle's on the
    # oracle-built pyramids (fisheye frames in the same batch are untouched)
    from paper_2509_10757_gb300.batch import PackedBatch, run_batch
    frames = scenes.pinhole_batch(seed=5, n_frames=5) + [scenes.fisheye_frame(50)]
    pb = PackedBatch(frames, device_pyramids=True)
    pb.upload()
    pb.clear_outputs()
    run_batch(ctx, pb)
    pb.download()
    assert ctx.sync_status() == 0
    for f, fr in enumerate(frames):
        if fr.camera != "pinhole":
            check_frame(pb, f, what="device pyramids")
            continue
        ref = _with_oracle_pyramids(fr)
        for side, levels in (("L", ref.pyr_left), ("R", ref.pyr_right)):
            for l in range(1, len(levels)):
                assert np.array_equal(pb.device_level(f, side, l), levels[l]), (f, side, l)
        out = pb.outputs(f)
        st, se = orc.track_frame(_oracle_params(), ref)
        assert_stereo_equal(out, st, f"device pyramids frame {f}: ")
        assert_search_equal(out, se, "l", None, f"device pyramids frame {f}: ")


def test_build_pyramid_per_call_and_size_check(ctx, lib):
    from paper_2509_10757_gb300.batch import PackedBatch, stream_handle
    fr = scenes.pinhole_frame(51, W=640, H=480, n_left=300, n_map=300)
    pb = PackedBatch([fr], device_pyramids=True)
    pb.upload()
    pyr = pb.pyramid(0, "R")
    lib.check(ctx.lib.ft_build_pyramid(ctx.ptr, stream_handle(), None, C.byref(pyr)), "ft_build_pyramid")
    torch.cuda.synchronize()
    ref = orc.build_pyramid(fr.pyr_right[0])
    for l in range(1, len(ref)):
        assert np.array_equal(pb.device_level(0, "R", l), ref[l]), l
    # the library's sizes are the oracle's
    w = (C.c_int * 8)()
    h = (C.c_int * 8)()
    lib.check(ctx.lib.ft_pyramid_sizes(640, 480, None, w, h), "ft_pyramid_sizes")
    assert (list(w), list(h)) == tuple(map(list, orc.pyramid_sizes(640, 480)))
    # a level of another size is refused before anything runs
    pyr.width[3] += 1
    assert ctx.lib.ft_build_pyramid(ctx.ptr, stream_handle(), None, C.byref(pyr)) == lib.FT_EINVAL


def test_build_pyramids_many_images_in_one_launch(ctx, lib):
    # five images of three sizes (an odd count: the last job builds one image)
    from paper_2509_10757_gb300.batch import PackedBatch, stream_handle
    frames = [scenes.pinhole_frame(52, W=640, H=480, n_left=200, n_map=100),
              scenes.pinhole_frame(53, W=752, H=480, n_left=200, n_map=100),
              scenes.pinhole_frame(54, W=320, H=240, n_left=200, n_map=100)]
    pb = PackedBatch(frames, device_pyramids=True)
    pb.upload()
    sides = [(0, "L"), (0, "R"), (1, "L"), (1, "R"), (2, "L")]
    arr = (lib.ft_pyramid * len(sides))(*[pb.pyramid(f, s) for f, s in sides])
    n0 = ctx.launches()
    lib.check(ctx.lib.ft_build_pyramids(ctx.ptr, stream_handle(), None, len(sides), arr), "ft_build_pyramids")
    torch.cuda.synchronize()
    assert ctx.launches() - n0 == 1
    for f, s in sides:
        fr = frames[f]
        ref = orc.build_pyramid((fr.pyr_left if s == "L" else fr.pyr_right)[0])
        for l in range(1, len(ref)):
            assert np.array_equal(pb.device_level(f, s, l), ref[l]), (f, s, l)


@pytest.mark.parametrize("W,H,nlevels,scale,seed", [(752, 480, 8, 1.2, 752), (333, 77, 8, 1.2, 1),
                                                     (6000, 37, 6, 1.3, 2), (17, 9, 3, 1.5, 3),
                                                     (641, 203, 5, 2.0, 4), (2, 3, 4, 1.2, 5),
                                                     (1000, 1000, 4, 3.5, 6), (753, 17, 8, 1.2, 7),
                                                     (1504, 33, 6, 1.5, 8)])
def test_build_pyramid_shapes_and_scales(ctx, lib, W, H, nlevels, scale, seed):
    # odd widths, flat and tiny images, a level wider than 4096 (several
    # column tiles of 752 source columns), level 0 one column and one row past
    # a whole number of tiles (a last tile of one source column and a last
    # slab of one source row) or exactly two tiles wide, and scale factors
    # from 1.2 to 3.5; level 0's row
    # padding holds junk the result must not depend on, levels 1.. start as
    # junk and must come out zero past their width.  The first image has a
    # pixel (level 5, row 9, column 225) whose value is an exact tie, 177.5,
    # only when both products are rounded before the sum: a fused
    # multiply-add there gives 177 instead of 178.
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    _check_built_pyramid(ctx, lib, img, nlevels, scale, rng)


def _check_built_pyramid(ctx, lib, img, nlevels, scale, rng):
    """Build levels 1.. of img's pyramid with ft_build_pyramid into buffers
    whose row padding (level 0) and contents (levels 1..) start as junk, and
    compare every level with the oracle's; bytes from a level's width to its
    width rounded up to 4 must come out zero."""
    from paper_2509_10757_gb300.batch import stream_handle
    ref = orc.build_pyramid(img, nlevels, scale)
    p = _params(lib, {"nlevels": nlevels, "scale_factor": scale})
    pyr = lib.ft_pyramid()
    pyr.nlevels = nlevels
    bufs = []
    for l, lev in enumerate(ref):
        h, w = lev.shape
        pitch = (w + 15) // 16 * 16
        host = rng.integers(0, 256, size=(h, pitch), dtype=np.uint8)
        if l == 0:
            host[:, :w] = lev
        t = torch.from_numpy(host.reshape(-1)).cuda()
        bufs.append(t)
        pyr.data[l] = t.data_ptr()
        pyr.width[l], pyr.height[l], pyr.pitch[l] = w, h, pitch
    lib.check(ctx.lib.ft_build_pyramid(ctx.ptr, stream_handle(), C.byref(p), C.byref(pyr)), "ft_build_pyramid")
    torch.cuda.synchronize()
    for l in range(1, nlevels):
        h, w = ref[l].shape
        got = bufs[l].cpu().numpy().reshape(h, -1)
        bad = np.argwhere(got[:, :w] != ref[l])
        assert len(bad) == 0, (img.shape, nlevels, scale, l, len(bad), bad[:4].tolist())
        w4 = (w + 3) // 4 * 4
        assert not got[:, w:w4].any(), l


def test_build_pyramid_random_shapes(ctx, lib):
    # seeded random image sizes (2-3000 x 2-600), scale factors (1.05-3.0)
    # and level counts (as many as keep every level at least one pixel, at
    # most 8), smooth and noisy content; every level equals the oracle's
    rng = np.random.default_rng(2024)
    for case in range(12):
        W, H = int(rng.integers(2, 3001)), int(rng.integers(2, 601))
        scale = float(np.float32(rng.uniform(1.05, 3.0)))
        nl = 1
        sc = np.float32(1.0)
        while nl < 8:
            nxt = np.float32(sc * np.float32(scale))
            if round(W / float(nxt)) < 1 or round(H / float(nxt)) < 1:
                break
            sc, nl = nxt, nl + 1
        if case % 2:
            img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
        else:
            yy, xx = np.mgrid[0:H, 0:W]
            img = (127.5 + 127.5 * np.sin(xx / 7.3 + rng.uniform(0, 6)) * np.cos(yy / 5.1)).astype(np.uint8)
        if nl >= 2:
            _check_built_pyramid(ctx, lib, img, nl, scale, rng)


def _split_search_rescans(fr, out, params):
    """Map points whose split search needs its second pass: more than four
    keypoints pass every test but the stereo consistency, and fewer than two
    of the four smallest (Hamming distance, index) keys among them are
    consistent.  Recomputed here in FP32 from the search's definition."""
    f32 = np.float32
    p = _oracle_params(params)
    sc = scenes.level_scales32(p["nlevels"], p["scale_factor"])
    cam = fr.cam
    iw = f32(64) / f32(f32(cam.max_x) - f32(cam.min_x))
    ih = f32(48) / f32(f32(cam.max_y) - f32(cam.min_y))
    kx, ky, ko = fr.left.x, fr.left.y, fr.left.oct.astype(np.int64)

    def rnd(v):                                        # roundf: half away from zero
        return np.sign(v) * np.floor(np.abs(v) + f32(0.5))

    gx = rnd((kx - f32(cam.min_x)).astype(f32) * iw)
    gy = rnd((ky - f32(cam.min_y)).astype(f32) * ih)
    in_grid = (gx >= 0) & (gx < 64) & (gy >= 0) & (gy < 48) & (fr.taken_l == 0)
    kbits = np.unpackbits(fr.left.desc, axis=1)
    ur_k = out["u_right"]
    proj, level = out["proj_l"], out["level_l"]
    n = 0
    for m in np.nonzero(level >= 0)[0]:
        lv = int(level[m])
        u, v, ur, vc = (f32(c) for c in proj[m])
        r = f32(p["radius_narrow"]) if vc > f32(p["view_cos_narrow"]) else f32(p["radius_wide"])
        r = f32(f32(r * f32(p["search_th"])) * sc[lv])
        cand = np.nonzero(in_grid & (ko >= lv - 1) & (ko <= lv) & (np.abs((kx - u).astype(f32)) < r) &
                          (np.abs((ky - v).astype(f32)) < r))[0]
        if len(cand) <= 4:
            continue
        d = (kbits[cand] != np.unpackbits(fr.map.desc[m])).sum(axis=1)
        top = cand[np.lexsort((cand, d))[:4]]
        w = ur_k[top]
        consistent = ~((w > 0) & (np.abs((f32(ur) - w).astype(f32)) > r))
        n += int(consistent.sum() < 2)
    return n


def test_split_search_second_pass_on_dense_windows(ctx, lib):
    # a pinhole frame whose stereo runs in the same launch splits its search:
    # the first half keeps each map point's four smallest candidates without
    # the stereo consistency, the second half applies it.  Dense keypoints and
    # a wide search radius give windows of many candidates whose stereo right
    # coordinates (other scene points' depths) mostly disagree with the map
    # point's: those points take the second, full pass.  The frame must equal
    # the oracle, and the second pass must have been needed.
    overrides = {"search_th": 3.0}
    fr = scenes.pinhole_frame(71, n_left=12000, n_map=3000, taken_frac=0.05)
    out = run_fused(ctx, [fr], params=overrides, lib=lib)
    check_frame(out, 0, params=overrides, what="dense windows")
    assert _split_search_rescans(fr, out.outputs(0), overrides) > 0
