"""The allocation-free pinhole stereo entry point, through the C ABI.

ft_stereo_match_pinhole_noalloc serves callers that must not allocate device
memory while they run (a deadline-bound tracking loop, a process that
reserved all device memory up front, a host framework that forbids foreign
allocations): it needs no context and keeps its scratch in a fixed device
array inside the library.  Its results must equal those of
ft_stereo_match_pinhole and those of the CPU oracle, call after call (the
shared scratch keeps the previous call's contents, so a second call checks
that nothing stale leaks into the next result).  This file is collected
last so that a failure here never hides another test's result.
"""
import ctypes as C

import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes
from tests.gpu_common import assert_stereo_equal, stereo_view

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


def _noalloc(L, pb, f, status):
    from paper_2509_10757_gb300.batch import pinhole_struct, stream_handle
    cam = pinhole_struct(pb.frames[f].cam)
    st = pb.stereo_frame(f)
    out = pb.stereo_out(f)
    return L.load().ft_stereo_match_pinhole_noalloc(stream_handle(), None, C.byref(cam), C.byref(st),
                                                    C.byref(out), C.c_void_p(status.data_ptr()))


def test_noalloc_equals_context_entry_point_twice(lib):
    from paper_2509_10757_gb300.batch import Context, PackedBatch, run_stereo
    frames = [scenes.single_pinhole(21), scenes.pinhole_frame(22, W=640, H=480, n_left=2000)]
    pb = PackedBatch(frames)
    pb.upload()
    ctx = Context(arena_bytes=64 << 20, max_frames=4)
    try:
        pb.clear_outputs()
        for f in range(len(frames)):
            run_stereo(ctx, pb, f)
        pb.download()
        assert ctx.sync_status() == 0
        ref = [{k: v.copy() for k, v in stereo_view(pb.outputs(f)).items()} for f in range(len(frames))]
    finally:
        ctx.close()
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    oracle_ref = [orc.stereo_frame(dict(scenes.DEFAULT_PARAMS), fr) for fr in frames]
    for call in range(2):
        for f in range(len(frames)):
            pb.clear_outputs(0x3c + call)
            lib.check(_noalloc(lib, pb, f, status), "ft_stereo_match_pinhole_noalloc")
            pb.download()
            assert int(status.item()) == 0
            got = stereo_view(pb.outputs(f))
            assert_stereo_equal(got, ref[f], f"call {call} frame {f} (context entry point): ")
            assert_stereo_equal(got, oracle_ref[f], f"call {call} frame {f} (oracle): ")


def test_noalloc_calls_leave_device_memory_unchanged(lib):
    """After the first call on the device (which may load the library's
    module and so reserve the array), further calls take no device memory:
    the free-memory figure of the device is the same before and after them."""
    from paper_2509_10757_gb300.batch import PackedBatch
    pb = PackedBatch([scenes.single_pinhole(24)])
    pb.upload()
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    lib.check(_noalloc(lib, pb, 0, status), "ft_stereo_match_pinhole_noalloc")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lib.check(_noalloc(lib, pb, 0, status), "ft_stereo_match_pinhole_noalloc")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes over three calls"
    assert int(status.item()) == 0


def test_noalloc_rejects_frames_above_its_limit(lib):
    from paper_2509_10757_gb300.batch import PackedBatch, pinhole_struct, stream_handle
    pb = PackedBatch([scenes.single_pinhole(23)])
    cam = pinhole_struct(pb.frames[0].cam)
    st = pb.stereo_frame(0)
    out = pb.stereo_out(0)
    st.left.n = 16385
    r = lib.load().ft_stereo_match_pinhole_noalloc(stream_handle(), None, C.byref(cam), C.byref(st),
                                                   C.byref(out), None)
    assert r == lib.FT_EINVAL
    assert "allocation-free limit" in lib.last_error()
    st.left.n = pb.frames[0].left.n
    cam.height = 5000
    r = lib.load().ft_stereo_match_pinhole_noalloc(stream_handle(), None, C.byref(cam), C.byref(st),
                                                   C.byref(out), None)
    assert r == lib.FT_EINVAL
