"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, exports every entry point that include/fasttrack.h declares,
its ctypes mirror has the C struct sizes, and its default parameters are the
readings the oracle uses.  No compute call runs here."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fasttrack.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2509_10757_gb300 import build
    build.build()
    from paper_2509_10757_gb300 import _lib as L
    L.load()
    return L


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ft_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ft_create", "ft_destroy", "ft_last_error", "ft_stereo_match_pinhole",
              "ft_stereo_match_fisheye", "ft_search_local_points", "ft_track_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = lib.load()
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    bound = {name for name, _, _ in lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_ctypes_struct_sizes_match_c(lib):
    structs = ["ft_params", "ft_keypoints", "ft_pyramid", "ft_pinhole", "ft_kb8", "ft_fisheye_rig",
               "ft_pose", "ft_map_view", "ft_stereo_frame", "ft_stereo_out", "ft_fisheye_out",
               "ft_search_cam_out", "ft_search_out", "ft_pose_out", "ft_orb_params", "ft_orb_out", "ft_frame_view", "ft_last_frame_view", "ft_frame_job", "ft_batch",
               "ft_ctx_desc", "ft_tuning", "ft_trace_record", "ft_server_desc", "ft_stream_desc",
               "ft_request", "ft_results", "ft_completion", "ft_server_stats"]
    prog = "#include <stdio.h>\n#include \"fasttrack.h\"\nint main(void){\n"
    prog += "".join(f'printf("%zu\\n", sizeof({s}));\n' for s in structs) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "sz.c")
        exe = os.path.join(d, "sz")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    for s, n in zip(structs, sizes):
        assert C.sizeof(getattr(lib, s)) == n, s


def test_default_params_are_the_oracle_readings(lib):
    from paper_2509_10757_gb300.scenes import DEFAULT_PARAMS
    p = lib.default_params()
    for name, v in DEFAULT_PARAMS.items():
        if name in ("sad_w", "sad_L"):
            continue
        got = getattr(p, name)
        assert np.float32(got) == np.float32(v), name


def test_create_fails_cleanly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    st = lib.load().ft_create(C.byref(ctx), None)
    assert st in (lib.FT_ECUDA, lib.FT_EINVAL)
    assert not ctx.value
    assert lib.last_error()


def test_noalloc_checks_params_before_any_device_work(lib):
    """The allocation-free entry point applies the same parameter checks as
    the context entry points and returns before any CUDA call: a scale table
    whose top level overflows the band arithmetic (10^10) and a negative
    median factor are refused with FT_EINVAL, here on a machine without a GPU."""
    so = lib.load()
    cam, st, out = lib.ft_pinhole(), lib.ft_stereo_frame(), lib.ft_stereo_out()
    cam.width, cam.height, cam.b = 752, 480, 0.11
    bad = [dict(scale_factor=10.0, nlevels=11), dict(median_factor=-1.0), dict(nlevels=0)]
    for over in bad:
        p = lib.default_params(over)
        r = so.ft_stereo_match_pinhole_noalloc(None, C.byref(p), C.byref(cam), C.byref(st), C.byref(out), None)
        assert r == lib.FT_EINVAL, over
        assert lib.last_error(), over


def test_scattered_reads_checks_arguments_before_any_device_work(lib):
    """The memory diagnostic refuses a missing output, a stride below 256 or
    not a multiple of 4, and a second read outside the stride, before any
    CUDA call (here on a machine without a GPU)."""
    so = lib.load()
    acc = C.c_int(-1)
    assert so.ft_scattered_reads(None, 1024, 0, None) == lib.FT_EINVAL
    for stride, second in ((128, 0), (1022, 0), (1024, 1024), (1024, -4), (1024, 6)):
        assert so.ft_scattered_reads(None, stride, second, C.byref(acc)) == lib.FT_EINVAL, (stride, second)
        assert lib.last_error()
    assert acc.value == -1
