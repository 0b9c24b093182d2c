"""ctypes binding of libfasttrack.so (include/fasttrack.h).

Names and structs mirror the C ABI one to one; this module only marshals
arguments.  There is no fallback: if the CUDA library was not built, loading
raises.  Build it with ``paper_2509_10757_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FT_LIB names another build of the library (for instance a variant compiled
# with different launch bounds); default: the in-tree build
LIB_PATH = os.environ.get("FT_LIB") or os.path.join(HERE, "libfasttrack.so")

FT_DESC_BYTES = 32
FT_MAX_LEVELS = 16
FT_GRID_COLS = 64
FT_GRID_ROWS = 48
FT_NO_SHIFT = -128
FT_CAMERA_PINHOLE = 0
FT_CAMERA_FISHEYE = 1
STATUS = {0: "FT_OK", 1: "FT_EINVAL", 2: "FT_EALIGN", 3: "FT_ENOMEM", 4: "FT_EBUSY",
          5: "FT_ECUDA", 6: "FT_ETIMEOUT"}
FT_OK, FT_EINVAL, FT_EALIGN, FT_ENOMEM, FT_EBUSY, FT_ECUDA, FT_ETIMEOUT = range(7)

vp = C.c_void_p
f32 = C.c_float
i32 = C.c_int


class ft_params(C.Structure):
    _fields_ = [("nlevels", i32), ("scale_factor", f32), ("th_stereo", i32),
                ("median_factor", f32), ("fisheye_ratio", f32), ("th_search", i32),
                ("nn_ratio", f32), ("ratio_any_octave", i32), ("search_th", f32),
                ("view_cos_min", f32), ("view_cos_narrow", f32), ("radius_narrow", f32),
                ("radius_wide", f32), ("dist_lo", f32), ("dist_hi", f32), ("th_last", f32), ("kb_iters", i32),
                ("min_depth", f32), ("po_rounds", i32), ("po_iters", i32), ("po_chi2_mono", f32),
                ("po_chi2_stereo", f32), ("po_huber", i32)]


class ft_keypoints(C.Structure):
    _fields_ = [("n", i32), ("x", vp), ("y", vp), ("oct", vp), ("desc", vp)]


class ft_pyramid(C.Structure):
    _fields_ = [("nlevels", i32), ("data", vp * FT_MAX_LEVELS), ("width", i32 * FT_MAX_LEVELS),
                ("height", i32 * FT_MAX_LEVELS), ("pitch", i32 * FT_MAX_LEVELS)]


class ft_pinhole(C.Structure):
    _fields_ = [("fx", f32), ("fy", f32), ("cx", f32), ("cy", f32), ("b", f32), ("bf", f32),
                ("width", i32), ("height", i32), ("min_x", f32), ("max_x", f32),
                ("min_y", f32), ("max_y", f32)]


class ft_kb8(C.Structure):
    _fields_ = [("fx", f32), ("fy", f32), ("cx", f32), ("cy", f32), ("k", f32 * 4),
                ("width", i32), ("height", i32), ("min_x", f32), ("max_x", f32),
                ("min_y", f32), ("max_y", f32)]


class ft_fisheye_rig(C.Structure):
    _fields_ = [("left", ft_kb8), ("right", ft_kb8), ("R_rl", f32 * 9), ("t_rl", f32 * 3),
                ("b", f32), ("lap_l0", f32), ("lap_l1", f32), ("lap_r0", f32), ("lap_r1", f32)]


class ft_pose(C.Structure):
    _fields_ = [("R", f32 * 9), ("t", f32 * 3), ("O", f32 * 3)]


class ft_map_view(C.Structure):
    _fields_ = [("n", i32), ("pos", vp), ("nrm", vp), ("desc", vp), ("skip", vp)]


class ft_stereo_frame(C.Structure):
    _fields_ = [("left", ft_keypoints), ("right", ft_keypoints), ("pyr_left", ft_pyramid),
                ("pyr_right", ft_pyramid)]


class ft_stereo_out(C.Structure):
    _fields_ = [("best_r", vp), ("dist", vp), ("sad_shift", vp), ("sad_best", vp),
                ("u_right", vp), ("depth", vp)]


class ft_fisheye_out(C.Structure):
    _fields_ = [("r_idx", vp), ("d1", vp), ("d2", vp), ("depth", vp), ("xyz", vp)]


class ft_search_cam_out(C.Structure):
    _fields_ = [("level", vp), ("proj", vp), ("mp_kp", vp), ("mp_d1", vp), ("mp_d2", vp),
                ("kp_mp", vp)]


class ft_search_out(C.Structure):
    _fields_ = [("left", ft_search_cam_out), ("right", ft_search_cam_out)]


class ft_frame_view(C.Structure):
    _fields_ = [("camera", i32), ("pinhole", ft_pinhole), ("fisheye", ft_fisheye_rig),
                ("left", ft_keypoints), ("right", ft_keypoints), ("u_right", vp),
                ("taken_left", vp), ("taken_right", vp), ("O_right", f32 * 3)]


class ft_last_frame_view(C.Structure):
    _fields_ = [("n", i32), ("pos", vp), ("desc", vp), ("oct", vp), ("skip", vp), ("pose", ft_pose)]


class ft_pose_out(C.Structure):
    _fields_ = [("Rt", vp), ("inlier", vp), ("n_inliers", vp)]


class ft_orb_params(C.Structure):
    _fields_ = [("fast_th", i32), ("edge", i32), ("max_kp", i32 * FT_MAX_LEVELS), ("pattern", vp)]


class ft_orb_out(C.Structure):
    _fields_ = [("x", vp), ("y", vp), ("oct", vp), ("score", vp), ("cs", vp), ("desc", vp), ("n_level", vp)]


class ft_frame_job(C.Structure):
    _fields_ = [("camera", i32), ("pinhole", ft_pinhole), ("fisheye", ft_fisheye_rig),
                ("left", ft_keypoints), ("right", ft_keypoints), ("pyr_left", ft_pyramid),
                ("pyr_right", ft_pyramid), ("taken_left", vp), ("taken_right", vp),
                ("pose", ft_pose), ("O_right", f32 * 3), ("map", ft_map_view),
                ("stereo", ft_stereo_out), ("fisheye_out", ft_fisheye_out),
                ("search", ft_search_out), ("last", C.POINTER(ft_last_frame_view)),
                ("build_pyramids", i32), ("pose_out", C.POINTER(ft_pose_out))]


class ft_batch(C.Structure):
    _fields_ = [("n", i32), ("frames", C.POINTER(ft_frame_job)), ("stage_in_host", vp),
                ("stage_in_dev", vp), ("stage_in_bytes", C.c_size_t), ("stage_out_dev", vp),
                ("stage_out_host", vp), ("stage_out_bytes", C.c_size_t)]


class ft_ctx_desc(C.Structure):
    _fields_ = [("device", i32), ("arena_bytes", C.c_size_t), ("max_frames", i32),
                ("use_graphs", i32)]


class ft_tuning(C.Structure):
    _fields_ = [("strip_rows", i32), ("search_tile", i32), ("fisheye_tile", i32),
                ("resolve_tile", i32), ("ctas_per_sm", i32), ("search_stage", i32), ("split_search", i32)]


class ft_trace_record(C.Structure):
    _fields_ = [("item", i32), ("kind", i32), ("frame", i32), ("sm", i32),
                ("t_start", C.c_uint64), ("t_end", C.c_uint64), ("wait_ns", C.c_uint64),
                ("mark", C.c_uint64 * 4)]


class ft_server_desc(C.Structure):
    _fields_ = [("device", i32), ("hbm_budget", C.c_size_t), ("n_slots", i32), ("max_batch", i32),
                ("slot_arena_bytes", C.c_size_t), ("dry_run", i32), ("dry_run_latency_us", C.c_double),
                ("queue_depth", i32)]


class ft_stream_desc(C.Structure):
    _fields_ = [("camera", i32), ("pinhole", ft_pinhole), ("fisheye", ft_fisheye_rig),
                ("nlevels", i32), ("level_width", i32 * FT_MAX_LEVELS),
                ("level_height", i32 * FT_MAX_LEVELS), ("max_left", i32), ("max_right", i32),
                ("max_map", i32)]


class ft_request(C.Structure):
    _fields_ = [("stream_id", i32), ("tag", C.c_uint64), ("left", ft_keypoints),
                ("right", ft_keypoints), ("taken_left", vp), ("taken_right", vp),
                ("pose", ft_pose), ("O_right", f32 * 3), ("image_left", vp), ("image_right", vp),
                ("image_pitch", i32)]


class ft_results(C.Structure):
    _fields_ = [("n_left", i32), ("n_right", i32), ("n_map", i32), ("stereo", ft_stereo_out),
                ("fisheye", ft_fisheye_out), ("search", ft_search_out)]


class ft_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("stream_id", i32), ("status", C.c_int32),
                ("t_submit_us", C.c_double), ("t_start_us", C.c_double), ("t_done_us", C.c_double),
                ("results", ft_results)]


class ft_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("frames_launched", C.c_uint64), ("streams_open", C.c_uint64),
                ("pending", C.c_uint64), ("pool_used", C.c_size_t), ("pool_capacity", C.c_size_t),
                ("last_error", C.c_int32)]


# (name, restype, argtypes): every entry point the header declares
SIGNATURES = [
    ("ft_params_default", None, [C.POINTER(ft_params)]),
    ("ft_last_error", C.c_char_p, []),
    ("ft_create", i32, [C.POINTER(vp), C.POINTER(ft_ctx_desc)]),
    ("ft_destroy", None, [vp]),
    ("ft_sync_status", i32, [vp, C.POINTER(C.c_int32)]),
    ("ft_stereo_match_pinhole", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_pinhole),
                                      C.POINTER(ft_stereo_frame), C.POINTER(ft_stereo_out)]),
    ("ft_stereo_match_fisheye", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_fisheye_rig),
                                      C.POINTER(ft_keypoints), C.POINTER(ft_keypoints),
                                      C.POINTER(ft_fisheye_out)]),
    ("ft_search_local_points", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_frame_view),
                                     C.POINTER(ft_pose), C.POINTER(ft_map_view),
                                     C.POINTER(ft_search_out)]),
    ("ft_search_last_frame", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_frame_view),
                                   C.POINTER(ft_pose), C.POINTER(ft_last_frame_view),
                                   C.POINTER(ft_search_out)]),
    ("ft_optimize_pose", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_frame_view), C.POINTER(ft_pose),
                               C.POINTER(ft_map_view), vp, C.POINTER(ft_pose_out)]),
    ("ft_extract_orb", i32, [vp, vp, C.POINTER(ft_params), i32, C.POINTER(ft_pyramid), C.POINTER(ft_orb_params),
                             C.POINTER(ft_orb_out)]),
    ("ft_pyramid_sizes", i32, [i32, i32, C.POINTER(ft_params), vp, vp]),
    ("ft_measure_popcount", i32, [vp, C.POINTER(C.c_double)]),
    ("ft_scattered_reads", i32, [vp, i32, i32, C.POINTER(i32)]),
    ("ft_build_pyramid", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_pyramid)]),
    ("ft_build_pyramids", i32, [vp, vp, C.POINTER(ft_params), i32, C.POINTER(ft_pyramid)]),
    ("ft_track_batch", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_batch)]),
    ("ft_autotune", i32, [vp, vp, C.POINTER(ft_params), C.POINTER(ft_batch), i32,
                          C.POINTER(ft_tuning)]),
    ("ft_autotune_stream", i32, [C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(ft_params),
                                 C.POINTER(C.POINTER(ft_batch)), i32, C.POINTER(ft_tuning)]),
    ("ft_set_tuning", i32, [vp, C.POINTER(ft_batch), C.POINTER(ft_tuning)]),
    ("ft_get_tuning", i32, [vp, C.POINTER(ft_batch), C.POINTER(ft_tuning)]),
    ("ft_save_tuning", i32, [vp, C.c_char_p]),
    ("ft_load_tuning", i32, [vp, C.c_char_p]),
    ("ft_set_debug", i32, [vp, C.c_uint, C.c_uint64]),
    ("ft_set_trace", i32, [vp, i32]),
    ("ft_read_trace", i32, [vp, C.POINTER(ft_trace_record), i32, C.POINTER(i32)]),
    ("ft_launch_count", C.c_uint64, [vp]),
    ("ft_server_desc_default", None, [C.POINTER(ft_server_desc)]),
    ("ft_server_create", i32, [C.POINTER(vp), C.POINTER(ft_server_desc), C.POINTER(ft_params)]),
    ("ft_server_destroy", None, [vp]),
    ("ft_server_open_stream", i32, [vp, C.POINTER(ft_stream_desc), C.POINTER(i32)]),
    ("ft_server_close_stream", i32, [vp, i32]),
    ("ft_server_set_pyramids", i32, [vp, i32, C.POINTER(ft_pyramid), C.POINTER(ft_pyramid)]),
    ("ft_server_set_map", i32, [vp, i32, C.POINTER(ft_map_view)]),
    ("ft_server_submit", i32, [vp, C.POINTER(ft_request)]),
    ("ft_server_poll", i32, [vp, C.POINTER(ft_completion), i32, i32]),
    ("ft_server_get_stats", i32, [vp, C.POINTER(ft_server_stats)]),
    ("ft_stereo_match_pinhole_noalloc", i32, [vp, C.POINTER(ft_params), C.POINTER(ft_pinhole),
                                              C.POINTER(ft_stereo_frame), C.POINTER(ft_stereo_out),
                                              vp]),
]

_lib = None


def load():
    """Load libfasttrack.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_2509_10757_gb300.build.build() (needs nvcc)")
        lib = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):
    # ft_* names resolve to the loaded C functions (same names as the C ABI)
    if name.startswith("ft_"):
        return getattr(load(), name)
    raise AttributeError(name)


def last_error() -> str:
    return load().ft_last_error().decode()


def check(status: int, what: str = ""):
    if status != FT_OK:
        raise RuntimeError(f"{what}: {STATUS.get(status, status)}: {last_error()}")


def default_params(overrides: dict | None = None) -> ft_params:
    p = ft_params()
    load().ft_params_default(C.byref(p))
    for k, v in (overrides or {}).items():
        setattr(p, k, v)
    return p
