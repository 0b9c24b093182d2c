"""ctypes front end of the plain CPU oracle (``ft_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the library never does.  It imports
nothing from the CUDA package: inputs are duck-typed objects (keypoints with
``x, y, oct, desc``; cameras, poses and maps with the documented fields) made
by the seeded scene generator.

Every function returns freshly allocated numpy arrays.  Steps and readings are
documented in ``ft_oracle.c`` (paper sections II-B, II-D, IV-C and IV-E).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libft_oracle.so")
# A prebuilt copy (for instance one with a planted mistake, used by the
# mutation test) can be loaded instead of the default build.
_OVERRIDE = os.environ.get("FT_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 16
NO_SHIFT = -128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, IEEE FP32)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ft_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(C.Structure):
    _fields_ = [
        ("nlevels", C.c_int), ("scale_factor", C.c_float),
        ("th_stereo", C.c_int), ("sad_w", C.c_int), ("sad_L", C.c_int),
        ("median_factor", C.c_float), ("fisheye_ratio", C.c_float),
        ("th_search", C.c_int), ("nn_ratio", C.c_float), ("ratio_any_octave", C.c_int),
        ("search_th", C.c_float), ("view_cos_min", C.c_float),
        ("view_cos_narrow", C.c_float), ("radius_narrow", C.c_float),
        ("radius_wide", C.c_float), ("dist_lo", C.c_float), ("dist_hi", C.c_float),
        ("th_last", C.c_float), ("kb_iters", C.c_int), ("min_depth", C.c_float),
        ("po_rounds", C.c_int), ("po_iters", C.c_int), ("po_chi2_mono", C.c_float),
        ("po_chi2_stereo", C.c_float), ("po_huber", C.c_int),
    ]


class OrcPinhole(C.Structure):
    _fields_ = [
        ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
        ("b", C.c_float), ("bf", C.c_float), ("width", C.c_int), ("height", C.c_int),
        ("min_x", C.c_float), ("max_x", C.c_float), ("min_y", C.c_float), ("max_y", C.c_float),
    ]


class OrcKB8(C.Structure):
    _fields_ = [
        ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
        ("k", C.c_float * 4), ("width", C.c_int), ("height", C.c_int),
        ("min_x", C.c_float), ("max_x", C.c_float), ("min_y", C.c_float), ("max_y", C.c_float),
    ]


class OrcPose(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("O", C.c_float * 3)]


class OrcPyramid(C.Structure):
    _fields_ = [
        ("nlevels", C.c_int),
        ("data", C.c_void_p * MAX_LEVELS),
        ("width", C.c_int * MAX_LEVELS), ("height", C.c_int * MAX_LEVELS),
        ("pitch", C.c_int * MAX_LEVELS),
    ]


class OrcKeypoints(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("x", C.c_void_p), ("y", C.c_void_p),
        ("oct", C.c_void_p), ("desc", C.c_void_p),
    ]


class OrcOrbParams(C.Structure):
    _fields_ = [("fast_th", C.c_int), ("edge", C.c_int), ("max_kp", C.c_int * MAX_LEVELS),
                ("pattern", C.c_void_p)]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            if _OVERRIDE:
                lib = C.CDLL(_OVERRIDE)
            else:
                build()
                lib = C.CDLL(_LIB_PATH)
            P = C.POINTER
            vp = C.c_void_p
            lib.orc_hamming.restype = C.c_int
            lib.orc_hamming.argtypes = [vp, vp]
            lib.orc_scale_table.argtypes = [C.c_int, C.c_float, vp, vp]
            lib.orc_atan2_pos.restype = C.c_float
            lib.orc_atan2_pos.argtypes = [C.c_float, C.c_float]
            lib.orc_row_index.restype = C.c_int
            lib.orc_row_index.argtypes = [C.c_int, vp, vp, vp, C.c_int, vp, vp, C.c_int]
            lib.orc_stereo_best.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcKeypoints),
                                            P(OrcKeypoints), vp, vp, vp, vp]
            lib.orc_sad_vector.restype = C.c_int
            lib.orc_sad_vector.argtypes = [P(OrcParams), P(OrcPyramid), P(OrcPyramid),
                                           C.c_int, C.c_int, C.c_int, C.c_int, vp]
            lib.orc_subpixel.restype = C.c_int
            lib.orc_subpixel.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                                         C.c_float, C.c_float, P(C.c_float), P(C.c_float),
                                         P(C.c_float)]
            lib.orc_median_reject.argtypes = [C.c_int, vp, C.c_float, vp, vp]
            lib.orc_stereo_pinhole.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcKeypoints),
                                               P(OrcKeypoints), P(OrcPyramid), P(OrcPyramid),
                                               vp, vp, vp, vp, vp, vp]
            lib.orc_stereo_fisheye.argtypes = [P(OrcParams), P(OrcKeypoints), P(OrcKeypoints),
                                               C.c_float, C.c_float, C.c_float, C.c_float,
                                               vp, vp, vp]
            lib.orc_sin_series.restype = C.c_float
            lib.orc_sin_series.argtypes = [C.c_float]
            lib.orc_cos_series.restype = C.c_float
            lib.orc_cos_series.argtypes = [C.c_float]
            lib.orc_unproject_kb8.restype = C.c_int
            lib.orc_unproject_kb8.argtypes = [P(OrcKB8), C.c_int, C.c_float, C.c_float, vp]
            lib.orc_triangulate.restype = C.c_int
            lib.orc_triangulate.argtypes = [vp, vp, vp, vp, C.c_float, vp]
            lib.orc_fisheye_triangulate.argtypes = [P(OrcParams), P(OrcKB8), P(OrcKB8), vp, vp,
                                                    P(OrcKeypoints), P(OrcKeypoints), vp, vp, vp]
            lib.orc_pyramid_sizes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, vp, vp]
            lib.orc_resample_level.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, C.c_int, C.c_int, C.c_int]
            lib.orc_motion.restype = C.c_int
            lib.orc_motion.argtypes = [P(OrcPose), P(OrcPose), C.c_float]
            lib.orc_search_last_camera.argtypes = [P(OrcParams), C.c_float, C.c_float, C.c_float,
                                                   C.c_float, P(OrcKeypoints), vp, vp, C.c_int, vp,
                                                   vp, vp, C.c_int, vp, vp, vp, vp]
            lib.orc_search_last_pinhole.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcPose), P(OrcPose),
                                                    P(OrcKeypoints), vp, vp, C.c_int, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp, vp]
            lib.orc_search_last_fisheye.argtypes = [P(OrcParams), P(OrcKB8), P(OrcKB8), vp, vp,
                                                    C.c_float, P(OrcPose), P(OrcPose), P(OrcKeypoints),
                                                    vp, P(OrcKeypoints), vp, C.c_int, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_grid_cell.restype = C.c_int
            lib.orc_grid_cell.argtypes = [C.c_float, C.c_float, C.c_float, C.c_float,
                                          C.c_float, C.c_float, P(C.c_int), P(C.c_int)]
            lib.orc_project_pinhole.restype = C.c_int
            lib.orc_project_pinhole.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcPose), vp, vp,
                                                C.c_float, C.c_float, vp, P(C.c_int)]
            lib.orc_project_kb8.restype = C.c_int
            lib.orc_project_kb8.argtypes = [P(OrcParams), P(OrcKB8), vp, vp, vp, vp, vp,
                                            C.c_float, C.c_float, vp, P(C.c_int)]
            lib.orc_search_camera.argtypes = [P(OrcParams), C.c_float, C.c_float, C.c_float,
                                              C.c_float, P(OrcKeypoints), vp, vp, C.c_int,
                                              vp, vp, vp, vp, vp, vp, vp]
            lib.orc_search_pinhole.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcPose),
                                               P(OrcKeypoints), vp, vp, C.c_int, vp, vp, vp,
                                               vp, vp, vp, vp, vp, vp, vp]
            lib.orc_search_fisheye.argtypes = [P(OrcParams), P(OrcKB8), P(OrcKB8), vp, vp,
                                               P(OrcPose), vp, P(OrcKeypoints), vp,
                                               P(OrcKeypoints), vp, C.c_int, vp, vp, vp, vp,
                                               vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_fast_score.restype = C.c_int
            lib.orc_fast_score.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
            lib.orc_smooth_level.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
            lib.orc_orientation.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
            lib.orc_describe.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp]
            lib.orc_extract_orb.restype = C.c_int
            lib.orc_extract_orb.argtypes = [P(OrcParams), P(OrcPyramid), P(OrcOrbParams), vp, vp, vp, vp, vp,
                                            vp, vp]
            lib.orc_se3_exp.argtypes = [vp, vp, vp]
            lib.orc_pose_residual.restype = C.c_int
            lib.orc_pose_residual.argtypes = [P(OrcPinhole), vp, vp, vp, vp, C.c_int, vp, vp]
            lib.orc_optimize_pose_pinhole.restype = C.c_int
            lib.orc_optimize_pose_pinhole.argtypes = [P(OrcParams), P(OrcPinhole), P(OrcPose),
                                                      P(OrcKeypoints), vp, C.c_int, vp, vp, vp, vp, vp,
                                                      vp, vp]
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def params_struct(p: dict) -> OrcParams:
    s = OrcParams()
    for name, _ in OrcParams._fields_:
        setattr(s, name, p[name])
    return s


def pinhole_struct(cam) -> OrcPinhole:
    s = OrcPinhole()
    for name, _ in OrcPinhole._fields_:
        setattr(s, name, getattr(cam, name))
    return s


def kb8_struct(cam) -> OrcKB8:
    s = OrcKB8()
    for name in ("fx", "fy", "cx", "cy", "width", "height", "min_x", "max_x", "min_y", "max_y"):
        setattr(s, name, getattr(cam, name))
    for i in range(4):
        s.k[i] = float(cam.k[i])
    return s


def pose_struct(pose) -> OrcPose:
    s = OrcPose()
    for i in range(9):
        s.R[i] = float(pose.R[i])
    for i in range(3):
        s.t[i] = float(pose.t[i])
        s.O[i] = float(pose.O[i])
    return s


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def add(self, a):
        self.refs.append(a)
        return a


def kps_struct(k, keep: _Keep) -> OrcKeypoints:
    s = OrcKeypoints()
    x = keep.add(_c(k.x, np.float32))
    y = keep.add(_c(k.y, np.float32))
    o = keep.add(_c(k.oct, np.int8))
    d = keep.add(_c(k.desc, np.uint8).reshape(-1, 32))
    s.n = len(x)
    s.x, s.y, s.oct, s.desc = _ptr(x), _ptr(y), _ptr(o), _ptr(d)
    return s


def pyramid_struct(levels, keep: _Keep) -> OrcPyramid:
    s = OrcPyramid()
    s.nlevels = len(levels)
    for l, img in enumerate(levels):
        img = keep.add(_c(img, np.uint8))
        s.data[l] = _ptr(img)
        s.height[l], s.width[l] = img.shape
        s.pitch[l] = img.strides[0]
    return s


# --------------------------------------------------------------------------
# public oracle functions
# --------------------------------------------------------------------------
def hamming(a: np.ndarray, b: np.ndarray) -> int:
    a = _c(a, np.uint8)
    b = _c(b, np.uint8)
    return _lib_handle().orc_hamming(_ptr(a), _ptr(b))


def scale_table(nlevels: int, s: float):
    sc = np.zeros(nlevels, np.float32)
    isc = np.zeros(nlevels, np.float32)
    _lib_handle().orc_scale_table(nlevels, s, _ptr(sc), _ptr(isc))
    return sc, isc


def atan2_pos(y: float, x: float) -> float:
    return float(np.float32(_lib_handle().orc_atan2_pos(y, x)))


def row_index(params: dict, yr, octr, H: int):
    """a1: CSR (row_ptr[H+1], row_idx) of the right keypoints' row bands."""
    lib = _lib_handle()
    sc, _ = scale_table(params["nlevels"], params["scale_factor"])
    y = _c(yr, np.float32)
    o = _c(octr, np.int8)
    row_ptr = np.zeros(H + 1, np.int32)
    cap = max(1, 64 * len(y))
    row_idx = np.zeros(cap, np.int32)
    n = lib.orc_row_index(len(y), _ptr(y), _ptr(o), _ptr(sc), H, _ptr(row_ptr), _ptr(row_idx), cap)
    assert n >= 0
    return row_ptr, row_idx[:n].copy()


def stereo_best(params: dict, cam, left, right):
    """a1 + a2: best right keypoint and its distance per left keypoint."""
    lib = _lib_handle()
    row_ptr, row_idx = row_index(params, right.y, right.oct, cam.height)
    keep = _Keep()
    L, R = kps_struct(left, keep), kps_struct(right, keep)
    n = L.n
    best_r = np.zeros(n, np.int32)
    dist = np.zeros(n, np.int32)
    p, c = params_struct(params), pinhole_struct(cam)
    lib.orc_stereo_best(C.byref(p), C.byref(c), C.byref(L), C.byref(R), _ptr(row_ptr),
                        _ptr(np.ascontiguousarray(row_idx) if len(row_idx) else np.zeros(1, np.int32)),
                        _ptr(best_r), _ptr(dist))
    return best_r, dist


def sad_vector(params: dict, pyr_left, pyr_right, level: int, ul: int, vl: int, ur0: int):
    """a3: the 2L+1 SAD values, or None if a window leaves the level image."""
    lib = _lib_handle()
    keep = _Keep()
    pl, pr = pyramid_struct(pyr_left, keep), pyramid_struct(pyr_right, keep)
    sad = np.zeros(2 * params["sad_L"] + 1, np.int32)
    p = params_struct(params)
    ok = lib.orc_sad_vector(C.byref(p), C.byref(pl), C.byref(pr), level, ul, vl, ur0, _ptr(sad))
    return sad if ok else None


def subpixel(sad, L: int, kbest: int, ur0: int, scale: float, xl: float, bf: float, disp_hi: float):
    """a4: (accepted, u_right, depth, delta) for a SAD vector with minimum at kbest."""
    s = _c(sad, np.int32)
    ur, dp, de = C.c_float(-1), C.c_float(-1), C.c_float(0)
    ok = _lib_handle().orc_subpixel(_ptr(s), L, kbest, ur0, scale, xl, bf, disp_hi, C.byref(ur),
                                    C.byref(dp), C.byref(de))
    return bool(ok), ur.value, dp.value, de.value


def median_reject(sad_best, u_right, depth, factor: float):
    """a5: copies of u_right, depth after median-based rejection."""
    sb = _c(sad_best, np.int32)
    ur = np.array(u_right, np.float32, copy=True)
    dp = np.array(depth, np.float32, copy=True)
    _lib_handle().orc_median_reject(len(sb), _ptr(sb), factor, _ptr(ur), _ptr(dp))
    return ur, dp


def stereo_pinhole(params: dict, cam, left, right, pyr_left, pyr_right) -> dict:
    """a1-a5 for one pinhole stereo frame."""
    lib = _lib_handle()
    keep = _Keep()
    L, R = kps_struct(left, keep), kps_struct(right, keep)
    pl, pr = pyramid_struct(pyr_left, keep), pyramid_struct(pyr_right, keep)
    n = L.n
    out = dict(
        best_r=np.zeros(n, np.int32), dist=np.zeros(n, np.int32),
        sad_shift=np.zeros(n, np.int32), sad_best=np.zeros(n, np.int32),
        u_right=np.zeros(n, np.float32), depth=np.zeros(n, np.float32),
    )
    p, c = params_struct(params), pinhole_struct(cam)
    lib.orc_stereo_pinhole(C.byref(p), C.byref(c), C.byref(L), C.byref(R), C.byref(pl),
                           C.byref(pr), *[_ptr(out[k]) for k in
                                          ("best_r", "dist", "sad_shift", "sad_best",
                                           "u_right", "depth")])
    return out


def stereo_fisheye(params: dict, rig, left, right) -> dict:
    """a6 for one fisheye stereo frame, then f1: the accepted matches
    triangulated (depth and left-camera point per left keypoint)."""
    lib = _lib_handle()
    keep = _Keep()
    L, R = kps_struct(left, keep), kps_struct(right, keep)
    n = L.n
    out = dict(r_idx=np.zeros(n, np.int32), d1=np.zeros(n, np.int32), d2=np.zeros(n, np.int32),
               fdepth=np.zeros(n, np.float32), xyz=np.zeros((n, 4), np.float32))
    p = params_struct(params)
    lib.orc_stereo_fisheye(C.byref(p), C.byref(L), C.byref(R), rig.lap_l0, rig.lap_l1,
                           rig.lap_r0, rig.lap_r1, _ptr(out["r_idx"]), _ptr(out["d1"]),
                           _ptr(out["d2"]))
    if rig.left is not None and rig.right is not None:   # matching-only rigs carry no cameras
        fisheye_triangulate(params, rig, left, right, out["r_idx"], out)
    return out


def unproject_kb8(cam, iters: int, u: float, v: float):
    """f1: (ok, ray) of a Kannala-Brandt pixel."""
    ray = np.zeros(3, np.float32)
    c = kb8_struct(cam)
    ok = _lib_handle().orc_unproject_kb8(C.byref(c), iters, u, v, _ptr(ray))
    return bool(ok), ray


def triangulate(ray_l, ray_r, R_rl, t_rl, min_depth: float):
    """f1: (ok, point in left-camera coordinates) of two rays."""
    arrs = [_c(a, np.float32) for a in (ray_l, ray_r, R_rl, t_rl)]
    P = np.zeros(3, np.float32)
    ok = _lib_handle().orc_triangulate(*[_ptr(a) for a in arrs], min_depth, _ptr(P))
    return bool(ok), P


def fisheye_triangulate(params: dict, rig, left, right, r_idx, out: dict | None = None) -> dict:
    """f1 for one frame's accepted fisheye matches."""
    lib = _lib_handle()
    keep = _Keep()
    L, R = kps_struct(left, keep), kps_struct(right, keep)
    n = L.n
    if out is None:
        out = dict(fdepth=np.zeros(n, np.float32), xyz=np.zeros((n, 4), np.float32))
    ridx = _c(r_idx, np.int32)
    Rrl, trl = _c(rig.R_rl, np.float32), _c(rig.t_rl, np.float32)
    p, cl, cr = params_struct(params), kb8_struct(rig.left), kb8_struct(rig.right)
    lib.orc_fisheye_triangulate(C.byref(p), C.byref(cl), C.byref(cr), _ptr(Rrl), _ptr(trl),
                                C.byref(L), C.byref(R), _ptr(ridx), _ptr(out["fdepth"]),
                                _ptr(out["xyz"]))
    return out


def sin_series(t: float) -> float:
    return float(_lib_handle().orc_sin_series(t))


def cos_series(t: float) -> float:
    return float(_lib_handle().orc_cos_series(t))


def grid_cell(x: float, y: float, min_x: float, max_x: float, min_y: float, max_y: float):
    cx, cy = C.c_int(), C.c_int()
    ok = _lib_handle().orc_grid_cell(x, y, min_x, max_x, min_y, max_y, C.byref(cx), C.byref(cy))
    return bool(ok), cx.value, cy.value


def project_pinhole(params: dict, cam, pose, P, n, dmin: float, dmax: float):
    """a8 for one point: (in_view, (u, v, u_right, view_cos), level)."""
    out = np.zeros(4, np.float32)
    lv = C.c_int(-1)
    Pw = _c(P, np.float32)
    nr = _c(n, np.float32)
    p, c, T = params_struct(params), pinhole_struct(cam), pose_struct(pose)
    ok = _lib_handle().orc_project_pinhole(C.byref(p), C.byref(c), C.byref(T), _ptr(Pw), _ptr(nr),
                                           dmin, dmax, _ptr(out), C.byref(lv))
    return bool(ok), out, lv.value


def project_kb8(params: dict, cam, R, t, O, P, n, dmin: float, dmax: float):
    out = np.zeros(4, np.float32)
    lv = C.c_int(-1)
    arrs = [_c(a, np.float32) for a in (R, t, O, P, n)]
    p, c = params_struct(params), kb8_struct(cam)
    ok = _lib_handle().orc_project_kb8(C.byref(p), C.byref(c), *[_ptr(a) for a in arrs],
                                       dmin, dmax, _ptr(out), C.byref(lv))
    return bool(ok), out, lv.value


def search_camera(params: dict, bounds, kps, u_right, taken, mp_desc, level, proj) -> dict:
    """a9 + a10 for one camera given the a8 results (level, proj)."""
    lib = _lib_handle()
    keep = _Keep()
    K = kps_struct(kps, keep)
    M = len(level)
    lv = keep.add(_c(level, np.int8))
    pj = keep.add(_c(proj, np.float32).reshape(-1, 4))
    md = keep.add(_c(mp_desc, np.uint8).reshape(-1, 32))
    ur = None if u_right is None else keep.add(_c(u_right, np.float32))
    tk = None if taken is None else keep.add(_c(taken, np.uint8))
    out = dict(mp_kp=np.zeros(M, np.int32), mp_d1=np.zeros(M, np.int32),
               mp_d2=np.zeros(M, np.int32), kp_mp=np.zeros(K.n, np.int32))
    p = params_struct(params)
    lib.orc_search_camera(C.byref(p), *[float(b) for b in bounds], C.byref(K), _ptr(ur), _ptr(tk),
                          M, _ptr(md), _ptr(lv), _ptr(pj), _ptr(out["mp_kp"]),
                          _ptr(out["mp_d1"]), _ptr(out["mp_d2"]), _ptr(out["kp_mp"]))
    return out


def search_pinhole(params: dict, cam, pose, kps, u_right, taken, lmap) -> dict:
    """a7-a10 for a pinhole frame (left keypoints only)."""
    lib = _lib_handle()
    keep = _Keep()
    K = kps_struct(kps, keep)
    M = len(lmap.pos)
    pos = keep.add(_c(lmap.pos, np.float32).reshape(-1, 4))
    nrm = keep.add(_c(lmap.nrm, np.float32).reshape(-1, 4))
    md = keep.add(_c(lmap.desc, np.uint8).reshape(-1, 32))
    sk = keep.add(_c(lmap.skip, np.uint8))
    ur = None if u_right is None else keep.add(_c(u_right, np.float32))
    tk = None if taken is None else keep.add(_c(taken, np.uint8))
    out = dict(level=np.zeros(M, np.int8), proj=np.zeros((M, 4), np.float32),
               mp_kp=np.zeros(M, np.int32), mp_d1=np.zeros(M, np.int32),
               mp_d2=np.zeros(M, np.int32), kp_mp=np.zeros(K.n, np.int32))
    p, c, T = params_struct(params), pinhole_struct(cam), pose_struct(pose)
    lib.orc_search_pinhole(C.byref(p), C.byref(c), C.byref(T), C.byref(K), _ptr(ur), _ptr(tk), M,
                           _ptr(pos), _ptr(nrm), _ptr(md), _ptr(sk), *[_ptr(out[k]) for k in
                                                                       ("level", "proj", "mp_kp",
                                                                        "mp_d1", "mp_d2",
                                                                        "kp_mp")])
    return out


def search_fisheye(params: dict, rig, pose, O_right, left, taken_l, right, taken_r, lmap) -> dict:
    """a7-a10 for a fisheye frame: left and right cameras, each with its grid."""
    lib = _lib_handle()
    keep = _Keep()
    KL, KR = kps_struct(left, keep), kps_struct(right, keep)
    M = len(lmap.pos)
    pos = keep.add(_c(lmap.pos, np.float32).reshape(-1, 4))
    nrm = keep.add(_c(lmap.nrm, np.float32).reshape(-1, 4))
    md = keep.add(_c(lmap.desc, np.uint8).reshape(-1, 32))
    sk = keep.add(_c(lmap.skip, np.uint8))
    tl = None if taken_l is None else keep.add(_c(taken_l, np.uint8))
    tr = None if taken_r is None else keep.add(_c(taken_r, np.uint8))
    Rrl = keep.add(_c(rig.R_rl, np.float32))
    trl = keep.add(_c(rig.t_rl, np.float32))
    Orr = keep.add(_c(O_right, np.float32))
    out = {}
    for side, n in (("l", KL.n), ("r", KR.n)):
        out[f"level_{side}"] = np.zeros(M, np.int8)
        out[f"proj_{side}"] = np.zeros((M, 4), np.float32)
        out[f"mp_kp_{side}"] = np.zeros(M, np.int32)
        out[f"mp_d1_{side}"] = np.zeros(M, np.int32)
        out[f"mp_d2_{side}"] = np.zeros(M, np.int32)
        out[f"kp_mp_{side}"] = np.zeros(n, np.int32)
    p, cl, cr, T = params_struct(params), kb8_struct(rig.left), kb8_struct(rig.right), pose_struct(pose)
    lib.orc_search_fisheye(C.byref(p), C.byref(cl), C.byref(cr), _ptr(Rrl), _ptr(trl), C.byref(T),
                           _ptr(Orr), C.byref(KL), _ptr(tl), C.byref(KR), _ptr(tr), M, _ptr(pos),
                           _ptr(nrm), _ptr(md), _ptr(sk),
                           *[_ptr(out[f"{k}_l"]) for k in ("level", "proj", "mp_kp", "mp_d1",
                                                            "mp_d2", "kp_mp")],
                           *[_ptr(out[f"{k}_r"]) for k in ("level", "proj", "mp_kp", "mp_d1",
                                                            "mp_d2", "kp_mp")])
    return out


def stereo_frame(params: dict, frame) -> dict:
    """Stereo step of one generated frame (pinhole a1-a5 or fisheye a6)."""
    if frame.camera == "pinhole":
        return stereo_pinhole(params, frame.cam, frame.left, frame.right, frame.pyr_left,
                              frame.pyr_right)
    return stereo_fisheye(params, frame.rig, frame.left, frame.right)


def search_frame(params: dict, frame, stereo: dict | None) -> dict:
    """Search step of one generated frame; pinhole frames use the stereo u_right."""
    if frame.camera == "pinhole":
        ur = stereo["u_right"] if stereo is not None else None
        return search_pinhole(params, frame.cam, frame.pose, frame.left, ur, frame.taken_l,
                              frame.map)
    return search_fisheye(params, frame.rig, frame.pose, frame.O_right, frame.left, frame.taken_l,
                          frame.right, frame.taken_r, frame.map)


def track_frame(params: dict, frame) -> tuple[dict, dict]:
    """Stereo then search for one frame, as the tracking thread runs them."""
    st = stereo_frame(params, frame)
    return st, search_frame(params, frame, st)


def motion(cur_pose, last_pose, b: float) -> int:
    """f2: +1 if the camera moved forward by more than b, -1 backward, else 0."""
    a, c = pose_struct(cur_pose), pose_struct(last_pose)
    return int(_lib_handle().orc_motion(C.byref(a), C.byref(c), b))


def search_last_frame(params: dict, frame, last, u_right=None) -> dict:
    """f2: the last frame's points searched in `frame` (pinhole: left camera
    with the stereo u_right; fisheye: both cameras).  Keys as search_frame."""
    lib = _lib_handle()
    keep = _Keep()
    M = last.n
    pos = keep.add(_c(last.pos, np.float32).reshape(-1, 4))
    md = keep.add(_c(last.desc, np.uint8).reshape(-1, 32))
    lo = keep.add(_c(last.oct, np.int8))
    sk = keep.add(_c(last.skip, np.uint8))
    p = params_struct(params)
    T, TL = pose_struct(frame.pose), pose_struct(last.pose)
    keys = ("level", "proj", "mp_kp", "mp_d1", "mp_d2", "kp_mp")

    def alloc(nk, sfx=""):
        return {f"level{sfx}": np.zeros(M, np.int8), f"proj{sfx}": np.zeros((M, 4), np.float32),
                f"mp_kp{sfx}": np.zeros(M, np.int32), f"mp_d1{sfx}": np.zeros(M, np.int32),
                f"mp_d2{sfx}": np.zeros(M, np.int32), f"kp_mp{sfx}": np.zeros(nk, np.int32)}

    if frame.camera == "pinhole":
        K = kps_struct(frame.left, keep)
        out = alloc(K.n)
        ur = None if u_right is None else keep.add(_c(u_right, np.float32))
        tk = None if frame.taken_l is None else keep.add(_c(frame.taken_l, np.uint8))
        c = pinhole_struct(frame.cam)
        lib.orc_search_last_pinhole(C.byref(p), C.byref(c), C.byref(T), C.byref(TL), C.byref(K), _ptr(ur),
                                    _ptr(tk), M, _ptr(pos), _ptr(md), _ptr(lo), _ptr(sk),
                                    *[_ptr(out[k]) for k in keys])
        return out
    rig = frame.rig
    KL, KR = kps_struct(frame.left, keep), kps_struct(frame.right, keep)
    out = {**alloc(KL.n, "_l"), **alloc(KR.n, "_r")}
    tl = None if frame.taken_l is None else keep.add(_c(frame.taken_l, np.uint8))
    tr = None if frame.taken_r is None else keep.add(_c(frame.taken_r, np.uint8))
    Rrl, trl = keep.add(_c(rig.R_rl, np.float32)), keep.add(_c(rig.t_rl, np.float32))
    cl, cr = kb8_struct(rig.left), kb8_struct(rig.right)
    lib.orc_search_last_fisheye(C.byref(p), C.byref(cl), C.byref(cr), _ptr(Rrl), _ptr(trl), rig.b,
                                C.byref(T), C.byref(TL), C.byref(KL), _ptr(tl), C.byref(KR), _ptr(tr), M,
                                _ptr(pos), _ptr(md), _ptr(lo), _ptr(sk),
                                *[_ptr(out[k + "_l"]) for k in keys], *[_ptr(out[k + "_r"]) for k in keys])
    return out


def search_last_camera(params: dict, bounds, kps, u_right, taken, desc, level, proj, motion_: int) -> dict:
    """f2 search of one camera from given projections (for hand-built cases)."""
    lib = _lib_handle()
    keep = _Keep()
    K = kps_struct(kps, keep)
    M = len(level)
    md = keep.add(_c(desc, np.uint8).reshape(-1, 32))
    lv = keep.add(_c(level, np.int8))
    pj = keep.add(_c(proj, np.float32).reshape(-1, 4))
    ur = None if u_right is None else keep.add(_c(u_right, np.float32))
    tk = None if taken is None else keep.add(_c(taken, np.uint8))
    out = dict(mp_kp=np.zeros(M, np.int32), mp_d1=np.zeros(M, np.int32), mp_d2=np.zeros(M, np.int32),
               kp_mp=np.zeros(K.n, np.int32))
    p = params_struct(params)
    lib.orc_search_last_camera(C.byref(p), *[float(b) for b in bounds], C.byref(K), _ptr(ur), _ptr(tk), M,
                               _ptr(md), _ptr(lv), _ptr(pj), motion_,
                               *[_ptr(out[k]) for k in ("mp_kp", "mp_d1", "mp_d2", "kp_mp")])
    return out


def pyramid_sizes(W: int, H: int, nlevels: int = 8, s: float = 1.2):
    """f3: (widths, heights) of the pyramid levels."""
    w = np.zeros(nlevels, np.int32)
    h = np.zeros(nlevels, np.int32)
    _lib_handle().orc_pyramid_sizes(W, H, nlevels, s, _ptr(w), _ptr(h))
    return [int(v) for v in w], [int(v) for v in h]


def resample_level(img, w: int, h: int) -> np.ndarray:
    """f3: one pyramid level from level 0."""
    src = _c(img, np.uint8)
    out = np.zeros((h, w), np.uint8)
    _lib_handle().orc_resample_level(_ptr(src), src.shape[1], src.shape[0], src.strides[0], _ptr(out), w, h, w)
    return out


def build_pyramid(img, nlevels: int = 8, s: float = 1.2) -> list:
    """f3: the pyramid of a level-0 image (level 0 itself first)."""
    ws, hs = pyramid_sizes(img.shape[1], img.shape[0], nlevels, s)
    return [np.ascontiguousarray(img, np.uint8)] + [resample_level(img, ws[l], hs[l]) for l in range(1, nlevels)]


# --------------------------------------------------------------------------
# f4: pose optimization (double precision)
# --------------------------------------------------------------------------
def se3_exp(d6):
    """exp of a twist d = (w, v): (R_d, V) as 3x3 arrays."""
    d = _c(d6, np.float64)
    R = np.zeros(9, np.float64)
    V = np.zeros(9, np.float64)
    _lib_handle().orc_se3_exp(_ptr(d), _ptr(R), _ptr(V))
    return R.reshape(3, 3), V.reshape(3, 3)


def pose_residual(cam, R, t, P, obs, stereo: bool):
    """(in front, residual e [3], Jacobian [3][6]) of one observation."""
    Rd = _c(np.asarray(R, np.float64).reshape(9), np.float64)
    td = _c(t, np.float64)
    Pw = _c(list(P) + [0.0] * (4 - len(P)), np.float32)
    ob = _c(list(obs) + [0.0] * (3 - len(obs)), np.float64)
    e = np.zeros(3, np.float64)
    J = np.zeros(18, np.float64)
    c = pinhole_struct(cam)
    ok = _lib_handle().orc_pose_residual(C.byref(c), _ptr(Rd), _ptr(td), _ptr(Pw), _ptr(ob), int(stereo),
                                         _ptr(e), _ptr(J))
    return bool(ok), e, J.reshape(3, 6)


def optimize_pose(params: dict, cam, pose, kps, u_right, pos, mp_kp) -> dict:
    """f4 for a pinhole frame: the refined pose (R, t, double), per map point
    inlier flags (1, 0, -1 unmatched) and final chi2, the number of inliers,
    the smallest relative distance of a classification's chi2 to its
    threshold, and the rounds run."""
    lib = _lib_handle()
    keep = _Keep()
    K = kps_struct(kps, keep)
    P = keep.add(_c(pos, np.float32).reshape(-1, 4))
    M = len(P)
    mk = keep.add(_c(mp_kp, np.int32))
    ur = None if u_right is None else keep.add(_c(u_right, np.float32))
    Rt = np.zeros(12, np.float64)
    inl = np.zeros(M, np.int8)
    c2 = np.zeros(M, np.float64)
    margin = C.c_double(0.0)
    rounds = C.c_int(0)
    p, c, T = params_struct(params), pinhole_struct(cam), pose_struct(pose)
    n = lib.orc_optimize_pose_pinhole(C.byref(p), C.byref(c), C.byref(T), C.byref(K), _ptr(ur), M, _ptr(P),
                                      _ptr(mk), _ptr(Rt), _ptr(inl), _ptr(c2), C.byref(margin), C.byref(rounds))
    return dict(R=Rt[:9].reshape(3, 3).copy(), t=Rt[9:].copy(), inlier=inl, chi2=c2, n_inliers=int(n),
                min_margin=margin.value, rounds=rounds.value)


# --------------------------------------------------------------------------
# f3: keypoint detection and description
# --------------------------------------------------------------------------
def fast_score(img, x: int, y: int, t: int) -> int:
    """FAST-9 score of pixel (x, y) (-1: not a corner at threshold t)."""
    a = _c(img, np.uint8)
    return int(_lib_handle().orc_fast_score(_ptr(a), a.strides[0], x, y, t))


def smooth_level(img) -> np.ndarray:
    a = _c(img, np.uint8)
    h, w = a.shape
    out = np.zeros((h, w), np.uint8)
    _lib_handle().orc_smooth_level(_ptr(a), w, h, a.strides[0], _ptr(out))
    return out


def orientation(img, x: int, y: int) -> np.ndarray:
    a = _c(img, np.uint8)
    cs = np.zeros(2, np.float32)
    _lib_handle().orc_orientation(_ptr(a), a.strides[0], x, y, _ptr(cs))
    return cs


def describe(smooth, x: int, y: int, cs, pattern) -> np.ndarray:
    a = _c(smooth, np.uint8)
    c = _c(cs, np.float32)
    pt = _c(pattern, np.int8).reshape(-1)
    d = np.zeros(32, np.uint8)
    _lib_handle().orc_describe(_ptr(a), a.strides[0], x, y, _ptr(c), _ptr(pt), _ptr(d))
    return d


def extract_orb(params: dict, levels, fast_th: int, edge: int, max_kp, pattern) -> dict:
    """f3 on one image pyramid: fixed slots per level (max_kp[l] each, in
    level order), padding after each level's keypoints."""
    keep = _Keep()
    pyr = pyramid_struct(levels, keep)
    op = OrcOrbParams()
    op.fast_th, op.edge = fast_th, edge
    for l, m in enumerate(max_kp):
        op.max_kp[l] = int(m)
    pt = keep.add(_c(pattern, np.int8).reshape(-1))
    op.pattern = _ptr(pt)
    n = int(sum(max_kp))
    out = dict(x=np.zeros(n, np.float32), y=np.zeros(n, np.float32), oct=np.zeros(n, np.int8),
               score=np.zeros(n, np.int32), cs=np.zeros((n, 2), np.float32), desc=np.zeros((n, 32), np.uint8),
               n_level=np.zeros(len(levels) + 1, np.int32))
    p = params_struct(params)
    _lib_handle().orc_extract_orb(C.byref(p), C.byref(pyr), C.byref(op), *[_ptr(out[k]) for k in
                                                                          ("x", "y", "oct", "score", "cs", "desc",
                                                                           "n_level")])
    return out
