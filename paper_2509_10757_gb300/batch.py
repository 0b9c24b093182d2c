"""Argument marshalling for libfasttrack.so: lay frames out in device memory
and build the C structs that point into it.

A PackedBatch puts every input of a list of frames into ONE contiguous blob
(pinned host copy + device copy) and every output into a second blob, each
array 256-byte aligned.  The C structs (ft_frame_job, ft_stereo_frame, ...)
hold device pointers into those blobs.  Nothing here computes any step of
the method: the work runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

ALIGN = 256


def _align(n: int) -> int:
    return (n + ALIGN - 1) // ALIGN * ALIGN


class _Layout:
    def __init__(self):
        self.items = []           # (key, offset, dtype, shape)
        self.index = {}
        self.size = 0

    def add(self, key, dtype, shape):
        nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
        off = self.size
        self.items.append((key, off, np.dtype(dtype), tuple(shape)))
        self.index[key] = len(self.items) - 1
        self.size = _align(off + max(nbytes, 1))
        return off


def _input_arrays(f, fr, last=None, device_pyramids=False):
    """(key, array) pairs of frame `f`'s inputs (and of its last frame's
    points); with device_pyramids only level 0 of each pyramid is an input."""
    out = [((f, "lx"), fr.left.x), ((f, "ly"), fr.left.y), ((f, "loct"), fr.left.oct),
           ((f, "ldesc"), fr.left.desc), ((f, "rx"), fr.right.x), ((f, "ry"), fr.right.y),
           ((f, "roct"), fr.right.oct), ((f, "rdesc"), fr.right.desc),
           ((f, "taken_l"), fr.taken_l)]
    if fr.camera == "pinhole":
        nl = 1 if device_pyramids else len(fr.pyr_left)
        for l, img in enumerate(fr.pyr_left[:nl]):
            out.append(((f, f"pyrL{l}"), pad_rows(img)))
        for l, img in enumerate(fr.pyr_right[:nl]):
            out.append(((f, f"pyrR{l}"), pad_rows(img)))
    else:
        out.append(((f, "taken_r"), fr.taken_r))
    out += [((f, "pos"), fr.map.pos), ((f, "nrm"), fr.map.nrm), ((f, "mdesc"), fr.map.desc),
            ((f, "skip"), fr.map.skip)]
    if last is not None:
        out += [((f, "lf_pos"), last.pos), ((f, "lf_desc"), last.desc), ((f, "lf_oct"), last.oct),
                ((f, "lf_skip"), last.skip)]
    return out


def _output_specs(f, fr, last=None, pose=False):
    nl, nr, m = fr.left.n, fr.right.n, fr.map.n
    spec = []
    if pose and fr.camera == "pinhole":
        npts = last.n if last is not None else m
        spec += [((f, "po_Rt"), np.float32, (12,)), ((f, "po_inlier"), np.int8, (npts,)),
                 ((f, "po_n"), np.int32, (1,))]
    if fr.camera == "pinhole":
        spec += [((f, k), np.int32, (nl,)) for k in ("best_r", "dist", "sad_shift", "sad_best")]
        spec += [((f, "u_right"), np.float32, (nl,)), ((f, "depth"), np.float32, (nl,))]
        sides = (("l", nl),)
    else:
        spec += [((f, k), np.int32, (nl,)) for k in ("r_idx", "d1", "d2")]
        spec += [((f, "fdepth"), np.float32, (nl,)), ((f, "xyz"), np.float32, (nl, 4))]
        sides = (("l", nl), ("r", nr))
    for s, nk in sides:
        spec += [((f, f"level_{s}"), np.int8, (m,)), ((f, f"proj_{s}"), np.float32, (m, 4))]
        spec += [((f, f"{k}_{s}"), np.int32, (m,)) for k in ("mp_kp", "mp_d1", "mp_d2")]
        spec += [((f, f"kp_mp_{s}"), np.int32, (nk,))]
    if last is not None:
        for s, nk in sides:
            spec += [((f, f"lf_level_{s}"), np.int8, (last.n,)), ((f, f"lf_proj_{s}"), np.float32, (last.n, 4))]
            spec += [((f, f"lf_{k}_{s}"), np.int32, (last.n,)) for k in ("mp_kp", "mp_d1", "mp_d2")]
            spec += [((f, f"lf_kp_mp_{s}"), np.int32, (nk,))]
    return spec


def pad_rows(img: np.ndarray, align: int = 16) -> np.ndarray:
    """Copy of a level image with its row pitch rounded up to `align` bytes
    (the library reads pyramid rows as 32-bit words)."""
    h, w = img.shape
    pitch = (w + align - 1) // align * align
    out = np.zeros((h, pitch), np.uint8)
    out[:, :w] = img
    return out


def _f32(a):
    return [float(v) for v in np.asarray(a, np.float32).reshape(-1)]


def pinhole_struct(cam) -> L.ft_pinhole:
    s = L.ft_pinhole()
    for name, _ in L.ft_pinhole._fields_:
        setattr(s, name, getattr(cam, name))
    return s


def kb8_struct(cam) -> L.ft_kb8:
    s = L.ft_kb8()
    for name in ("fx", "fy", "cx", "cy", "width", "height", "min_x", "max_x", "min_y", "max_y"):
        setattr(s, name, getattr(cam, name))
    s.k[:] = _f32(cam.k)
    return s


def rig_struct(rig) -> L.ft_fisheye_rig:
    s = L.ft_fisheye_rig()
    s.left = kb8_struct(rig.left)
    s.right = kb8_struct(rig.right)
    s.R_rl[:] = _f32(rig.R_rl)
    s.t_rl[:] = _f32(rig.t_rl)
    for name in ("b", "lap_l0", "lap_l1", "lap_r0", "lap_r1"):
        setattr(s, name, getattr(rig, name))
    return s


def pose_struct(pose) -> L.ft_pose:
    s = L.ft_pose()
    s.R[:] = _f32(pose.R)
    s.t[:] = _f32(pose.t)
    s.O[:] = _f32(pose.O)
    return s


class PackedBatch:
    """Inputs and outputs of a list of generated frames, packed for the GPU."""

    def __init__(self, frames, device: str | torch.device = "cuda", pin: bool = True, lasts=None,
                 device_pyramids: bool = False, pose: bool = False):
        """lasts: optional per-frame scenes.LastFrame (or None); a frame with
        one gets the last frame's points packed too, its batch job searches
        them instead of the local map, and its results go to the lf_* outputs.
        device_pyramids: pinhole frames carry only level 0 of their images;
        levels 1.. live in a device buffer the launch fills (ft_frame_job
        build_pyramids), with the sizes ft_pyramid_sizes gives.
        pose: pinhole frames get pose optimization outputs (po_Rt, po_inlier,
        po_n) and their batch jobs optimize the pose after the search."""
        self.frames = list(frames)
        self.lasts = list(lasts) if lasts is not None else [None] * len(self.frames)
        self.device_pyramids = device_pyramids
        self.device = torch.device(device)
        self.lin = _Layout()
        self.lout = _Layout()
        arrays = []
        for f, fr in enumerate(self.frames):
            for key, a in _input_arrays(f, fr, self.lasts[f], device_pyramids):
                a = np.ascontiguousarray(a)
                self.lin.add(key, a.dtype, a.shape)
                arrays.append(a)
            for key, dt, shape in _output_specs(f, fr, self.lasts[f], pose):
                self.lout.add(key, dt, shape)
        self.host_in = torch.empty(self.lin.size, dtype=torch.uint8, pin_memory=pin)
        self.host_out = torch.empty(self.lout.size, dtype=torch.uint8, pin_memory=pin)
        hin = self.host_in.numpy()
        for (key, off, dt, shape), a in zip(self.lin.items, arrays):
            hin[off:off + a.nbytes] = a.reshape(-1).view(np.uint8)
        self.dev_in = torch.empty(self.lin.size, dtype=torch.uint8, device=self.device)
        self.dev_out = torch.empty(self.lout.size, dtype=torch.uint8, device=self.device)
        self.in_base = self.dev_in.data_ptr()
        self.out_base = self.dev_out.data_ptr()
        # device-built pyramid levels 1.. (16-byte aligned rows)
        self.lpyr = _Layout()
        if device_pyramids:
            for f, fr in enumerate(self.frames):
                if fr.camera != "pinhole":
                    continue
                for side, levels in (("L", fr.pyr_left), ("R", fr.pyr_right)):
                    for l in range(1, len(levels)):
                        h, w = levels[l].shape
                        self.lpyr.add((f, f"pyr{side}{l}"), np.uint8, (h, (w + 15) // 16 * 16))
        self.dev_pyr = torch.empty(max(self.lpyr.size, 1), dtype=torch.uint8, device=self.device)
        self.last_views = [self.last_view(f) if self.lasts[f] is not None else None
                           for f in range(len(self.frames))]
        self.pose_outs = [self.pose_out(f) if self.has_out(f, "po_Rt") else None
                          for f in range(len(self.frames))]
        self.jobs = (L.ft_frame_job * max(1, len(self.frames)))()
        for f in range(len(self.frames)):
            self.jobs[f] = self.job(f)

    # ---------------------------------------------------------------- pointers
    def pin_(self, f, key):
        return self.in_base + self.lin.items[self.lin.index[(f, key)]][1]

    def pout(self, f, key):
        return self.out_base + self.lout.items[self.lout.index[(f, key)]][1]

    def has_out(self, f, key):
        return (f, key) in self.lout.index

    # ---------------------------------------------------------------- structs
    def keypoints(self, f, side: str) -> L.ft_keypoints:
        fr = self.frames[f]
        k = fr.left if side == "l" else fr.right
        s = L.ft_keypoints()
        s.n = k.n
        s.x, s.y = self.pin_(f, side + "x"), self.pin_(f, side + "y")
        s.oct, s.desc = self.pin_(f, side + "oct"), self.pin_(f, side + "desc")
        return s

    def pyramid(self, f, side: str) -> L.ft_pyramid:
        fr = self.frames[f]
        levels = fr.pyr_left if side == "L" else fr.pyr_right
        s = L.ft_pyramid()
        s.nlevels = len(levels)
        for l, img in enumerate(levels):
            key = (f, f"pyr{side}{l}")
            if l > 0 and self.device_pyramids:
                s.data[l] = self.dev_pyr.data_ptr() + self.lpyr.items[self.lpyr.index[key]][1]
            else:
                s.data[l] = self.pin_(f, f"pyr{side}{l}")
            s.height[l], s.width[l] = img.shape
            s.pitch[l] = pad_rows(img[:1]).shape[1]
        return s

    def device_level(self, f, side: str, l: int) -> np.ndarray:
        """A device-built level (levels >= 1 with device_pyramids) copied to the host."""
        key, off, dt, shape = self.lpyr.items[self.lpyr.index[(f, f"pyr{side}{l}")]]
        n = int(np.prod(shape))
        a = self.dev_pyr[off:off + n].cpu().numpy().reshape(shape)
        w = (self.frames[f].pyr_left if side == "L" else self.frames[f].pyr_right)[l].shape[1]
        return a[:, :w]

    def map_view(self, f) -> L.ft_map_view:
        s = L.ft_map_view()
        s.n = self.frames[f].map.n
        s.pos, s.nrm = self.pin_(f, "pos"), self.pin_(f, "nrm")
        s.desc, s.skip = self.pin_(f, "mdesc"), self.pin_(f, "skip")
        return s

    def stereo_out(self, f) -> L.ft_stereo_out:
        s = L.ft_stereo_out()
        for k in ("best_r", "dist", "sad_shift", "sad_best", "u_right", "depth"):
            setattr(s, k, self.pout(f, k))
        return s

    def fisheye_out(self, f) -> L.ft_fisheye_out:
        s = L.ft_fisheye_out()
        for k in ("r_idx", "d1", "d2"):
            setattr(s, k, self.pout(f, k))
        s.depth = self.pout(f, "fdepth")
        s.xyz = self.pout(f, "xyz")
        return s

    def search_out(self, f, prefix: str = "") -> L.ft_search_out:
        s = L.ft_search_out()
        for side, dst in (("l", s.left), ("r", s.right)):
            if self.has_out(f, f"{prefix}level_{side}"):
                for k in ("level", "proj", "mp_kp", "mp_d1", "mp_d2", "kp_mp"):
                    setattr(dst, k, self.pout(f, f"{prefix}{k}_{side}"))
        return s

    def pose_out(self, f) -> L.ft_pose_out:
        s = L.ft_pose_out()
        s.Rt, s.inlier, s.n_inliers = self.pout(f, "po_Rt"), self.pout(f, "po_inlier"), self.pout(f, "po_n")
        return s

    def last_view(self, f) -> L.ft_last_frame_view:
        last = self.lasts[f]
        s = L.ft_last_frame_view()
        s.n = last.n
        s.pos, s.desc = self.pin_(f, "lf_pos"), self.pin_(f, "lf_desc")
        s.oct, s.skip = self.pin_(f, "lf_oct"), self.pin_(f, "lf_skip")
        s.pose = pose_struct(last.pose)
        return s

    def frame_view(self, f, u_right: bool = True) -> L.ft_frame_view:
        fr = self.frames[f]
        s = L.ft_frame_view()
        s.left = self.keypoints(f, "l")
        s.right = self.keypoints(f, "r")
        s.taken_left = self.pin_(f, "taken_l")
        if fr.camera == "pinhole":
            s.camera = L.FT_CAMERA_PINHOLE
            s.pinhole = pinhole_struct(fr.cam)
            s.u_right = self.pout(f, "u_right") if u_right else None
        else:
            s.camera = L.FT_CAMERA_FISHEYE
            s.fisheye = rig_struct(fr.rig)
            s.taken_right = self.pin_(f, "taken_r")
            s.O_right[:] = _f32(fr.O_right)
        return s

    def stereo_frame(self, f) -> L.ft_stereo_frame:
        s = L.ft_stereo_frame()
        s.left, s.right = self.keypoints(f, "l"), self.keypoints(f, "r")
        s.pyr_left, s.pyr_right = self.pyramid(f, "L"), self.pyramid(f, "R")
        return s

    def job(self, f) -> L.ft_frame_job:
        fr = self.frames[f]
        j = L.ft_frame_job()
        j.left, j.right = self.keypoints(f, "l"), self.keypoints(f, "r")
        j.taken_left = self.pin_(f, "taken_l")
        j.pose = pose_struct(fr.pose)
        j.map = self.map_view(f)
        j.search = self.search_out(f)
        if self.last_views[f] is not None:
            j.last = C.pointer(self.last_views[f])
            j.search = self.search_out(f, "lf_")
        if fr.camera == "pinhole":
            j.camera = L.FT_CAMERA_PINHOLE
            j.pinhole = pinhole_struct(fr.cam)
            j.pyr_left, j.pyr_right = self.pyramid(f, "L"), self.pyramid(f, "R")
            j.stereo = self.stereo_out(f)
            j.build_pyramids = 1 if self.device_pyramids else 0
            if self.pose_outs[f] is not None:
                j.pose_out = C.pointer(self.pose_outs[f])
        else:
            j.camera = L.FT_CAMERA_FISHEYE
            j.fisheye = rig_struct(fr.rig)
            j.taken_right = self.pin_(f, "taken_r")
            j.O_right[:] = _f32(fr.O_right)
            j.fisheye_out = self.fisheye_out(f)
        return j

    def batch(self, stage: bool = False) -> L.ft_batch:
        b = L.ft_batch()
        b.n = len(self.frames)
        b.frames = C.cast(self.jobs, C.POINTER(L.ft_frame_job))
        if stage:
            b.stage_in_host = self.host_in.data_ptr()
            b.stage_in_dev = self.in_base
            b.stage_in_bytes = self.lin.size
            b.stage_out_dev = self.out_base
            b.stage_out_host = self.host_out.data_ptr()
            b.stage_out_bytes = self.lout.size
        return b

    # ---------------------------------------------------------------- data movement
    def upload(self):
        self.dev_in.copy_(self.host_in)

    def download(self):
        torch.cuda.synchronize(self.device)
        self.host_out.copy_(self.dev_out)

    def clear_outputs(self, value: int = 0x5a):
        self.dev_out.fill_(value)

    @property
    def in_bytes(self) -> int:
        return self.lin.size

    @property
    def out_bytes(self) -> int:
        return self.lout.size

    def outputs(self, f) -> dict:
        """numpy views of frame f's outputs in the pinned host copy."""
        h = self.host_out.numpy()
        out = {}
        for key, off, dt, shape in self.lout.items:
            if key[0] != f:
                continue
            n = int(np.prod(shape)) * dt.itemsize
            out[key[1]] = h[off:off + n].view(dt).reshape(shape)
        return out


class OrbOutputs:
    """Device outputs of ft_extract_orb for n images with the given slots per
    level (one blob), the ft_orb_out structs pointing into it, and the
    pattern and parameters of the call."""

    KEYS = (("x", np.float32, ()), ("y", np.float32, ()), ("oct", np.int8, ()), ("score", np.int32, ()),
            ("cs", np.float32, (2,)), ("desc", np.uint8, (32,)))

    def __init__(self, n_images: int, max_kp, pattern, fast_th: int = 20, edge: int = 19, nlevels: int = 8,
                 device: str | torch.device = "cuda"):
        self.n = n_images
        self.nslots = int(sum(max_kp))
        self.nlevels = nlevels
        self.lay = _Layout()
        for i in range(n_images):
            for k, dt, tail in self.KEYS:
                self.lay.add((i, k), dt, (self.nslots,) + tail)
            self.lay.add((i, "n_level"), np.int32, (nlevels + 1,))
        self.dev = torch.zeros(max(self.lay.size, 1), dtype=torch.uint8, device=device)
        self.base = self.dev.data_ptr()
        self.pattern = np.ascontiguousarray(pattern, np.int8).reshape(256, 4)
        self.params = L.ft_orb_params()
        self.params.fast_th, self.params.edge = fast_th, edge
        for l, m in enumerate(max_kp):
            self.params.max_kp[l] = int(m)
        self.params.pattern = self.pattern.ctypes.data
        self.outs = (L.ft_orb_out * max(1, n_images))()
        for i in range(n_images):
            o = self.outs[i]
            for k, _, _ in self.KEYS:
                setattr(o, k, self.ptr(i, k))
            o.n_level = self.ptr(i, "n_level")

    def ptr(self, i, key):
        return self.base + self.lay.items[self.lay.index[(i, key)]][1]

    def keypoints(self, i) -> L.ft_keypoints:
        """ft_keypoints view of image i's slots (device pointers)."""
        k = L.ft_keypoints()
        k.n = self.nslots
        k.x, k.y, k.oct, k.desc = self.ptr(i, "x"), self.ptr(i, "y"), self.ptr(i, "oct"), self.ptr(i, "desc")
        return k

    def download(self, i) -> dict:
        h = self.dev.cpu().numpy()
        out = {}
        for key, off, dt, shape in self.lay.items:
            if key[0] == i:
                n = int(np.prod(shape)) * dt.itemsize
                out[key[1]] = h[off:off + n].view(dt).reshape(shape)
        return out

    def download_all(self) -> list:
        h = self.dev.cpu().numpy()
        res = [dict() for _ in range(self.n)]
        for key, off, dt, shape in self.lay.items:
            n = int(np.prod(shape)) * dt.itemsize
            res[key[0]][key[1]] = h[off:off + n].view(dt).reshape(shape)
        return res


def run_extract(ctx: "Context", pyramids, oo: OrbOutputs, params: L.ft_params | None = None, stream=None):
    """ft_extract_orb on the ft_pyramid structs `pyramids` (device data)."""
    arr = (L.ft_pyramid * max(1, len(pyramids)))(*pyramids)
    L.check(ctx.lib.ft_extract_orb(ctx.ptr, stream_handle(stream), C.byref(params) if params is not None else None,
                                   len(pyramids), arr, C.byref(oo.params), oo.outs), "ft_extract_orb")


class Context:
    """Owns an ft_ctx (device arena, staging, graphs, tuning table)."""

    def __init__(self, device: int = 0, arena_bytes: int = 256 << 20, max_frames: int = 256,
                 use_graphs: bool = False):
        self.lib = L.load()
        d = L.ft_ctx_desc(device=device, arena_bytes=arena_bytes, max_frames=max_frames,
                          use_graphs=int(use_graphs))
        self.ptr = C.c_void_p()
        L.check(self.lib.ft_create(C.byref(self.ptr), C.byref(d)), "ft_create")

    def close(self):
        if self.ptr:
            self.lib.ft_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self) -> int:
        st = C.c_int32(-1)
        L.check(self.lib.ft_sync_status(self.ptr, C.byref(st)), "ft_sync_status")
        return st.value

    def launches(self) -> int:
        return int(self.lib.ft_launch_count(self.ptr))


def stream_handle(stream: torch.cuda.Stream | None = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def run_stereo(ctx: Context, pb: PackedBatch, f: int, params: L.ft_params | None = None, stream=None):
    """Per-frame stereo entry point (pinhole or fisheye) on frame f."""
    fr = pb.frames[f]
    p = C.byref(params) if params is not None else None
    if fr.camera == "pinhole":
        st = pb.stereo_frame(f)
        out = pb.stereo_out(f)
        cam = pinhole_struct(fr.cam)
        r = ctx.lib.ft_stereo_match_pinhole(ctx.ptr, stream_handle(stream), p, C.byref(cam),
                                            C.byref(st), C.byref(out))
        L.check(r, "ft_stereo_match_pinhole")
    else:
        rig = rig_struct(fr.rig)
        kl, kr = pb.keypoints(f, "l"), pb.keypoints(f, "r")
        out = pb.fisheye_out(f)
        r = ctx.lib.ft_stereo_match_fisheye(ctx.ptr, stream_handle(stream), p, C.byref(rig),
                                            C.byref(kl), C.byref(kr), C.byref(out))
        L.check(r, "ft_stereo_match_fisheye")


def run_search(ctx: Context, pb: PackedBatch, f: int, params: L.ft_params | None = None,
               stream=None, u_right: bool = True):
    """Per-frame search entry point on frame f (pinhole uses the stereo u_right)."""
    fv = pb.frame_view(f, u_right=u_right)
    pose = pose_struct(pb.frames[f].pose)
    mv = pb.map_view(f)
    out = pb.search_out(f)
    p = C.byref(params) if params is not None else None
    r = ctx.lib.ft_search_local_points(ctx.ptr, stream_handle(stream), p, C.byref(fv),
                                       C.byref(pose), C.byref(mv), C.byref(out))
    L.check(r, "ft_search_local_points")


def run_search_last(ctx: Context, pb: PackedBatch, f: int, params: L.ft_params | None = None,
                    stream=None, u_right: bool = True):
    """Per-frame search of the last frame's points (pb built with lasts)."""
    fv = pb.frame_view(f, u_right=u_right)
    pose = pose_struct(pb.frames[f].pose)
    lv = pb.last_views[f]
    out = pb.search_out(f, "lf_")
    p = C.byref(params) if params is not None else None
    r = ctx.lib.ft_search_last_frame(ctx.ptr, stream_handle(stream), p, C.byref(fv), C.byref(pose),
                                     C.byref(lv), C.byref(out))
    L.check(r, "ft_search_last_frame")


def run_pose(ctx: Context, pb: PackedBatch, f: int, params: L.ft_params | None = None, stream=None,
             u_right: bool = True):
    """ft_optimize_pose on frame f (pinhole): its local-map search matches
    (mp_kp_l) from the frame's starting pose, with its stereo u_right."""
    fr = pb.frames[f]
    fv = pb.frame_view(f, u_right=u_right)
    pose = pose_struct(fr.pose)
    mv = pb.map_view(f)
    out = pb.pose_outs[f]
    L.check(ctx.lib.ft_optimize_pose(ctx.ptr, stream_handle(stream), C.byref(params) if params is not None else None,
                                     C.byref(fv), C.byref(pose), C.byref(mv), C.c_void_p(pb.pout(f, "mp_kp_l")),
                                     C.byref(out)), "ft_optimize_pose")


def run_batch(ctx: Context, pb: PackedBatch, params: L.ft_params | None = None, stream=None,
              stage: bool = False):
    """Fused stereo + search over all frames of pb (one launch)."""
    b = pb.batch(stage=stage)
    p = C.byref(params) if params is not None else None
    L.check(ctx.lib.ft_track_batch(ctx.ptr, stream_handle(stream), p, C.byref(b)),
            "ft_track_batch")


def autotune_stream(ctxs, streams, pbs, iters: int = 3, params: L.ft_params | None = None) -> L.ft_tuning:
    """ft_autotune_stream over the contexts, streams and batches given in
    turn; returns the chosen launch shape (kept in every context)."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*[c.ptr for c in ctxs])
    ss = (C.c_void_p * n)(*[stream_handle(s).value for s in streams])
    keep = [pb.batch() for pb in pbs]
    bs = (C.POINTER(L.ft_batch) * n)(*[C.pointer(b) for b in keep])
    best = L.ft_tuning()
    p = C.byref(params) if params is not None else None
    L.check(ctxs[0].lib.ft_autotune_stream(cs, ss, n, p, bs, iters, C.byref(best)), "ft_autotune_stream")
    return best


# ---------------------------------------------------------------- served loop marshalling
def stream_desc_of(frame, slack: float = 1.0) -> L.ft_stream_desc:
    """Stream description for frames shaped like `frame` (capacities scaled by slack)."""
    d = L.ft_stream_desc()
    if frame.camera == "pinhole":
        d.camera = L.FT_CAMERA_PINHOLE
        d.pinhole = pinhole_struct(frame.cam)
        d.nlevels = len(frame.pyr_left)
        for l, img in enumerate(frame.pyr_left):
            d.level_height[l], d.level_width[l] = img.shape
    else:
        d.camera = L.FT_CAMERA_FISHEYE
        d.fisheye = rig_struct(frame.rig)
        d.nlevels = 8
    d.max_left = int(frame.left.n * slack)
    d.max_right = int(frame.right.n * slack)
    d.max_map = int(frame.map.n * slack)
    return d


class HostFrame:
    """Host arrays of one frame kept alive for ft_request / ft_server_set_* calls."""

    def __init__(self, frame):
        self.frame = frame
        c = np.ascontiguousarray
        self.lx, self.ly = c(frame.left.x, np.float32), c(frame.left.y, np.float32)
        self.lo, self.ld = c(frame.left.oct, np.int8), c(frame.left.desc, np.uint8)
        self.rx, self.ry = c(frame.right.x, np.float32), c(frame.right.y, np.float32)
        self.ro, self.rd = c(frame.right.oct, np.int8), c(frame.right.desc, np.uint8)
        self.tl = c(frame.taken_l, np.uint8)
        self.tr = c(frame.taken_r, np.uint8) if frame.taken_r is not None else None
        self.pos, self.nrm = c(frame.map.pos, np.float32), c(frame.map.nrm, np.float32)
        self.md, self.sk = c(frame.map.desc, np.uint8), c(frame.map.skip, np.uint8)
        self.pyr = None
        if frame.camera == "pinhole":
            self.pyr = [[c(x, np.uint8) for x in frame.pyr_left], [c(x, np.uint8) for x in frame.pyr_right]]

    def request(self, sid: int, tag: int, images: bool = False) -> L.ft_request:
        """The frame as a served request; images: it carries its level-0
        images (the server rebuilds the pyramid levels on the device)."""
        r = L.ft_request()
        r.stream_id, r.tag = sid, tag
        if images:
            a, b = self.pyr[0][0], self.pyr[1][0]
            r.image_left, r.image_right, r.image_pitch = a.ctypes.data, b.ctypes.data, a.strides[0]
        r.left = L.ft_keypoints(self.frame.left.n, self.lx.ctypes.data, self.ly.ctypes.data,
                                self.lo.ctypes.data, self.ld.ctypes.data)
        r.right = L.ft_keypoints(self.frame.right.n, self.rx.ctypes.data, self.ry.ctypes.data,
                                 self.ro.ctypes.data, self.rd.ctypes.data)
        r.taken_left = self.tl.ctypes.data
        r.taken_right = None if self.tr is None else self.tr.ctypes.data
        r.pose = pose_struct(self.frame.pose)
        if self.frame.O_right is not None:
            r.O_right[:] = _f32(self.frame.O_right)
        return r

    def map_view(self) -> L.ft_map_view:
        return L.ft_map_view(self.frame.map.n, self.pos.ctypes.data, self.nrm.ctypes.data,
                             self.md.ctypes.data, self.sk.ctypes.data)

    def pyramids(self):
        out = []
        for levels in self.pyr:
            p = L.ft_pyramid()
            p.nlevels = len(levels)
            for l, img in enumerate(levels):
                p.data[l] = img.ctypes.data
                p.height[l], p.width[l] = img.shape
                p.pitch[l] = img.shape[1]
            out.append(p)
        return out


def results_arrays(c: L.ft_completion, camera: str) -> dict:
    """numpy copies of a completion's host results."""
    r = c.results
    nl, nr, m = r.n_left, r.n_right, r.n_map

    def arr(ptr, n, ct, dt, shape=None):
        if n == 0 or not ptr:
            return np.zeros(shape or (n,), dt)
        a = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(n,)).copy()
        return a.reshape(shape) if shape else a

    out = {}
    if camera == "pinhole":
        s = r.stereo
        for k in ("best_r", "dist", "sad_shift", "sad_best"):
            out[k] = arr(getattr(s, k), nl, C.c_int32, np.int32)
        out["u_right"] = arr(s.u_right, nl, C.c_float, np.float32)
        out["depth"] = arr(s.depth, nl, C.c_float, np.float32)
        sides = (("l", r.search.left, nl),)
    else:
        for k in ("r_idx", "d1", "d2"):
            out[k] = arr(getattr(r.fisheye, k), nl, C.c_int32, np.int32)
        out["fdepth"] = arr(r.fisheye.depth, nl, C.c_float, np.float32)
        out["xyz"] = arr(r.fisheye.xyz, 4 * nl, C.c_float, np.float32, (nl, 4))
        sides = (("l", r.search.left, nl), ("r", r.search.right, nr))
    for sfx, o, nk in sides:
        out["level_" + sfx] = arr(o.level, m, C.c_int8, np.int8)
        out["proj_" + sfx] = arr(o.proj, 4 * m, C.c_float, np.float32, (m, 4))
        for k in ("mp_kp", "mp_d1", "mp_d2"):
            out[f"{k}_{sfx}"] = arr(getattr(o, k), m, C.c_int32, np.int32)
        out["kp_mp_" + sfx] = arr(o.kp_mp, nk, C.c_int32, np.int32)
    return out
