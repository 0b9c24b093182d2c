"""Seeded synthetic tracking inputs shaped like the paper's workloads.

The paper evaluates on EuRoC (752x480 pinhole stereo) and TUM-VI (512x512
fisheye stereo) in stereo-inertial mode (section V).  Neither dataset is
available here, so these generators stand in for them.  They build images,
pyramids, keypoints, descriptors, camera models, poses and local-map records
from a seed.  They contain no step of the matching method itself: no Hamming
search, no SAD, no projection test.  Both the CUDA library and the CPU oracle
take their inputs from here, and nothing else is shared between them.

Recipe (pinhole, 752x480 by default):
  * left image: white noise smoothed by a Gaussian (band-limited), scaled to
    mean 128 and std 45, clipped to uint8;
  * depth: 6 fronto-parallel planes at depths U[1, 10] m laid out as Voronoi
    cells of 6 random seeds; right image = left image shifted by each plane's
    disparity fx*b/Z with a z-buffer (nearest plane wins), linear
    interpolation in x, plus N(0, 2^2) noise;
  * pyramid: 8 levels, level l is (round(W/1.2^l), round(H/1.2^l)), each level
    bilinearly resampled from level 0;
  * left keypoints: octave l drawn with probability proportional to 1.2^-l,
    integer pixel (u, v) of level l, level-0 coordinates u*s_l, v*s_l (FP32);
  * right keypoints: the true correspondence of each left keypoint (same row,
    x shifted by the plane disparity and snapped to the level pixel grid)
    plus distractors (20% of the left count) at random pixels, shuffled;
  * descriptors: left uniform random 256 bits; right true = left with each
    bit flipped with probability 0.05; distractors random;
  * local map: points behind left keypoints (their plane depth, descriptor =
    left with flips) and random points in the frustum, each with dmax =
    distance * 1.2^level * U(0.9, 1.1), dmin = dmax / 1.2^7, a unit normal
    within 25 degrees of the viewing ray; a few points behind the camera,
    outside the image or facing away;
  * pose: the tracker's pose is the true pose perturbed by 2 cm and 0.5 deg.
Fisheye (512x512, Kannala-Brandt k1..k4 in +-0.01, baseline 0.10 m): 1500
left keypoints, 60% of them in the left/right overlap range with a true right
correspondence; the rest outside it; right distractors fill up to the left
count; local map of 6000 points.  Fisheye frames carry no images (the fisheye
path matches descriptors only).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DESC_BYTES = 32
NLEVELS = 8
SCALE = 1.2

# Constants of the method that the paper leaves unstated: the readings used by
# both the library defaults and the oracle (passed to each as input values).
DEFAULT_PARAMS = dict(
    nlevels=8,
    scale_factor=1.2,
    th_stereo=75,
    sad_w=5,
    sad_L=5,
    median_factor=float(np.float32(1.5) * np.float32(1.4)),
    fisheye_ratio=0.7,
    th_search=100,
    nn_ratio=0.8,
    ratio_any_octave=0,
    search_th=1.0,
    view_cos_min=0.5,
    view_cos_narrow=0.998,
    radius_narrow=2.5,
    radius_wide=4.0,
    dist_lo=0.8,
    dist_hi=1.2,
    th_last=7.0,
    kb_iters=10,
    min_depth=1e-4,
    po_rounds=4,
    po_iters=10,
    po_chi2_mono=5.991,
    po_chi2_stereo=7.815,
    po_huber=1,
)


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclass
class Keypoints:
    x: np.ndarray      # float32 [n], level-0 pixels
    y: np.ndarray      # float32 [n]
    oct: np.ndarray    # int8 [n]
    desc: np.ndarray   # uint8 [n, 32]

    @property
    def n(self) -> int:
        return int(len(self.x))


@dataclass
class PinholeCamera:
    fx: float
    fy: float
    cx: float
    cy: float
    b: float
    bf: float
    width: int
    height: int
    min_x: float
    max_x: float
    min_y: float
    max_y: float


@dataclass
class KB8Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    k: np.ndarray      # float32 [4]
    width: int
    height: int
    min_x: float
    max_x: float
    min_y: float
    max_y: float


@dataclass
class FisheyeRig:
    left: KB8Camera
    right: KB8Camera
    R_rl: np.ndarray   # float32 [9], right <- left rotation, row-major
    t_rl: np.ndarray   # float32 [3]
    b: float
    lap_l0: float
    lap_l1: float
    lap_r0: float
    lap_r1: float


@dataclass
class Pose:
    R: np.ndarray      # float32 [9], world -> camera, row-major
    t: np.ndarray      # float32 [3]
    O: np.ndarray      # float32 [3], camera centre in world


@dataclass
class LocalMap:
    pos: np.ndarray    # float32 [M, 4]: x, y, z, dmin
    nrm: np.ndarray    # float32 [M, 4]: nx, ny, nz, dmax
    desc: np.ndarray   # uint8 [M, 32]
    skip: np.ndarray   # uint8 [M]

    @property
    def n(self) -> int:
        return int(len(self.pos))


@dataclass
class LastFrame:
    """Points of the last frame to search in the current one: world position
    (x, y, z, unused), descriptor, the octave of the keypoint that observed
    the point in the last frame, a skip flag, and the last frame's pose."""
    pos: np.ndarray    # float32 [M, 4]
    desc: np.ndarray   # uint8 [M, 32]
    oct: np.ndarray    # int8 [M]
    skip: np.ndarray   # uint8 [M]
    pose: Pose

    @property
    def n(self) -> int:
        return int(len(self.pos))


@dataclass
class Frame:
    camera: str                       # "pinhole" or "fisheye"
    left: Keypoints
    right: Keypoints
    pose: Pose                        # pose the tracker projects with
    map: LocalMap
    taken_l: np.ndarray               # uint8 [NL]: keypoint already matched
    cam: PinholeCamera | None = None
    pyr_left: list | None = None
    pyr_right: list | None = None
    rig: FisheyeRig | None = None
    O_right: np.ndarray | None = None  # fisheye right camera centre (world)
    taken_r: np.ndarray | None = None
    pose_true: Pose | None = None
    truth: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# small helpers
# --------------------------------------------------------------------------
def level_scales32(nlevels: int = NLEVELS, s: float = SCALE) -> np.ndarray:
    """Level scales accumulated in FP32 (how keypoint coordinates are formed)."""
    sc = np.zeros(nlevels, np.float32)
    sc[0] = 1.0
    for l in range(1, nlevels):
        sc[l] = np.float32(sc[l - 1] * np.float32(s))
    return sc


def level_sizes(W: int, H: int, nlevels: int = NLEVELS, s: float = SCALE):
    return [(int(round(W / s ** l)), int(round(H / s ** l))) for l in range(nlevels)]


def octave_probs(nlevels: int = NLEVELS, s: float = SCALE) -> np.ndarray:
    w = (1.0 / s) ** np.arange(nlevels)
    return w / w.sum()


def gaussian_kernel(sigma: float) -> np.ndarray:
    r = int(np.ceil(3 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def band_limited_noise(rng: np.random.Generator, H: int, W: int, sigma: float = 1.5) -> np.ndarray:
    img = rng.standard_normal((H, W))
    k = gaussian_kernel(sigma)
    r = len(k) // 2
    p = np.pad(img, ((r, r), (r, r)), mode="reflect")
    tmp = sum(k[i] * p[:, i:i + W] for i in range(len(k)))
    out = sum(k[i] * tmp[i:i + H, :] for i in range(len(k)))
    out = (out - out.mean()) / (out.std() + 1e-12)
    return np.clip(np.rint(128.0 + 45.0 * out), 0, 255).astype(np.uint8)


def resample_bilinear(img: np.ndarray, w: int, h: int) -> np.ndarray:
    H, W = img.shape
    sx, sy = W / w, H / h
    xs = np.clip((np.arange(w) + 0.5) * sx - 0.5, 0, W - 1)
    ys = np.clip((np.arange(h) + 0.5) * sy - 0.5, 0, H - 1)
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    fx = (xs - x0)[None, :]
    fy = (ys - y0)[:, None]
    a = img.astype(np.float64)
    top = a[y0][:, x0] * (1 - fx) + a[y0][:, x1] * fx
    bot = a[y1][:, x0] * (1 - fx) + a[y1][:, x1] * fx
    return np.clip(np.rint(top * (1 - fy) + bot * fy), 0, 255).astype(np.uint8)


def build_pyramid(img: np.ndarray, nlevels: int = NLEVELS, s: float = SCALE) -> list:
    H, W = img.shape
    levels = [np.ascontiguousarray(img)]
    for l, (w, h) in enumerate(level_sizes(W, H, nlevels, s)[1:], start=1):
        levels.append(resample_bilinear(img, w, h))
    return levels


def random_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    ang = np.deg2rad(max_deg) * rng.uniform(0.0, 1.0)
    return axis_angle(axis, ang)


def axis_angle(axis: np.ndarray, ang: float) -> np.ndarray:
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)


def make_pose(R: np.ndarray, O: np.ndarray) -> Pose:
    t = -R @ O
    return Pose(R=R.astype(np.float32).reshape(9).copy(), t=t.astype(np.float32),
                O=O.astype(np.float32))


def perturb_pose(rng: np.random.Generator, R: np.ndarray, O: np.ndarray,
                 trans_m: float = 0.02, rot_deg: float = 0.5):
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    Rd = axis_angle(axis, np.deg2rad(rot_deg))
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    return Rd @ R, O + trans_m * d


def flip_bits(rng: np.random.Generator, desc: np.ndarray, p: float) -> np.ndarray:
    bits = np.unpackbits(desc, axis=-1)
    flips = (rng.random(bits.shape) < p).astype(np.uint8)
    return np.packbits(bits ^ flips, axis=-1)


def random_desc(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(0, 256, size=(n, DESC_BYTES), dtype=np.uint8)


def sample_octaves(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.choice(NLEVELS, size=n, p=octave_probs()).astype(np.int8)


def tilted_normals(rng: np.random.Generator, view: np.ndarray, max_deg: float) -> np.ndarray:
    """Unit vectors within max_deg of the unit vectors `view` (rotation about a
    random axis perpendicular to each)."""
    a = np.cross(view, rng.standard_normal(view.shape))
    a /= np.linalg.norm(a, axis=1, keepdims=True) + 1e-12
    th = np.deg2rad(max_deg) * rng.uniform(size=(len(view), 1))
    out = view * np.cos(th) + np.cross(a, view) * np.sin(th)
    return out / np.linalg.norm(out, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# pinhole stereo
# --------------------------------------------------------------------------
def pinhole_camera(W: int = 752, H: int = 480, fx: float | None = None, b: float = 0.11) -> PinholeCamera:
    if fx is None:
        fx = 435.0 * W / 752.0
    fx32 = np.float32(fx)
    b32 = np.float32(b)
    return PinholeCamera(fx=float(fx32), fy=float(fx32), cx=float(np.float32(W / 2)),
                         cy=float(np.float32(H / 2)), b=float(b32), bf=float(np.float32(fx32 * b32)),
                         width=W, height=H, min_x=0.0, max_x=float(W), min_y=0.0, max_y=float(H))


@dataclass
class _StereoImages:
    left: np.ndarray
    right: np.ndarray
    label: np.ndarray     # plane index per left pixel
    depth: np.ndarray     # plane depths [6]
    pyr_left: list
    pyr_right: list


def stereo_images(seed: int, cam: PinholeCamera, n_planes: int = 6, noise_sigma: float = 2.0) -> _StereoImages:
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    left = band_limited_noise(rng, H, W)
    seeds = rng.uniform([0, 0], [W, H], size=(n_planes, 2))
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = [(xx - sx) ** 2 + (yy - sy) ** 2 for sx, sy in seeds]
    label = np.argmin(np.stack(d2), axis=0).astype(np.int8)
    depth = rng.uniform(1.0, 10.0, size=n_planes)
    disp = cam.fx * cam.b / depth
    # right pixel xr shows the nearest plane i whose left region contains xr + d_i
    best_z = np.full((H, W), np.inf)
    src_x = np.full((H, W), np.nan)
    for i in range(n_planes):
        xl = xx + disp[i]
        xi = np.rint(xl).astype(np.int64)
        ok = (xi >= 0) & (xi < W)
        lab = np.full((H, W), -1, np.int64)
        lab[ok] = label[yy[ok], xi[ok]]
        vis = ok & (lab == i) & (depth[i] < best_z)
        best_z[vis] = depth[i]
        src_x[vis] = xl[vis]
    right = rng.integers(0, 256, size=(H, W)).astype(np.float64)
    have = ~np.isnan(src_x)
    xs = np.clip(src_x[have], 0, W - 1)
    x0 = np.floor(xs).astype(np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    f = xs - x0
    rows = yy[have]
    lf = left.astype(np.float64)
    right[have] = lf[rows, x0] * (1 - f) + lf[rows, x1] * f
    right += rng.normal(0.0, noise_sigma, size=(H, W))
    right = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return _StereoImages(left=left, right=right, label=label, depth=depth,
                         pyr_left=build_pyramid(left), pyr_right=build_pyramid(right))


def _level_pixel_keypoints(rng, n, W, H, sc32, octs=None):
    octs = sample_octaves(rng, n) if octs is None else octs
    sizes = level_sizes(W, H)
    x = np.empty(n, np.float32)
    y = np.empty(n, np.float32)
    for i, l in enumerate(octs):
        w, h = sizes[l]
        u = rng.integers(0, w)
        v = rng.integers(0, h)
        x[i] = np.float32(np.float32(u) * sc32[l])
        y[i] = np.float32(np.float32(v) * sc32[l])
    return x, y, octs


def _local_map(rng, n_map, cam_proj, cam_unproj, W, H, Rt, Ot, kp_x, kp_y, kp_oct, kp_desc,
               kp_depth, flip_p, frac_assoc=0.6):
    """Map points: some behind keypoints, the rest random in the frustum."""
    sc64 = SCALE ** np.arange(NLEVELS)
    n_assoc = min(int(frac_assoc * n_map), len(kp_x))
    pick = rng.choice(len(kp_x), size=n_assoc, replace=False) if n_assoc else np.zeros(0, np.int64)
    n_rand = n_map - n_assoc
    u = np.concatenate([kp_x[pick].astype(np.float64), rng.uniform(0, W, n_rand)])
    v = np.concatenate([kp_y[pick].astype(np.float64), rng.uniform(0, H, n_rand)])
    z = np.concatenate([kp_depth[pick], rng.uniform(1.0, 10.0, n_rand)])
    lev = np.concatenate([kp_oct[pick].astype(np.int64), rng.choice(NLEVELS, n_rand, p=octave_probs())])
    desc = np.concatenate([flip_bits(rng, kp_desc[pick], flip_p), random_desc(rng, n_rand)])
    Pc = cam_unproj(u, v, z)
    Pw = (Pc - (-Rt @ Ot)[None, :]) @ Rt        # R^T (Pc - t)
    # a few points behind the camera or outside the image
    m = len(Pw)
    bad = rng.random(m)
    behind = bad < 0.03
    Pw[behind] = Ot + (Ot - Pw[behind])          # mirrored through the camera centre
    outside = (bad >= 0.03) & (bad < 0.06)
    Pw[outside] = Pw[outside] + (Rt.T @ np.array([3.0, 0.0, 0.0]))[None, :] * z[outside, None]
    view = Pw - Ot
    dist = np.linalg.norm(view, axis=1)
    view_u = view / dist[:, None]
    nrm = tilted_normals(rng, view_u, 25.0)      # mean viewing direction (camera -> point)
    away = rng.random(m) < 0.04
    nrm[away] = -nrm[away]
    dmax = dist * sc64[lev] * rng.uniform(0.9, 1.1, m)
    dmin = dmax / sc64[NLEVELS - 1]
    pos = np.concatenate([Pw, dmin[:, None]], axis=1).astype(np.float32)
    nr = np.concatenate([nrm, dmax[:, None]], axis=1).astype(np.float32)
    skip = (rng.random(m) < 0.05).astype(np.uint8)
    return LocalMap(pos=pos, nrm=nr, desc=desc.astype(np.uint8), skip=skip), pick


def pinhole_frame(seed: int, W: int = 752, H: int = 480, n_left: int = 1200,
                  distractor_frac: float = 0.2, flip_p: float = 0.05, n_map: int = 3000,
                  images: _StereoImages | None = None, cam: PinholeCamera | None = None,
                  taken_frac: float = 0.1) -> Frame:
    """One pinhole stereo frame with its local map (the 752x480 single-frame workload)."""
    cam = cam or pinhole_camera(W, H)
    if images is None:
        images = stereo_images(seed * 7919 + 13, cam)
    rng = np.random.default_rng(seed)
    sc32 = level_scales32()
    lx, ly, loct = _level_pixel_keypoints(rng, n_left, W, H, sc32)
    ldesc = random_desc(rng, n_left)
    lab = images.label[np.clip(np.rint(ly).astype(np.int64), 0, H - 1),
                       np.clip(np.rint(lx).astype(np.int64), 0, W - 1)]
    zl = images.depth[lab]
    disp = cam.fx * cam.b / zl
    xr_true = lx.astype(np.float64) - disp
    # right keypoint of each correspondence, snapped to its level's pixel grid
    keep = xr_true >= 0
    rx_t = np.array([np.float32(np.float32(np.rint(xr / sc32[l])) * sc32[l])
                     for xr, l in zip(xr_true[keep], loct[keep])], np.float32)
    ry_t = ly[keep].copy()
    ro_t = loct[keep].copy()
    rd_t = flip_bits(rng, ldesc[keep], flip_p)
    n_d = int(round(distractor_frac * n_left))
    dx, dy, do = _level_pixel_keypoints(rng, n_d, W, H, sc32)
    rx = np.concatenate([rx_t, dx])
    ry = np.concatenate([ry_t, dy])
    ro = np.concatenate([ro_t, do])
    rd = np.concatenate([rd_t, random_desc(rng, n_d)])
    perm = rng.permutation(len(rx))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    right = Keypoints(x=rx[perm].astype(np.float32), y=ry[perm].astype(np.float32),
                      oct=ro[perm].astype(np.int8), desc=np.ascontiguousarray(rd[perm]))
    true_r = np.full(n_left, -1, np.int64)
    true_r[np.nonzero(keep)[0]] = inv[np.arange(keep.sum())]
    left = Keypoints(x=lx, y=ly, oct=loct, desc=ldesc)

    # poses: true pose and the perturbed estimate the tracker uses
    R_true = random_rotation(rng, 10.0)
    O_true = rng.normal(0.0, 1.0, 3)
    R_est, O_est = perturb_pose(rng, R_true, O_true)

    def unproj(u, v, z):
        return np.stack([(u - cam.cx) / cam.fx * z, (v - cam.cy) / cam.fy * z, z], axis=1)

    lmap, assoc = _local_map(rng, n_map, None, unproj, W, H, R_true, O_true, lx, ly, loct, ldesc,
                             zl, flip_p)
    taken = (rng.random(n_left) < taken_frac).astype(np.uint8)
    return Frame(camera="pinhole", left=left, right=right, pose=make_pose(R_est, O_est),
                 map=lmap, taken_l=taken, cam=cam, pyr_left=images.pyr_left,
                 pyr_right=images.pyr_right, pose_true=make_pose(R_true, O_true),
                 truth=dict(true_r=true_r, disparity=disp.astype(np.float64), map_kp=assoc))


# --------------------------------------------------------------------------
# fisheye stereo (Kannala-Brandt, equidistant with 4 coefficients)
# --------------------------------------------------------------------------
def kb8_camera(rng: np.random.Generator, W: int = 512, H: int = 512, f: float = 190.0) -> KB8Camera:
    k = rng.uniform(-0.01, 0.01, 4).astype(np.float32)
    return KB8Camera(fx=float(np.float32(f)), fy=float(np.float32(f)), cx=float(np.float32(W / 2)),
                     cy=float(np.float32(H / 2)), k=k, width=W, height=H, min_x=0.0,
                     max_x=float(W), min_y=0.0, max_y=float(H))


def kb8_project64(cam: KB8Camera, P: np.ndarray) -> np.ndarray:
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    rho = np.hypot(x, y)
    th = np.arctan2(rho, z)
    k = cam.k.astype(np.float64)
    thd = th * (1 + k[0] * th ** 2 + k[1] * th ** 4 + k[2] * th ** 6 + k[3] * th ** 8)
    s = np.where(rho > 0, thd / np.where(rho > 0, rho, 1.0), 0.0)
    return np.stack([cam.fx * x * s + cam.cx, cam.fy * y * s + cam.cy], axis=1)


def kb8_unproject64(cam: KB8Camera, u: np.ndarray, v: np.ndarray, dist: np.ndarray) -> np.ndarray:
    mx = (u - cam.cx) / cam.fx
    my = (v - cam.cy) / cam.fy
    thd = np.hypot(mx, my)
    k = cam.k.astype(np.float64)
    th = thd.copy()
    for _ in range(20):
        f = th * (1 + k[0] * th ** 2 + k[1] * th ** 4 + k[2] * th ** 6 + k[3] * th ** 8) - thd
        df = 1 + 3 * k[0] * th ** 2 + 5 * k[1] * th ** 4 + 7 * k[2] * th ** 6 + 9 * k[3] * th ** 8
        th = th - f / df
    s = np.where(thd > 0, np.sin(th) / np.where(thd > 0, thd, 1.0), 0.0)
    d = np.stack([mx * s, my * s, np.cos(th)], axis=1)
    return d * dist[:, None]


def fisheye_rig(seed: int, W: int = 512, H: int = 512, b: float = 0.10) -> FisheyeRig:
    rng = np.random.default_rng(seed)
    left = kb8_camera(rng, W, H)
    right = kb8_camera(rng, W, H)
    R_rl = random_rotation(rng, 0.5)
    t_rl = -R_rl @ np.array([b, 0.0, 0.0])
    return FisheyeRig(left=left, right=right, R_rl=R_rl.astype(np.float32).reshape(9),
                      t_rl=t_rl.astype(np.float32), b=float(np.float32(b)),
                      lap_l0=float(0.3 * W), lap_l1=float(W - 1), lap_r0=0.0,
                      lap_r1=float(0.7 * W - 1))


def fisheye_frame(seed: int, n_left: int = 1500, overlap_frac: float = 0.6, flip_p: float = 0.05,
                  n_map: int = 6000, rig: FisheyeRig | None = None, taken_frac: float = 0.1) -> Frame:
    """One fisheye stereo frame with its local map (the 512x512 workload)."""
    rig = rig or fisheye_rig(seed * 31 + 7)
    rng = np.random.default_rng(seed)
    W, H = rig.left.width, rig.left.height
    n_ov = int(round(overlap_frac * n_left))
    loct = sample_octaves(rng, n_left)
    lx = np.concatenate([rng.uniform(rig.lap_l0, rig.lap_l1, n_ov),
                         rng.uniform(0.0, rig.lap_l0 - 1.0, n_left - n_ov)]).astype(np.float32)
    ly = rng.uniform(0.0, H - 1.0, n_left).astype(np.float32)
    ldesc = random_desc(rng, n_left)
    dist = rng.uniform(1.0, 10.0, n_left)
    Pl = kb8_unproject64(rig.left, lx.astype(np.float64), ly.astype(np.float64), dist)
    Rrl = rig.R_rl.reshape(3, 3).astype(np.float64)
    Pr = Pl @ Rrl.T + rig.t_rl.astype(np.float64)[None, :]
    uvr = kb8_project64(rig.right, Pr)
    ok = ((np.arange(n_left) < n_ov) & (Pr[:, 2] > 0.1) & (uvr[:, 0] >= rig.lap_r0)
          & (uvr[:, 0] <= rig.lap_r1) & (uvr[:, 1] >= 0) & (uvr[:, 1] < H))
    rx_t = uvr[ok, 0].astype(np.float32)
    ry_t = uvr[ok, 1].astype(np.float32)
    ro_t = loct[ok]
    rd_t = flip_bits(rng, ldesc[ok], flip_p)
    n_d = max(0, n_left - len(rx_t))
    rx = np.concatenate([rx_t, rng.uniform(0.0, W - 1.0, n_d).astype(np.float32)])
    ry = np.concatenate([ry_t, rng.uniform(0.0, H - 1.0, n_d).astype(np.float32)])
    ro = np.concatenate([ro_t, sample_octaves(rng, n_d)])
    rd = np.concatenate([rd_t, random_desc(rng, n_d)])
    perm = rng.permutation(len(rx))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    right = Keypoints(x=rx[perm], y=ry[perm], oct=ro[perm].astype(np.int8),
                      desc=np.ascontiguousarray(rd[perm]))
    true_r = np.full(n_left, -1, np.int64)
    true_r[np.nonzero(ok)[0]] = inv[np.arange(ok.sum())]
    left = Keypoints(x=lx, y=ly, oct=loct, desc=ldesc)

    R_true = random_rotation(rng, 10.0)
    O_true = rng.normal(0.0, 1.0, 3)
    R_est, O_est = perturb_pose(rng, R_true, O_true)

    def unproj(u, v, z):
        return kb8_unproject64(rig.left, u, v, z)

    lmap, assoc = _local_map(rng, n_map, None, unproj, W, H, R_true, O_true, lx, ly, loct, ldesc,
                             dist, flip_p)
    # right camera centre in world, from the estimated pose: O_r = O + R^T * c_rl,
    # with c_rl = -R_rl^T t_rl the right centre in left coordinates
    c_rl = -Rrl.T @ rig.t_rl.astype(np.float64)
    O_right = (O_est + R_est.T @ c_rl).astype(np.float32)
    taken_l = (rng.random(n_left) < taken_frac).astype(np.uint8)
    taken_r = (rng.random(right.n) < taken_frac).astype(np.uint8)
    return Frame(camera="fisheye", left=left, right=right, pose=make_pose(R_est, O_est), map=lmap,
                 taken_l=taken_l, rig=rig, O_right=O_right, taken_r=taken_r,
                 pose_true=make_pose(R_true, O_true),
                 truth=dict(true_r=true_r, map_kp=assoc, P_left=Pl))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
_IMAGE_POOL: dict = {}


def _pooled_images(key, cam: PinholeCamera, seed: int) -> _StereoImages:
    k = (key, cam.width, cam.height, seed)
    if k not in _IMAGE_POOL:
        _IMAGE_POOL[k] = stereo_images(seed, cam)
    return _IMAGE_POOL[k]


def single_pinhole(seed: int = 0) -> Frame:
    """752x480 pinhole frame, 1200 left keypoints, 20% distractors, 3000 map points."""
    return pinhole_frame(seed)


def pinhole_batch(seed: int = 0, n_frames: int = 64, nl_range=(1000, 1500), m_range=(2000, 5000),
                  W: int = 752, H: int = 480, distractor_frac: float = 0.2, flip_p: float = 0.05,
                  image_pool: int = 8) -> list:
    """Ragged batch of pinhole frames (the 64-frame batched workload)."""
    rng = np.random.default_rng(10_000 + seed)
    cam = pinhole_camera(W, H)
    frames = []
    for f in range(n_frames):
        imgs = _pooled_images("pin", cam, 1000 * seed + (f % image_pool))
        nl = int(rng.integers(nl_range[0], nl_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        frames.append(pinhole_frame(seed * 100_003 + f, W, H, nl, distractor_frac, flip_p, m,
                                    images=imgs, cam=cam))
    return frames


def fisheye_batch(seed: int = 0, n_frames: int = 32, n_left: int = 1500, n_map: int = 6000) -> list:
    """Batch of fisheye frames (the 32-frame 512x512 workload)."""
    rig = fisheye_rig(seed * 31 + 7)
    return [fisheye_frame(seed * 100_003 + f, n_left, n_map=n_map, rig=rig) for f in range(n_frames)]


def stress_batch(seed: int = 0, n_frames: int = 32, n_left: int = 8000, n_map: int = 100_000,
                 image_pool: int = 2) -> list:
    """1920x1080, 8000 keypoints, 100k map points, 8% flips, 40% distractors."""
    cam = pinhole_camera(1920, 1080)
    frames = []
    for f in range(n_frames):
        imgs = _pooled_images("stress", cam, 1000 * seed + (f % image_pool))
        frames.append(pinhole_frame(seed * 100_003 + f, 1920, 1080, n_left, 0.4, 0.08, n_map,
                                    images=imgs, cam=cam))
    return frames


SERVED_RESOLUTIONS = ((640, 480, "pinhole"), (752, 480, "pinhole"), (1280, 720, "pinhole"),
                      (512, 512, "fisheye"))


def served_stream_frame(seed: int, stream: int) -> Frame:
    """One frame of a served camera stream: resolution uniform among the four
    served shapes, 500-4000 keypoints, 1k-20k map points."""
    rng = np.random.default_rng(50_000 + 7 * stream + seed)
    W, H, kind = SERVED_RESOLUTIONS[int(rng.integers(0, len(SERVED_RESOLUTIONS)))]
    nl = int(rng.integers(500, 4001))
    m = int(rng.integers(1000, 20001))
    if kind == "fisheye":
        return fisheye_frame(seed * 100_003 + stream, nl, n_map=m, rig=fisheye_rig(stream))
    cam = pinhole_camera(W, H)
    imgs = _pooled_images("served", cam, stream % 4)
    return pinhole_frame(seed * 100_003 + stream, W, H, nl, 0.2, 0.05, m, images=imgs, cam=cam)


def last_frame(fr: Frame, seed: int, motion: str = "none", n: int | None = None) -> LastFrame:
    """Last-frame points for frame `fr`: its local-map points (those placed
    behind keypoints keep about their keypoint's octave, the others get a
    random one; a few get an octave outside the pyramid), and a last pose
    with the current orientation whose centre lies behind ("forward"), ahead
    of ("backward") or beside ("none") the current one along the viewing
    axis, 0.3 m away (more than a stereo baseline) or 2 cm for "none"."""
    rng = np.random.default_rng(seed)
    m = fr.map
    M = m.n if n is None else min(n, m.n)
    oct_ = sample_octaves(rng, M).astype(np.int64)
    assoc = np.asarray(fr.truth.get("map_kp", np.zeros(0, np.int64))) if fr.truth else np.zeros(0, np.int64)
    na = min(len(assoc), M)
    if na:
        oct_[:na] = np.clip(fr.left.oct[assoc[:na]].astype(np.int64) + rng.integers(-1, 2, na), 0, NLEVELS - 1)
    bad = rng.random(M) < 0.02
    oct_[bad] = rng.choice([-1, NLEVELS, 100], bad.sum())
    R = fr.pose.R.reshape(3, 3).astype(np.float64)
    O = fr.pose.O.astype(np.float64)
    axis = R[2]                                     # viewing axis in world coordinates
    side = R[0]
    if motion == "forward":
        O_last = O - 0.3 * axis
    elif motion == "backward":
        O_last = O + 0.3 * axis
    else:
        O_last = O + 0.02 * side
    return LastFrame(pos=np.ascontiguousarray(m.pos[:M]), desc=np.ascontiguousarray(m.desc[:M]),
                     oct=oct_.astype(np.int8), skip=np.ascontiguousarray(m.skip[:M]),
                     pose=make_pose(R, O_last))


# --------------------------------------------------------------------------
# keypoint extraction inputs (next row f3)
# --------------------------------------------------------------------------
ORB_FAST_TH = 20
ORB_EDGE = 19


def orb_pattern(seed: int = 2011) -> np.ndarray:
    """256 test pairs (x1, y1, x2, y2) as int8: points drawn i.i.d. from an
    isotropic Gaussian of sigma 31/5 around the keypoint, rounded, kept if
    inside the disk of radius 13; pairs of equal points are drawn again."""
    rng = np.random.default_rng(seed)
    out = np.zeros((256, 4), np.int8)
    i = 0
    while i < 256:
        p = np.rint(rng.normal(0.0, 31.0 / 5.0, 4))
        if p[0] ** 2 + p[1] ** 2 > 169 or p[2] ** 2 + p[3] ** 2 > 169 or (p[0] == p[2] and p[1] == p[3]):
            continue
        out[i] = p.astype(np.int8)
        i += 1
    return out


def orb_level_caps(n_features: int, nlevels: int = NLEVELS, s: float = SCALE) -> list:
    """Keypoint slots per level: a geometric share (1/s)^l of n_features per
    level, the last level taking what remains."""
    f = 1.0 / s
    n0 = n_features * (1.0 - f) / (1.0 - f ** nlevels)
    caps = [int(round(n0 * f ** l)) for l in range(nlevels - 1)]
    caps.append(max(0, n_features - sum(caps)))
    return caps


def frame_with_keypoints(seed: int, cam: PinholeCamera, images: _StereoImages, left: Keypoints,
                         right: Keypoints, n_map: int = 3000, flip_p: float = 0.05) -> Frame:
    """A pinhole frame with the given keypoints (for instance extracted from
    its own images): its local map is placed behind the left keypoints that
    are not padding (x >= 0) at the depth of the image's plane there, plus
    random points, as in pinhole_frame."""
    rng = np.random.default_rng(seed)
    W, H = cam.width, cam.height
    valid = np.nonzero(left.x >= 0)[0]
    lx, ly = left.x[valid], left.y[valid]
    lab = images.label[np.clip(np.rint(ly).astype(np.int64), 0, H - 1), np.clip(np.rint(lx).astype(np.int64), 0, W - 1)]
    zl = images.depth[lab]
    R_true = random_rotation(rng, 10.0)
    O_true = rng.normal(0.0, 1.0, 3)
    R_est, O_est = perturb_pose(rng, R_true, O_true)

    def unproj(u, v, z):
        return np.stack([(u - cam.cx) / cam.fx * z, (v - cam.cy) / cam.fy * z, z], axis=1)

    lmap, assoc = _local_map(rng, n_map, None, unproj, W, H, R_true, O_true, lx, ly, left.oct[valid],
                             left.desc[valid], zl, flip_p)
    return Frame(camera="pinhole", left=left, right=right, pose=make_pose(R_est, O_est), map=lmap,
                 taken_l=np.zeros(left.n, np.uint8), cam=cam, pyr_left=images.pyr_left,
                 pyr_right=images.pyr_right, pose_true=make_pose(R_true, O_true),
                 truth=dict(map_kp=valid[assoc]))
