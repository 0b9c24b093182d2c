// ft_api.cu -- host side of libfasttrack.so: the C ABI of fasttrack.h.
//
// Context = one device arena allocated once at creation (the paper
// preallocates all GPU memory at start-up and reuses it, section IV-A),
// a ring of pinned staging slots for the per-call batch table, events, a
// CUDA-graph cache and the tuning table.  Every entry point turns its
// arguments into a batch table (see ft_internal.h), copies it into the
// arena with one cudaMemcpyAsync and launches the fused persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "ft_internal.h"

using namespace ft;

namespace {

thread_local std::string g_last_error;

ft_status fail(ft_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define FT_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(FT_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

constexpr int kSlots = 4;
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct TableLayout {
    size_t hdr, queue, counters, prefix, frames, total;
};

TableLayout table_layout(int n)
{
    TableLayout L{};
    size_t off = 0;
    L.hdr = off;
    off = align_up(off + sizeof(BatchHeader));
    L.queue = off;
    off = align_up(off + 64);
    L.counters = off;
    off = align_up(off + sizeof(unsigned) * kCounters * (size_t)std::max(n, 1));
    L.prefix = off;
    off = align_up(off + sizeof(int) * K_KINDS * (size_t)(n + 1));
    L.frames = off;
    off = align_up(off + sizeof(FrameDev) * (size_t)std::max(n, 1));
    L.total = off;
    return L;
}

// bytes of an extraction table of n images: header, images, counters
size_t orb_table_bytes(int n)
{
    const size_t o_img = align_up(sizeof(OrbHeader));
    const size_t o_cnt = align_up(o_img + sizeof(OrbImage) * (size_t)std::max(n, 1));
    return align_up(o_cnt + sizeof(unsigned) * FT_MAX_LEVELS * (size_t)std::max(n, 1));
}

struct Bucket {
    int frames_p2, has_pinhole, has_fisheye, nl_p2, m_p2;
    bool operator<(const Bucket &o) const
    {
        return std::tie(frames_p2, has_pinhole, has_fisheye, nl_p2, m_p2) <
               std::tie(o.frames_p2, o.has_pinhole, o.has_fisheye, o.nl_p2, o.m_p2);
    }
};

// One frame as the table builder sees it (built from the public structs).
struct Job {
    int camera = FT_CAMERA_PINHOLE;
    bool do_stereo = false, do_search = false, wait_stereo = false;
    ft_pinhole pin{};
    ft_fisheye_rig rig{};
    ft_keypoints left{}, right{};
    ft_pyramid pyr_l{}, pyr_r{};
    const uint8_t *taken_l = nullptr, *taken_r = nullptr;
    ft_pose pose{};
    float O_right[3] = {0, 0, 0};
    ft_map_view map{};
    ft_stereo_out st{};
    ft_fisheye_out fo{};
    ft_search_out so{};
    const float *u_right_in = nullptr;
    int build_pyr = 0;                    // levels 1.. built on the device from level 0: bit 0 the left
                                          // pyramid, bit 1 the right one
    int search_mode = 0;                  // 0: local map; 1: the last frame's points (map.nrm unused)
    const int8_t *last_oct = nullptr;
    ft_pose last_pose{};
    bool do_pose = false;                 // pose optimization after the search (pinhole)
    ft_pose_out po{};
    const int32_t *po_mp_kp = nullptr;    // matches when the call does no search
};

// the map view and mode of a last-frame search
void set_last(Job &j, const ft_last_frame_view &l)
{
    j.search_mode = 1;
    j.map = ft_map_view{};
    j.map.n = l.n;
    j.map.pos = l.pos;
    j.map.desc = l.desc;
    j.map.skip = l.skip;
    j.last_oct = l.oct;
    j.last_pose = l.pose;
}

}  // namespace

struct ft_ctx {
    int device = 0;
    int sm_count = 0;
    int occ = 1;                      // max resident CTAs per SM of the fused kernel
    char *arena = nullptr;
    size_t arena_bytes = 0;
    int max_frames = 0;
    size_t table_cap = 0;             // bytes of the table region
    size_t scratch_off = 0;           // scratch region offset in the arena
    unsigned *status = nullptr;       // device status word
    char *staging[kSlots] = {};
    cudaEvent_t slot_done[kSlots] = {};
    int slot = 0;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
    bool use_graphs = false;
    cudaStream_t capture_stream = nullptr;
    // graphs by (bucket frames, CTAs/SM, slot, pyramid frames, pyramid
    // blocks per image, pyramid levels, pose frames)
    std::map<std::tuple<int, int, int, int, int, int, int>, cudaGraphExec_t> graphs;
    std::map<Bucket, ft_tuning> tuning;
    uint64_t launches = 0;
    unsigned debug_flags = 0;
    unsigned long long timeout_ns = 2000000000ull;
    ft_trace_record *trace = nullptr;  // device buffer (tracing on)
    int trace_cap = 0;
};

namespace {

ft_tuning default_tuning()
{
    ft_tuning t{};
    t.strip_rows = 32;
    t.search_tile = 512;
    t.fisheye_tile = 128;
    t.resolve_tile = 2048;
    t.ctas_per_sm = 0;
    t.search_stage = 0;
    t.split_search = 0;
    return t;
}

}  // namespace

// parameter checks shared by every entry point (ft_noalloc.cu included)
ft_status ft::check_params(const ft_params &p)
{
    if (p.nlevels < 1 || p.nlevels > FT_MAX_LEVELS) return fail(FT_EINVAL, "nlevels %d out of [1, 16]", p.nlevels);
    if (!(p.scale_factor >= 1.0f) || !std::isfinite(p.scale_factor))
        return fail(FT_EINVAL, "scale_factor must be >= 1");
    if (!(p.median_factor >= 0.0f)) return fail(FT_EINVAL, "median_factor must be >= 0");
    if (!(p.search_th > 0.0f)) return fail(FT_EINVAL, "search_th must be > 0");
    if (!(p.th_last > 0.0f) || !std::isfinite(p.th_last)) return fail(FT_EINVAL, "th_last must be > 0");
    if (p.kb_iters < 1 || p.kb_iters > 64) return fail(FT_EINVAL, "kb_iters %d out of [1, 64]", p.kb_iters);
    if (!(p.min_depth >= 0.0f) || !std::isfinite(p.min_depth)) return fail(FT_EINVAL, "min_depth must be >= 0");
    if (p.po_rounds < 1 || p.po_rounds > 16) return fail(FT_EINVAL, "po_rounds %d out of [1, 16]", p.po_rounds);
    if (p.po_iters < 1 || p.po_iters > 64) return fail(FT_EINVAL, "po_iters %d out of [1, 64]", p.po_iters);
    if (!(p.po_chi2_mono > 0.0f) || !std::isfinite(p.po_chi2_mono) || !(p.po_chi2_stereo > 0.0f) ||
        !std::isfinite(p.po_chi2_stereo))
        return fail(FT_EINVAL, "pose optimization chi2 thresholds must be finite and > 0");
    float sc = 1.0f;
    for (int l = 1; l < p.nlevels; ++l) sc = sc * p.scale_factor;
    if (!(2.0f * sc < 1.0e6f)) return fail(FT_EINVAL, "scale_factor^(nlevels-1) = %g is too large", sc);
    return FT_OK;
}

namespace {

ft_status check_kps(const ft_keypoints &k, const char *what)
{
    if (k.n < 0 || k.n >= FT_MAX_KEYPOINTS) return fail(FT_EINVAL, "%s: n=%d out of range", what, k.n);
    if (k.n == 0) return FT_OK;
    if (!k.x || !k.y || !k.oct || !k.desc) return fail(FT_EINVAL, "%s: NULL array", what);
    if (!aligned16(k.desc)) return fail(FT_EALIGN, "%s: desc not 16-byte aligned", what);
    return FT_OK;
}

// level sizes of a device-built pyramid: round(size / scale[l]), scale[l]
// the FP32 product of the scale factor (the device table's values)
void pyramid_sizes(int W, int H, const ft_params &p, int *w, int *h)
{
    float sc = 1.0f;
    for (int l = 0; l < p.nlevels; ++l) {
        if (l > 0) sc = sc * p.scale_factor;
        w[l] = (int)std::round((float)W / sc);
        h[l] = (int)std::round((float)H / sc);
    }
}

ft_status check_pyramid(const ft_pyramid &p, int nlevels, const char *what)
{
    if (p.nlevels < nlevels) return fail(FT_EINVAL, "%s: %d levels, need %d", what, p.nlevels, nlevels);
    for (int l = 0; l < nlevels; ++l) {
        if (!p.data[l]) return fail(FT_EINVAL, "%s: level %d is NULL", what, l);
        if (p.width[l] <= 0 || p.height[l] <= 0 || p.pitch[l] < p.width[l])
            return fail(FT_EINVAL, "%s: level %d has bad size %dx%d pitch %d", what, l, p.width[l],
                        p.height[l], p.pitch[l]);
        if ((reinterpret_cast<uintptr_t>(p.data[l]) & 15u) || (p.pitch[l] & 15))
            return fail(FT_EALIGN, "%s: level %d needs a 16-byte aligned pointer and pitch (pitch %d)", what, l,
                        p.pitch[l]);
    }
    return FT_OK;
}

ft_status check_bounds(float a, float b, const char *what)
{
    if (!(b > a) || !std::isfinite(a) || !std::isfinite(b)) return fail(FT_EINVAL, "%s: empty range", what);
    return FT_OK;
}

ft_status check_job(const Job &j, const ft_params &p)
{
    ft_status s;
    if ((s = check_kps(j.left, "left keypoints")) != FT_OK) return s;
    if (j.camera == FT_CAMERA_FISHEYE || j.do_stereo)
        if ((s = check_kps(j.right, "right keypoints")) != FT_OK) return s;
    if (j.build_pyr) {
        if (j.camera != FT_CAMERA_PINHOLE) return fail(FT_EINVAL, "pyramids are built for pinhole frames only");
        const ft_pyramid *pp[2] = {&j.pyr_l, &j.pyr_r};
        for (const ft_pyramid *py : pp) {
            if ((s = check_pyramid(*py, p.nlevels, "pyramid")) != FT_OK) return s;
            int w[FT_MAX_LEVELS], h[FT_MAX_LEVELS];
            pyramid_sizes(py->width[0], py->height[0], p, w, h);
            for (int l = 1; l < p.nlevels; ++l)
                if (py->width[l] != w[l] || py->height[l] != h[l])
                    return fail(FT_EINVAL, "pyramid level %d is %dx%d, a built level is %dx%d", l, py->width[l],
                                py->height[l], w[l], h[l]);
            for (int l = 0; l < p.nlevels; ++l)
                if ((long long)py->pitch[l] * py->height[l] > kPyrMaxLevelBytes)
                    return fail(FT_EINVAL, "pyramid level %d (%d rows of pitch %d) exceeds 2^31 bytes", l,
                                py->height[l], py->pitch[l]);
        }
    }
    if (j.camera == FT_CAMERA_PINHOLE) {
        if (j.pin.width <= 0 || j.pin.height <= 0) return fail(FT_EINVAL, "pinhole: bad image size");
        if (j.do_search) {
            if ((s = check_bounds(j.pin.min_x, j.pin.max_x, "pinhole x bounds")) != FT_OK) return s;
            if ((s = check_bounds(j.pin.min_y, j.pin.max_y, "pinhole y bounds")) != FT_OK) return s;
        }
        if (j.do_stereo) {
            if (!(j.pin.b > 0.0f)) return fail(FT_EINVAL, "pinhole: baseline must be > 0");
            if (j.pin.height > kMaxRows)
                return fail(FT_EINVAL, "pinhole: %d rows exceed the %d-row stereo limit", j.pin.height, kMaxRows);
            if ((s = check_pyramid(j.pyr_l, p.nlevels, "left pyramid")) != FT_OK) return s;
            if ((s = check_pyramid(j.pyr_r, p.nlevels, "right pyramid")) != FT_OK) return s;
            const ft_stereo_out &o = j.st;
            if (j.left.n > 0 && (!o.best_r || !o.dist || !o.sad_shift || !o.sad_best || !o.u_right || !o.depth))
                return fail(FT_EINVAL, "stereo output: NULL array");
        }
    } else if (j.camera == FT_CAMERA_FISHEYE) {
        if (j.do_stereo && j.fo.xyz && !aligned16(j.fo.xyz))
            return fail(FT_EALIGN, "fisheye output: xyz not 16-byte aligned");
        if (j.do_stereo && j.left.n > 0 && (!j.fo.r_idx || !j.fo.d1 || !j.fo.d2))
            return fail(FT_EINVAL, "fisheye output: NULL array");
        if (j.do_search) {
            const ft_kb8 *c[2] = {&j.rig.left, &j.rig.right};
            for (auto *cam : c) {
                if ((s = check_bounds(cam->min_x, cam->max_x, "fisheye x bounds")) != FT_OK) return s;
                if ((s = check_bounds(cam->min_y, cam->max_y, "fisheye y bounds")) != FT_OK) return s;
            }
        }
    } else {
        return fail(FT_EINVAL, "unknown camera model %d", j.camera);
    }
    if (j.do_pose) {
        if (j.camera != FT_CAMERA_PINHOLE) return fail(FT_EINVAL, "pose optimization: pinhole frames only");
        const ft_map_view &m = j.map;
        if (m.n < 0 || m.n >= FT_MAX_MAP_POINTS) return fail(FT_EINVAL, "map: n=%d out of range", m.n);
        if (!j.po.Rt || !j.po.n_inliers || (m.n > 0 && !j.po.inlier))
            return fail(FT_EINVAL, "pose output: NULL array");
        if (m.n > 0 && (!m.pos || !aligned16(m.pos))) return fail(FT_EALIGN, "map: pos NULL or not 16-byte aligned");
        if (!j.do_search && m.n > 0 && !j.po_mp_kp) return fail(FT_EINVAL, "pose optimization: NULL mp_kp");
        if (!j.do_search && (s = check_kps(j.left, "left keypoints")) != FT_OK) return s;
    }
    if (j.do_search) {
        const ft_map_view &m = j.map;
        if (m.n < 0 || m.n >= FT_MAX_MAP_POINTS) return fail(FT_EINVAL, "map: n=%d out of range", m.n);
        if (m.n > 0 && j.search_mode == 0) {
            if (!m.pos || !m.nrm || !m.desc) return fail(FT_EINVAL, "map: NULL array");
            if (!aligned16(m.pos) || !aligned16(m.nrm) || !aligned16(m.desc))
                return fail(FT_EALIGN, "map: pos/nrm/desc not 16-byte aligned");
        }
        if (m.n > 0 && j.search_mode == 1) {
            if (!m.pos || !m.desc || !j.last_oct) return fail(FT_EINVAL, "last frame: NULL array");
            if (!aligned16(m.pos) || !aligned16(m.desc))
                return fail(FT_EALIGN, "last frame: pos/desc not 16-byte aligned");
        }
        const int ncam = j.camera == FT_CAMERA_FISHEYE ? 2 : 1;
        for (int c = 0; c < ncam; ++c) {
            const ft_search_cam_out &o = c ? j.so.right : j.so.left;
            const int nk = c ? j.right.n : j.left.n;
            if (m.n > 0 && (!o.level || !o.mp_kp || !o.mp_d1 || !o.mp_d2))
                return fail(FT_EINVAL, "search output: NULL array");
            if (nk > 0 && !o.kp_mp) return fail(FT_EINVAL, "search output: NULL kp_mp");
            if (o.proj && !aligned16(o.proj)) return fail(FT_EALIGN, "search output: proj not 16-byte aligned");
        }
    }
    return FT_OK;
}

}  // namespace

DevParams ft::make_dev_params(const ft_params &p)
{
    DevParams d{};
    d.nlevels = p.nlevels;
    d.th_stereo = p.th_stereo;
    d.th_search = p.th_search;
    d.ratio_any_octave = p.ratio_any_octave;
    float sc = 1.0f;
    float rmax = 0.0f;
    for (int l = 0; l < FT_MAX_LEVELS; ++l) {
        if (l > 0 && l < p.nlevels) sc = sc * p.scale_factor;
        d.sc[l] = sc;
        d.isc[l] = 1.0f / sc;
        d.band_r[l] = 2.0f * sc;
        if (l < p.nlevels) rmax = std::max(rmax, d.band_r[l]);
    }
    d.median_factor = p.median_factor;
    d.fisheye_ratio = p.fisheye_ratio;
    d.nn_ratio = p.nn_ratio;
    d.search_th = p.search_th;
    d.view_cos_min = p.view_cos_min;
    d.view_cos_narrow = p.view_cos_narrow;
    d.radius_narrow = p.radius_narrow;
    d.radius_wide = p.radius_wide;
    d.dist_lo = p.dist_lo;
    d.th_last = p.th_last;
    d.kb_iters = p.kb_iters;
    d.min_depth = p.min_depth;
    d.dist_hi = p.dist_hi;
    d.po_rounds = p.po_rounds;
    d.po_iters = p.po_iters;
    d.po_huber = p.po_huber;
    d.po_chi2_mono = p.po_chi2_mono;
    d.po_chi2_stereo = p.po_chi2_stereo;
    // a right keypoint's band reaches rows within ceil(r) + 2 of floor(y); +1 margin
    d.halo = (int)std::ceil(rmax) + 3;
    // a left keypoint of octave o only meets right octaves up to o + 1
    for (int o = 0; o < FT_MAX_LEVELS; ++o) {
        const int top = std::min(o + 1, std::max(p.nlevels - 1, 0));
        d.halo_oct[o] = (int)std::ceil(d.band_r[top]) + 3;
        d.halo_c[o] = (int)std::ceil(d.band_r[std::min(o, std::max(p.nlevels - 1, 0))]) + 3;
    }
    return d;
}

// Strip height of the pinhole stereo items: at most `want` rows and the
// image height; the staged window (strip + 2 halo rows) must fit kWinRows
// rows, and the right keypoints it is expected to hold (at the frame's mean
// density) 3/4 of the shared-memory stage.
int ft::stereo_strip_rows(int want, int H, int nr, int halo)
{
    int sr = std::max(1, want);
    sr = std::min(sr, std::max(1, H));
    sr = std::min(sr, std::max(1, kWinRows - 2 * halo));
    if (nr > 0) {
        const double per_row = (double)nr / (double)std::max(1, H);
        const int cap_rows = (int)(0.75 * kStageCap / per_row) - 2 * halo;
        sr = std::max(1, std::min(sr, cap_rows));
    }
    return sr;
}

namespace {

Bucket bucket_of(const std::vector<Job> &jobs)
{
    Bucket b{};
    b.frames_p2 = next_pow2((int)jobs.size());
    int nl = 1, m = 1;
    for (const Job &j : jobs) {
        if (j.camera == FT_CAMERA_FISHEYE) b.has_fisheye = 1;
        else b.has_pinhole = 1;
        nl = std::max(nl, j.left.n);
        m = std::max(m, j.map.n);
    }
    b.nl_p2 = next_pow2(nl);
    b.m_p2 = next_pow2(m);
    return b;
}

void fill_cam_kb8(CamDev &C, const ft_kb8 &k)
{
    C.model = FT_CAMERA_FISHEYE;
    C.fx = k.fx;
    C.fy = k.fy;
    C.cx = k.cx;
    C.cy = k.cy;
    for (int i = 0; i < 4; ++i) C.k[i] = k.k[i];
    C.minx = k.min_x;
    C.maxx = k.max_x;
    C.miny = k.min_y;
    C.maxy = k.max_y;
}

void fill_cam_out(CamDev &C, const ft_search_cam_out &o)
{
    C.level = o.level;
    C.proj = reinterpret_cast<float4 *>(o.proj);
    C.mp_kp = o.mp_kp;
    C.mp_d1 = o.mp_d1;
    C.mp_d2 = o.mp_d2;
    C.kp_mp = o.kp_mp;
}

void fill_cam_kps(CamDev &C, const ft_keypoints &k, const uint8_t *taken)
{
    C.nk = k.n;
    C.kx = k.x;
    C.ky = k.y;
    C.koct = k.oct;
    C.kdesc = reinterpret_cast<const uint4 *>(k.desc);
    C.taken = taken;
}

// Build the table for `jobs` into host buffer `h` (laid out for the device
// base `dev`), carving per-frame scratch from the arena.  Returns bytes used.
ft_status build_table(ft_ctx *ctx, const ft_params &params, const std::vector<Job> &jobs,
                      const ft_tuning &tune, char *h, char *dev, size_t *bytes_out, int *items_out)
{
    const int n = (int)jobs.size();
    const TableLayout L = table_layout(n);
    if (L.total > ctx->table_cap) return fail(FT_ENOMEM, "batch table of %d frames exceeds the context", n);
    std::memset(h, 0, L.total);
    BatchHeader &B = *reinterpret_cast<BatchHeader *>(h + L.hdr);
    B.p = make_dev_params(params);
    B.nframes = n;
    B.debug_flags = ctx->debug_flags;
    B.prefix = reinterpret_cast<const int *>(dev + L.prefix);
    B.frames = reinterpret_cast<const FrameDev *>(dev + L.frames);
    B.queue = reinterpret_cast<unsigned *>(dev + L.queue);
    B.status = ctx->status;
    B.timeout_ns = ctx->timeout_ns;
    B.trace = ctx->trace;
    B.trace_cap = ctx->trace_cap;
    unsigned *ctr_h = reinterpret_cast<unsigned *>(h + L.counters);
    unsigned *ctr_d = reinterpret_cast<unsigned *>(dev + L.counters);
    int *prefix = reinterpret_cast<int *>(h + L.prefix);
    FrameDev *frames = reinterpret_cast<FrameDev *>(h + L.frames);

    size_t scratch = ctx->scratch_off;
    auto carve = [&](size_t bytes) -> char * {
        char *p = ctx->arena + scratch;
        scratch = align_up(scratch + std::max<size_t>(bytes, 1));
        return p;
    };
    const int halo = B.p.halo;
    int counts[K_KINDS] = {};
    for (int f = 0; f < n; ++f) {
        const Job &j = jobs[f];
        FrameDev &F = frames[f];
        F.camera = j.camera;
        F.do_stereo = j.do_stereo;
        F.do_search = j.do_search;
        F.wait_stereo = j.wait_stereo;
        F.nl = j.left.n;
        F.nr = j.right.n;
        F.nm = (j.do_search || j.do_pose) ? j.map.n : 0;
        F.lx = j.left.x;
        F.ly = j.left.y;
        F.loct = j.left.oct;
        F.ldesc = reinterpret_cast<const uint4 *>(j.left.desc);
        F.rx = j.right.x;
        F.ry = j.right.y;
        F.roct = j.right.oct;
        F.rdesc = reinterpret_cast<const uint4 *>(j.right.desc);
        F.ctr = ctr_d + (size_t)kCounters * f;
        unsigned *ctr = ctr_h + (size_t)kCounters * f;
        int n_stereo = 0;
        if (j.camera == FT_CAMERA_PINHOLE) {
            F.H = j.pin.height;
            F.b = j.pin.b;
            F.bf = j.pin.bf;
            F.build_pyr = j.build_pyr;
            if (j.do_stereo || j.build_pyr) {
                for (int l = 0; l < params.nlevels; ++l) {
                    F.pyrL[l] = j.pyr_l.data[l];
                    F.lw[l] = j.pyr_l.width[l];
                    F.lh[l] = j.pyr_l.height[l];
                    F.lp[l] = j.pyr_l.pitch[l];
                    F.pyrR[l] = j.pyr_r.data[l];
                    F.rw[l] = j.pyr_r.width[l];
                    F.rh[l] = j.pyr_r.height[l];
                    F.rp[l] = j.pyr_r.pitch[l];
                }
            }
            if (j.do_stereo) {
                F.best_r = j.st.best_r;
                F.dist = j.st.dist;
                F.sad_shift = j.st.sad_shift;
                F.sad_best = j.st.sad_best;
                F.u_right = j.st.u_right;
                F.depth = j.st.depth;
                const int sr = stereo_strip_rows(tune.strip_rows, F.H, F.nr, halo);
                F.strip_rows = sr;
                n_stereo = (F.H + sr - 1) / sr;
                F.rowsort = kRowSortItems;
                F.row_ptr_l = reinterpret_cast<int *>(carve(sizeof(int) * (size_t)(F.H + 1)));
                F.row_ptr_r = reinterpret_cast<int *>(carve(sizeof(int) * (size_t)(F.H + 1)));
                F.ls_kp = reinterpret_cast<float4 *>(carve(sizeof(float4) * (size_t)F.nl));
                F.ls_desc = reinterpret_cast<uint4 *>(carve(sizeof(uint4) * 2 * (size_t)F.nl));
                F.rs_kp = reinterpret_cast<float4 *>(carve(sizeof(float4) * (size_t)F.nr));
                F.rs_desc = reinterpret_cast<uint4 *>(carve(sizeof(uint4) * 2 * (size_t)F.nr));
            }
        } else {
            F.lap_l0 = j.rig.lap_l0;
            F.lap_l1 = j.rig.lap_l1;
            F.lap_r0 = j.rig.lap_r0;
            F.lap_r1 = j.rig.lap_r1;
            for (int i = 0; i < 9; ++i) F.R_rl[i] = j.rig.R_rl[i];
            for (int i = 0; i < 3; ++i) F.t_rl[i] = j.rig.t_rl[i];
            const ft_kb8 *kb[2] = {&j.rig.left, &j.rig.right};
            for (int c = 0; c < 2; ++c) {
                float *d = c ? F.kbr : F.kbl;
                d[0] = kb[c]->fx;
                d[1] = kb[c]->fy;
                d[2] = kb[c]->cx;
                d[3] = kb[c]->cy;
                for (int i = 0; i < 4; ++i) d[4 + i] = kb[c]->k[i];
            }
            if (j.do_stereo) {
                F.r_idx = j.fo.r_idx;
                F.fd1 = j.fo.d1;
                F.fd2 = j.fo.d2;
                F.fdepth = j.fo.depth;
                F.fxyz = reinterpret_cast<float4 *>(j.fo.depth ? j.fo.xyz : nullptr);
                F.fisheye_tile = tune.fisheye_tile >= kFishTileMax ? kFishTileMax : kFishTileMax / 2;
                n_stereo = (F.nl + F.fisheye_tile - 1) / F.fisheye_tile;
            }
        }
        F.n_stereo_items = n_stereo;
        if (n_stereo == 0) ctr[C_STEREO_READY] = 1;

        int n_index = 0, n_search[2] = {0, 0}, n_resolve[2] = {0, 0};
        if (j.do_search) {
            F.ncam = j.camera == FT_CAMERA_FISHEYE ? 2 : 1;
            F.u_right_in = j.camera == FT_CAMERA_PINHOLE ? j.u_right_in : nullptr;
            F.pos = reinterpret_cast<const float4 *>(j.map.pos);
            F.nrm = reinterpret_cast<const float4 *>(j.map.nrm);
            F.mdesc = reinterpret_cast<const uint4 *>(j.map.desc);
            F.skip = j.map.skip;
            F.search_mode = j.search_mode;
            F.last_oct = j.last_oct;
            for (int i = 0; i < 9; ++i) F.last_R[i] = j.last_pose.R[i];
            for (int i = 0; i < 3; ++i) F.last_t[i] = j.last_pose.t[i];
            F.base = j.camera == FT_CAMERA_PINHOLE ? j.pin.b : j.rig.b;
            F.search_tile = std::max(kThreads, tune.search_tile / kThreads * kThreads);
            F.search_stage = tune.search_stage ? 1 : 0;
            F.resolve_tile = std::max(kThreads, tune.resolve_tile / kThreads * kThreads);
            for (int c = 0; c < F.ncam; ++c) {
                CamDev &C = F.cam[c];
                if (j.camera == FT_CAMERA_PINHOLE) {
                    C.model = FT_CAMERA_PINHOLE;
                    C.fx = j.pin.fx;
                    C.fy = j.pin.fy;
                    C.cx = j.pin.cx;
                    C.cy = j.pin.cy;
                    C.bf = j.pin.bf;
                    C.minx = j.pin.min_x;
                    C.maxx = j.pin.max_x;
                    C.miny = j.pin.min_y;
                    C.maxy = j.pin.max_y;
                } else {
                    fill_cam_kb8(C, c ? j.rig.right : j.rig.left);
                }
                for (int i = 0; i < 9; ++i) C.R[i] = j.pose.R[i];
                for (int i = 0; i < 3; ++i) {
                    C.t[i] = j.pose.t[i];
                    C.O[i] = c ? j.O_right[i] : j.pose.O[i];
                }
                fill_cam_kps(C, c ? j.right : j.left, c ? j.taken_r : j.taken_l);
                fill_cam_out(C, c ? j.so.right : j.so.left);
                C.cell_ptr = reinterpret_cast<int *>(carve(sizeof(int) * (kCells + 1)));
                C.cell16 = reinterpret_cast<uint16_t *>(carve(sizeof(uint16_t) * (kCells + 1)));
                C.gkp = reinterpret_cast<float4 *>(carve(sizeof(float4) * (size_t)C.nk));
                C.gdesc = reinterpret_cast<uint4 *>(carve(sizeof(uint4) * 2 * (size_t)C.nk));
                C.gpos = reinterpret_cast<int *>(carve(sizeof(int) * (size_t)C.nk));
                C.owner = reinterpret_cast<unsigned long long *>(carve(sizeof(unsigned long long) * (size_t)C.nk));
                // a pinhole frame whose stereo step runs in the same launch splits
                // its search around it (search items need not wait for it)
                F.split_search = j.wait_stereo && (tune.split_search > 0 || (tune.split_search == 0 && n <= 32));
                if (F.split_search) C.scan = reinterpret_cast<uint4 *>(carve(sizeof(uint4) * 2 * (size_t)F.nm));
                n_search[c] = (F.nm + F.search_tile - 1) / F.search_tile;
                n_resolve[c] = (std::max(F.nm, C.nk) + F.resolve_tile - 1) / F.resolve_tile;
            }
            // small frames: the last search item resolves (no resolve items wait)
            bool fold = true;
            for (int c = 0; c < F.ncam; ++c)
                fold = fold && n_search[c] > 0 && std::max(F.nm, F.cam[c].nk) <= kFoldResolveMax;
            if (fold) {
                F.fold_resolve = 1;
                n_resolve[0] = n_resolve[1] = 0;
            }
            F.n_grid_items = F.ncam;
        }
        if (j.do_pose) {
            CamDev &C = F.cam[0];
            if (!j.do_search) {
                // the standalone call: the camera, pose and keypoints the
                // search would have set up
                C.model = FT_CAMERA_PINHOLE;
                C.fx = j.pin.fx;
                C.fy = j.pin.fy;
                C.cx = j.pin.cx;
                C.cy = j.pin.cy;
                C.bf = j.pin.bf;
                for (int i = 0; i < 9; ++i) C.R[i] = j.pose.R[i];
                for (int i = 0; i < 3; ++i) C.t[i] = j.pose.t[i];
                fill_cam_kps(C, j.left, nullptr);
                F.u_right_in = j.u_right_in;
                F.pos = reinterpret_cast<const float4 *>(j.map.pos);
            }
            F.do_pose = 1;
            F.po_mp_kp = j.do_search ? j.so.left.mp_kp : j.po_mp_kp;
            F.po_Rt = j.po.Rt;
            F.po_inlier = j.po.inlier;
            F.po_n = j.po.n_inliers;
            F.po_list = reinterpret_cast<float4 *>(carve(sizeof(float4) * 2 * (size_t)std::max(F.nm, 1)));
        }
        n_index = F.rowsort + F.n_grid_items;
        if (scratch > ctx->arena_bytes)
            return fail(FT_ENOMEM, "arena of %zu bytes too small for this batch (needs %zu)", ctx->arena_bytes, scratch);
        F.n_index_items = n_index;
        F.n_search_items[0] = n_search[0];
        F.n_search_items[1] = n_search[1];
        F.n_resolve_items[0] = n_resolve[0];
        F.n_resolve_items[1] = n_resolve[1];
        const int per_kind[K_KINDS] = {n_index, n_stereo, n_search[0] + n_search[1],
                                       n_resolve[0] + n_resolve[1]};
        for (int k = 0; k < K_KINDS; ++k) {
            prefix[k * (n + 1) + f] = counts[k];
            counts[k] += per_kind[k];
        }
    }
    int total = 0;
    for (int k = 0; k < K_KINDS; ++k) {
        prefix[k * (n + 1) + n] = counts[k];
        B.kind_begin[k] = total;
        total += counts[k];
    }
    B.kind_begin[K_KINDS] = total;
    B.total_items = total;
    *bytes_out = L.total;
    *items_out = total;
    return FT_OK;
}

ft_status order_stream(ft_ctx *ctx, cudaStream_t s)
{
    if (ctx->have_last && ctx->last_stream != s) FT_CUDA(cudaStreamWaitEvent(s, ctx->done, 0));
    return FT_OK;
}

ft_status finish_call(ft_ctx *ctx, cudaStream_t s)
{
    FT_CUDA(cudaEventRecord(ctx->done, s));
    ctx->last_stream = s;
    ctx->have_last = true;
    return FT_OK;
}

ft_status get_graph(ft_ctx *ctx, char *table_dev, int frames_p2, int cps, int slot, int grid,
                    size_t copy_bytes, int pyr_frames, int pyr_blocks, int pyr_levels, int pose_frames,
                    cudaGraphExec_t *out)
{
    // the pyramid launch's shared memory depends on the level count
    const auto key = std::make_tuple(frames_p2, cps, slot, pyr_frames, pyr_blocks, pyr_levels, pose_frames);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = it->second;
        return FT_OK;
    }
    // captured on the context's own stream; the graph then runs on any stream
    cudaStream_t cs = ctx->capture_stream;
    cudaGraph_t g = nullptr;
    FT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e1 = cudaMemcpyAsync(table_dev, ctx->staging[slot], copy_bytes, cudaMemcpyHostToDevice, cs);
    const cudaError_t e0 =
        launch_pyramids(reinterpret_cast<const BatchHeader *>(table_dev), pyr_frames, pyr_levels, pyr_blocks, cs);
    cudaError_t e2 = e0 != cudaSuccess ? e0 : launch_fused(reinterpret_cast<const BatchHeader *>(table_dev),
                                                           grid, cs);
    if (e2 == cudaSuccess) e2 = launch_pose(reinterpret_cast<const BatchHeader *>(table_dev), pose_frames, cs);
    const cudaError_t e3 = cudaStreamEndCapture(cs, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(FT_ECUDA, "graph capture failed: %s / %s / %s", cudaGetErrorString(e1),
                    cudaGetErrorString(e2), cudaGetErrorString(e3));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e4 = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) return fail(FT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e4));
    ctx->graphs[key] = exec;
    *out = exec;
    return FT_OK;
}

ft_status submit(ft_ctx *ctx, cudaStream_t stream, const ft_params &params, const std::vector<Job> &jobs,
                 const ft_tuning *force_tuning, bool allow_graph)
{
    ft_status s = check_params(params);
    if (s != FT_OK) return s;
    if ((int)jobs.size() > ctx->max_frames)
        return fail(FT_EINVAL, "%zu frames exceed the context's max_frames %d", jobs.size(), ctx->max_frames);
    for (size_t f = 0; f < jobs.size(); ++f) {
        if ((s = check_job(jobs[f], params)) != FT_OK) {
            g_last_error = "frame " + std::to_string(f) + ": " + g_last_error;
            return s;
        }
    }
    FT_CUDA(cudaSetDevice(ctx->device));
    const Bucket bk = bucket_of(jobs);
    ft_tuning tune = default_tuning();
    if (force_tuning) tune = *force_tuning;
    else {
        auto it = ctx->tuning.find(bk);
        if (it != ctx->tuning.end()) tune = it->second;
    }
    const int slot = ctx->slot;
    ctx->slot = (ctx->slot + 1) % kSlots;
    FT_CUDA(cudaEventSynchronize(ctx->slot_done[slot]));      // staging slot free again
    char *table_dev = ctx->arena + align_up(sizeof(unsigned) * 64);
    size_t bytes = 0;
    int items = 0;
    if ((s = build_table(ctx, params, jobs, tune, ctx->staging[slot], table_dev, &bytes, &items)) != FT_OK)
        return s;
    if ((s = order_stream(ctx, stream)) != FT_OK) return s;
    const int cps = tune.ctas_per_sm > 0 ? std::min(tune.ctas_per_sm, ctx->occ) : ctx->occ;
    const int grid_max = ctx->sm_count * cps;
    // frames that build their pyramids first run the pyramid kernel, one
    // block per level-0 tile of the largest image (the blocks past a smaller
    // image's tiles exit)
    int pyr_frames = 0, pyr_blocks = 1;
    for (size_t f = 0; f < jobs.size(); ++f)
        if (jobs[f].build_pyr) pyr_frames = (int)f + 1;
    if (pyr_frames > 0) {
        int most = 1;
        for (int f = 0; f < pyr_frames; ++f)
            for (int side = 0; side < 2; ++side) {
                if (!(jobs[f].build_pyr & (1 << side))) continue;
                const ft_pyramid &py = side ? jobs[f].pyr_r : jobs[f].pyr_l;
                most = std::max(most, pyr_tiles(py.width[0], py.height[0]));
            }
        pyr_blocks = most;
    }
    // frames that optimize their pose run the pose kernel after the fused
    // kernel, one block per frame up to the last such frame
    int pose_frames = 0;
    for (size_t f = 0; f < jobs.size(); ++f)
        if (jobs[f].do_pose) pose_frames = (int)f + 1;
    if (items > 0 || pyr_frames > 0 || pose_frames > 0) {
        if (allow_graph && ctx->use_graphs && items > 0) {
            const int fp2 = bk.frames_p2;
            const size_t copy = std::max(bytes, table_layout(fp2).total);
            cudaGraphExec_t exec = nullptr;
            if ((s = get_graph(ctx, table_dev, fp2, cps, slot, grid_max, std::min(copy, ctx->table_cap),
                               pyr_frames > 0 ? fp2 : 0, pyr_blocks, params.nlevels, pose_frames > 0 ? fp2 : 0,
                               &exec)) != FT_OK)
                return s;
            FT_CUDA(cudaGraphLaunch(exec, stream));
        } else {
            FT_CUDA(cudaMemcpyAsync(table_dev, ctx->staging[slot], bytes, cudaMemcpyHostToDevice, stream));
            if (pyr_frames > 0)
                FT_CUDA(launch_pyramids(reinterpret_cast<const BatchHeader *>(table_dev), pyr_frames, params.nlevels,
                                        pyr_blocks,
                                        stream));
            if (items > 0)
                FT_CUDA(launch_fused(reinterpret_cast<const BatchHeader *>(table_dev), std::min(items, grid_max),
                                     stream));
            if (pose_frames > 0)
                FT_CUDA(launch_pose(reinterpret_cast<const BatchHeader *>(table_dev), pose_frames, stream));
        }
        ctx->launches += (items > 0 ? 1 : 0) + (pyr_frames > 0 ? 1 : 0) + (pose_frames > 0 ? 1 : 0);
    }
    FT_CUDA(cudaEventRecord(ctx->slot_done[slot], stream));
    return finish_call(ctx, stream);
}

}  // namespace

namespace {

// Popcount-only work for the popcount roofline: eight independent chains of
// 32-bit popcounts per thread (enough to keep the pipe busy), folded into one
// value the kernel writes so that nothing is optimised away.
constexpr int kPopcIters = 4096;

// One 4-byte read every stride_words words (and a second `second` words
// later), folded into a value the kernel writes only if it is impossible.
__global__ void __launch_bounds__(256) scattered_read_kernel(const int *a, long long stride_words, int n,
                                                             int second, int *sink)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    int s = 0;
    if (i < n) {
        const int *p = a + (long long)i * stride_words;
        s = __ldcg(p);
        if (second) s += __ldcg(p + second);
    }
    if (s == 0x7fffffff) sink[0] = s;
}

__global__ void __launch_bounds__(256) popcount_rate_kernel(unsigned seed, unsigned *sink)
{
    unsigned v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = seed * (threadIdx.x + 1u) + 0x9e3779b9u * (unsigned)k + blockIdx.x;
    for (int i = 0; i < kPopcIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = (unsigned)__popc(v[k]) + (v[k] << 1);
    }
    unsigned x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x ^= v[k];
    if (x == 0x12345678u) sink[blockIdx.x & 1023] = x;
}

}  // namespace

void ft::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

// ======================================================================== C ABI
extern "C" {

void ft_params_default(ft_params *p)
{
    if (!p) return;
    p->nlevels = 8;
    p->scale_factor = 1.2f;
    p->th_stereo = 75;
    p->median_factor = 1.5f * 1.4f;
    p->fisheye_ratio = 0.7f;
    p->th_search = 100;
    p->nn_ratio = 0.8f;
    p->ratio_any_octave = 0;
    p->search_th = 1.0f;
    p->view_cos_min = 0.5f;
    p->view_cos_narrow = 0.998f;
    p->radius_narrow = 2.5f;
    p->radius_wide = 4.0f;
    p->dist_lo = 0.8f;
    p->dist_hi = 1.2f;
    p->th_last = 7.0f;
    p->kb_iters = 10;
    p->min_depth = 1e-4f;
    p->po_rounds = 4;
    p->po_iters = 10;
    p->po_chi2_mono = 5.991f;
    p->po_chi2_stereo = 7.815f;
    p->po_huber = 1;
}

const char *ft_last_error(void) { return g_last_error.c_str(); }

ft_status ft_create(ft_ctx **out, const ft_ctx_desc *desc)
{
    if (!out) return fail(FT_EINVAL, "ft_create: out is NULL");
    *out = nullptr;
    ft_ctx_desc d{};
    if (desc) d = *desc;
    if (d.arena_bytes == 0) d.arena_bytes = (size_t)64 << 20;
    if (d.max_frames <= 0) d.max_frames = 256;
    if (d.max_frames > 65536) return fail(FT_EINVAL, "max_frames %d too large", d.max_frames);
    int ndev = 0;
    FT_CUDA(cudaGetDeviceCount(&ndev));
    if (d.device < 0 || d.device >= ndev) return fail(FT_EINVAL, "device %d not present", d.device);
    FT_CUDA(cudaSetDevice(d.device));
    ft_ctx *c = new ft_ctx();
    c->device = d.device;
    c->max_frames = d.max_frames;
    c->use_graphs = d.use_graphs != 0;
    cudaDeviceProp prop{};
    cudaError_t e = cudaGetDeviceProperties(&prop, d.device);
    if (e == cudaSuccess) e = fused_occupancy(&c->occ);
    if (e == cudaSuccess) e = pyramid_setup();
    c->sm_count = prop.multiProcessorCount;
    if (c->occ < 1) c->occ = 1;
    // the table region holds a batch table of max_frames frames or an
    // extraction table of 4 x max_frames images
    c->table_cap = std::max(table_layout(d.max_frames).total, orb_table_bytes(4 * d.max_frames));
    const size_t head = align_up(sizeof(unsigned) * 64);
    c->scratch_off = align_up(head + c->table_cap);
    c->arena_bytes = std::max(d.arena_bytes, c->scratch_off + ((size_t)1 << 20));
    if (e == cudaSuccess) e = cudaMalloc(&c->arena, c->arena_bytes);
    if (e == cudaSuccess) {
        c->status = reinterpret_cast<unsigned *>(c->arena);
        e = cudaMemset(c->arena, 0, head);
    }
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&c->staging[i], c->table_cap);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->slot_done[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ft_destroy(c);
        return fail(e == cudaErrorMemoryAllocation ? FT_ENOMEM : FT_ECUDA, "ft_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return FT_OK;
}

void ft_destroy(ft_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    for (int i = 0; i < kSlots; ++i) {
        if (c->staging[i]) cudaFreeHost(c->staging[i]);
        if (c->slot_done[i]) cudaEventDestroy(c->slot_done[i]);
    }
    if (c->done) cudaEventDestroy(c->done);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->arena) cudaFree(c->arena);
    if (c->trace) cudaFree(c->trace);
    delete c;
}

ft_status ft_sync_status(ft_ctx *c, int32_t *status)
{
    if (!c || !status) return fail(FT_EINVAL, "ft_sync_status: NULL argument");
    FT_CUDA(cudaSetDevice(c->device));
    if (c->have_last) FT_CUDA(cudaStreamSynchronize(c->last_stream));
    unsigned v = 0;
    FT_CUDA(cudaMemcpy(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost));
    FT_CUDA(cudaMemset(c->status, 0, sizeof(unsigned)));
    *status = (v & kStatusTimeout) ? FT_ETIMEOUT : FT_OK;
    return FT_OK;
}

uint64_t ft_launch_count(ft_ctx *c) { return c ? c->launches : 0; }

ft_status ft_set_trace(ft_ctx *c, int capacity)
{
    if (!c || capacity < 0) return fail(FT_EINVAL, "ft_set_trace: bad argument");
    FT_CUDA(cudaSetDevice(c->device));
    if (c->have_last) FT_CUDA(cudaStreamSynchronize(c->last_stream));
    if (c->trace) {
        FT_CUDA(cudaFree(c->trace));
        c->trace = nullptr;
        c->trace_cap = 0;
    }
    if (capacity > 0) {
        FT_CUDA(cudaMalloc(&c->trace, sizeof(ft_trace_record) * (size_t)capacity));
        c->trace_cap = capacity;
    }
    return FT_OK;
}

ft_status ft_read_trace(ft_ctx *c, ft_trace_record *out, int max, int *n)
{
    if (!c || !n || (max > 0 && !out)) return fail(FT_EINVAL, "ft_read_trace: bad argument");
    FT_CUDA(cudaSetDevice(c->device));
    if (c->have_last) FT_CUDA(cudaStreamSynchronize(c->last_stream));
    unsigned cnt = 0;
    const char *queue = c->arena + align_up(sizeof(unsigned) * 64) + table_layout(1).queue;
    FT_CUDA(cudaMemcpy(&cnt, queue + sizeof(unsigned), sizeof(unsigned), cudaMemcpyDeviceToHost));
    *n = (int)cnt;
    const int k = std::min<int>(std::min<unsigned>(cnt, (unsigned)c->trace_cap), max);
    if (k > 0 && c->trace)
        FT_CUDA(cudaMemcpy(out, c->trace, sizeof(ft_trace_record) * (size_t)k, cudaMemcpyDeviceToHost));
    return FT_OK;
}

ft_status ft_set_debug(ft_ctx *c, unsigned flags, uint64_t timeout_ns)
{
    if (!c) return fail(FT_EINVAL, "ft_set_debug: NULL context");
    c->debug_flags = flags;
    c->timeout_ns = timeout_ns ? timeout_ns : 2000000000ull;
    return FT_OK;
}

ft_status ft_stereo_match_pinhole(ft_ctx *ctx, void *stream, const ft_params *params,
                                  const ft_pinhole *cam, const ft_stereo_frame *frame, ft_stereo_out *out)
{
    if (!ctx || !cam || !frame || !out) return fail(FT_EINVAL, "ft_stereo_match_pinhole: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = FT_CAMERA_PINHOLE;
    j.do_stereo = true;
    j.pin = *cam;
    j.left = frame->left;
    j.right = frame->right;
    j.pyr_l = frame->pyr_left;
    j.pyr_r = frame->pyr_right;
    j.st = *out;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_stereo_match_fisheye(ft_ctx *ctx, void *stream, const ft_params *params,
                                  const ft_fisheye_rig *rig, const ft_keypoints *left,
                                  const ft_keypoints *right, ft_fisheye_out *out)
{
    if (!ctx || !rig || !left || !right || !out) return fail(FT_EINVAL, "ft_stereo_match_fisheye: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = FT_CAMERA_FISHEYE;
    j.do_stereo = true;
    j.rig = *rig;
    j.left = *left;
    j.right = *right;
    j.fo = *out;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_search_local_points(ft_ctx *ctx, void *stream, const ft_params *params,
                                 const ft_frame_view *frame, const ft_pose *Tcw, const ft_map_view *map,
                                 ft_search_out *out)
{
    if (!ctx || !frame || !Tcw || !map || !out) return fail(FT_EINVAL, "ft_search_local_points: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = frame->camera;
    j.do_search = true;
    j.pin = frame->pinhole;
    j.rig = frame->fisheye;
    j.left = frame->left;
    j.right = frame->right;
    j.u_right_in = frame->u_right;
    j.taken_l = frame->taken_left;
    j.taken_r = frame->taken_right;
    j.pose = *Tcw;
    for (int i = 0; i < 3; ++i) j.O_right[i] = frame->O_right[i];
    j.map = *map;
    j.so = *out;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_search_last_frame(ft_ctx *ctx, void *stream, const ft_params *params,
                               const ft_frame_view *frame, const ft_pose *Tcw, const ft_last_frame_view *last,
                               ft_search_out *out)
{
    if (!ctx || !frame || !Tcw || !last || !out) return fail(FT_EINVAL, "ft_search_last_frame: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = frame->camera;
    j.do_search = true;
    j.pin = frame->pinhole;
    j.rig = frame->fisheye;
    j.left = frame->left;
    j.right = frame->right;
    j.u_right_in = frame->u_right;
    j.taken_l = frame->taken_left;
    j.taken_r = frame->taken_right;
    j.pose = *Tcw;
    for (int i = 0; i < 3; ++i) j.O_right[i] = frame->O_right[i];
    set_last(j, *last);
    j.so = *out;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_optimize_pose(ft_ctx *ctx, void *stream, const ft_params *params, const ft_frame_view *frame,
                           const ft_pose *Tcw, const ft_map_view *map, const int32_t *mp_kp, const ft_pose_out *out)
{
    if (!ctx || !frame || !Tcw || !map || !out) return fail(FT_EINVAL, "ft_optimize_pose: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = frame->camera;
    j.do_pose = true;
    j.pin = frame->pinhole;
    j.left = frame->left;
    j.u_right_in = frame->u_right;
    j.pose = *Tcw;
    j.map = *map;
    j.po = *out;
    j.po_mp_kp = mp_kp;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_extract_orb(ft_ctx *ctx, void *stream, const ft_params *params, int n, const ft_pyramid *pyr,
                         const ft_orb_params *orb, const ft_orb_out *out)
{
    if (!ctx || !orb || (n > 0 && (!pyr || !out))) return fail(FT_EINVAL, "ft_extract_orb: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    ft_status s = check_params(p);
    if (s != FT_OK) return s;
    if (n < 0 || n > 4 * std::max(ctx->max_frames, 1)) return fail(FT_EINVAL, "ft_extract_orb: n=%d out of range", n);
    if (orb->fast_th < 1 || orb->fast_th > 254) return fail(FT_EINVAL, "fast_th %d out of [1, 254]", orb->fast_th);
    if (orb->edge < 19 || orb->edge > kOrbMaxDim) return fail(FT_EINVAL, "edge %d below 19", orb->edge);
    if (!orb->pattern) return fail(FT_EINVAL, "ft_extract_orb: NULL pattern");
    for (int i = 0; i < 256 * 4; ++i)
        if (orb->pattern[i] < -13 || orb->pattern[i] > 13)
            return fail(FT_EINVAL, "pattern coordinate %d outside [-13, 13]", (int)orb->pattern[i]);
    int nslots = 0;
    for (int l = 0; l < p.nlevels; ++l) {
        if (orb->max_kp[l] < 0 || orb->max_kp[l] > kOrbMaxSlots)
            return fail(FT_EINVAL, "max_kp[%d] = %d out of [0, %d]", l, orb->max_kp[l], kOrbMaxSlots);
        nslots += orb->max_kp[l];
    }
    for (int i = 0; i < n; ++i) {
        if ((s = check_pyramid(pyr[i], p.nlevels, "pyramid")) != FT_OK) return s;
        for (int l = 0; l < p.nlevels; ++l)
            if (pyr[i].width[l] > kOrbMaxDim || pyr[i].height[l] > kOrbMaxDim)
                return fail(FT_EINVAL, "image %d level %d is larger than %d x %d", i, l, kOrbMaxDim, kOrbMaxDim);
        const ft_orb_out &o = out[i];
        if (!o.n_level || (nslots > 0 && (!o.x || !o.y || !o.oct || !o.score || !o.cs || !o.desc)))
            return fail(FT_EINVAL, "image %d: NULL output array", i);
        if (!aligned16(o.desc)) return fail(FT_EALIGN, "image %d: desc not 16-byte aligned", i);
    }
    // table: header, images, per-image counters (zeroed here)
    const size_t o_img = align_up(sizeof(OrbHeader));
    const size_t o_cnt = align_up(o_img + sizeof(OrbImage) * (size_t)std::max(n, 1));
    const size_t bytes = orb_table_bytes(n);
    if (bytes > ctx->table_cap) return fail(FT_ENOMEM, "extraction table of %d images exceeds the context", n);
    FT_CUDA(cudaSetDevice(ctx->device));
    const int slot = ctx->slot;
    ctx->slot = (ctx->slot + 1) % kSlots;
    FT_CUDA(cudaEventSynchronize(ctx->slot_done[slot]));
    char *h = ctx->staging[slot];
    char *dev = ctx->arena + align_up(sizeof(unsigned) * 64);
    std::memset(h, 0, bytes);
    OrbHeader &Hd = *reinterpret_cast<OrbHeader *>(h);
    Hd.nimages = n;
    Hd.nlevels = p.nlevels;
    Hd.fast_th = orb->fast_th;
    Hd.edge = orb->edge;
    const DevParams dp = make_dev_params(p);
    for (int l = 0; l < FT_MAX_LEVELS; ++l) Hd.sc[l] = dp.sc[l];
    std::memcpy(Hd.pattern, orb->pattern, sizeof(Hd.pattern));
    Hd.images = reinterpret_cast<const OrbImage *>(dev + o_img);
    size_t scratch = ctx->scratch_off;
    auto carve = [&](size_t b) -> char * {
        char *q = ctx->arena + scratch;
        scratch = align_up(scratch + std::max<size_t>(b, 1));
        return q;
    };
    int max_tiles = 0;
    for (int i = 0; i < n; ++i) {
        OrbImage &I = reinterpret_cast<OrbImage *>(h + o_img)[i];
        const ft_orb_out &o = out[i];
        int tiles = 0, slot0 = 0;
        for (int l = 0; l < p.nlevels; ++l) {
            OrbLevel &L = I.lv[l];
            L.img = pyr[i].data[l];
            L.w = pyr[i].width[l];
            L.h = pyr[i].height[l];
            L.pitch = pyr[i].pitch[l];
            L.spitch = (L.w + 15) & ~15;
            L.smooth = reinterpret_cast<uint8_t *>(carve((size_t)L.spitch * L.h));
            // suppressed corners are never 8-neighbours: at most one per 2 x 2 block
            L.cand_cap = ((L.w + 1) / 2) * ((L.h + 1) / 2);
            L.cand = reinterpret_cast<unsigned *>(carve(sizeof(unsigned) * (size_t)L.cand_cap));
            L.tiles_x = (L.w + kOrbTile - 1) / kOrbTile;
            L.tile0 = tiles;
            tiles += L.tiles_x * ((L.h + kOrbTile - 1) / kOrbTile);
            L.slot0 = slot0;
            L.max_kp = orb->max_kp[l];
            slot0 += L.max_kp;
        }
        I.tiles = tiles;
        I.nslots = nslots;
        I.x = o.x;
        I.y = o.y;
        I.oct = o.oct;
        I.score = o.score;
        I.cs = o.cs;
        I.desc = o.desc;
        I.n_level = o.n_level;
        I.sel = reinterpret_cast<unsigned *>(carve(sizeof(unsigned) * (size_t)std::max(nslots, 1)));
        I.cnt = reinterpret_cast<unsigned *>(dev + o_cnt) + (size_t)FT_MAX_LEVELS * i;
        max_tiles = std::max(max_tiles, tiles);
    }
    Hd.max_tiles = max_tiles;
    Hd.max_slots = nslots;
    if (scratch > ctx->arena_bytes)
        return fail(FT_ENOMEM, "arena of %zu bytes too small for this extraction (needs %zu)", ctx->arena_bytes,
                    scratch);
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = order_stream(ctx, st)) != FT_OK) return s;
    if (n > 0) {
        FT_CUDA(cudaMemcpyAsync(dev, h, bytes, cudaMemcpyHostToDevice, st));
        FT_CUDA(launch_orb(reinterpret_cast<const OrbHeader *>(dev), n, p.nlevels, max_tiles, nslots, st));
        ctx->launches += 3;
    }
    FT_CUDA(cudaEventRecord(ctx->slot_done[slot], st));
    return finish_call(ctx, st);
}

ft_status ft_pyramid_sizes(int width, int height, const ft_params *params, int *w, int *h)
{
    if (!w || !h || width <= 0 || height <= 0) return fail(FT_EINVAL, "ft_pyramid_sizes: bad argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    ft_status s = check_params(p);
    if (s != FT_OK) return s;
    pyramid_sizes(width, height, p, w, h);
    return FT_OK;
}

ft_status ft_measure_popcount(void *stream, double *popc_per_s)
{
    if (!popc_per_s) return fail(FT_EINVAL, "ft_measure_popcount: NULL argument");
    int dev = 0, sms = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *sink = nullptr;
    FT_CUDA(cudaMalloc(&sink, 1024 * sizeof(unsigned)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * 8;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // the first run warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) popcount_rate_kernel<<<blocks, 256, 0, st>>>(0x2545f491u + rep, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best_ms = std::min(best_ms, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(FT_ECUDA, "ft_measure_popcount: %s", cudaGetErrorString(e));
    *popc_per_s = (double)blocks * 256.0 * kPopcIters * 8.0 / (best_ms * 1e-3);
    return FT_OK;
}

ft_status ft_scattered_reads(void *stream, int stride_bytes, int second_bytes, int *accesses)
{
    if (!accesses) return fail(FT_EINVAL, "ft_scattered_reads: NULL argument");
    if (stride_bytes < 256 || (stride_bytes & 3) || second_bytes < 0 || (second_bytes & 3) ||
        second_bytes >= stride_bytes)
        return fail(FT_EINVAL, "ft_scattered_reads: stride %d, second read at %d", stride_bytes, second_bytes);
    const size_t bytes = (size_t)1 << 30;
    const int n = (int)(bytes / (size_t)stride_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    int *a = nullptr, *sink = nullptr;
    FT_CUDA(cudaMalloc(&a, bytes));
    cudaError_t e = cudaMalloc(&sink, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 1, bytes, st);
    if (e == cudaSuccess) {
        // the last read: (n - 1) * stride + second + 4 <= n * stride <= 1 GiB
        scattered_read_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, stride_bytes / 4, n, second_bytes / 4, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(a);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return fail(FT_ECUDA, "ft_scattered_reads: %s", cudaGetErrorString(e));
    *accesses = n;
    return FT_OK;
}

ft_status ft_build_pyramid(ft_ctx *ctx, void *stream, const ft_params *params, const ft_pyramid *pyr)
{
    if (!ctx || !pyr) return fail(FT_EINVAL, "ft_build_pyramid: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    Job j;
    j.camera = FT_CAMERA_PINHOLE;
    j.build_pyr = 1;           // one image: the left side names it
    j.pin.width = pyr->width[0];
    j.pin.height = pyr->height[0];
    j.pyr_l = *pyr;
    j.pyr_r = *pyr;
    return submit(ctx, (cudaStream_t)stream, p, {j}, nullptr, false);
}

ft_status ft_build_pyramids(ft_ctx *ctx, void *stream, const ft_params *params, int n, const ft_pyramid *pyr)
{
    if (!ctx || (n > 0 && !pyr)) return fail(FT_EINVAL, "ft_build_pyramids: NULL argument");
    if (n < 0 || (n + 1) / 2 > ctx->max_frames)
        return fail(FT_EINVAL, "ft_build_pyramids: %d images exceed the context (2 x max_frames)", n);
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    // two images per job: the pyramid kernel builds a job's left and right
    std::vector<Job> jobs((n + 1) / 2);
    for (int i = 0; i < n; i += 2) {
        Job &j = jobs[i / 2];
        j.camera = FT_CAMERA_PINHOLE;
        j.pin.width = pyr[i].width[0];
        j.pin.height = pyr[i].height[0];
        j.pyr_l = pyr[i];
        j.pyr_r = i + 1 < n ? pyr[i + 1] : pyr[i];
        j.build_pyr = i + 1 < n ? 3 : 1;
    }
    return submit(ctx, (cudaStream_t)stream, p, jobs, nullptr, false);
}

static ft_status jobs_of_batch(const ft_batch *batch, std::vector<Job> &jobs)
{
    if (!batch || batch->n < 0 || (batch->n > 0 && !batch->frames))
        return fail(FT_EINVAL, "batch: bad frame list");
    jobs.resize(batch->n);
    for (int f = 0; f < batch->n; ++f) {
        const ft_frame_job &s = batch->frames[f];
        Job &j = jobs[f];
        j.camera = s.camera;
        j.do_stereo = true;
        j.do_search = true;
        j.wait_stereo = s.camera == FT_CAMERA_PINHOLE;
        j.pin = s.pinhole;
        j.rig = s.fisheye;
        j.left = s.left;
        j.right = s.right;
        j.pyr_l = s.pyr_left;
        j.pyr_r = s.pyr_right;
        j.taken_l = s.taken_left;
        j.taken_r = s.taken_right;
        j.pose = s.pose;
        for (int i = 0; i < 3; ++i) j.O_right[i] = s.O_right[i];
        j.map = s.map;
        j.st = s.stereo;
        j.fo = s.fisheye_out;
        j.so = s.search;
        j.u_right_in = s.camera == FT_CAMERA_PINHOLE ? s.stereo.u_right : nullptr;
        if (s.last) set_last(j, *s.last);
        j.build_pyr = s.build_pyramids != 0 ? 3 : 0;
        if (s.pose_out) {
            j.do_pose = true;
            j.po = *s.pose_out;
        }
    }
    return FT_OK;
}

ft_status ft_track_batch(ft_ctx *ctx, void *stream, const ft_params *params, const ft_batch *batch)
{
    if (!ctx || !batch) return fail(FT_EINVAL, "ft_track_batch: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    std::vector<Job> jobs;
    ft_status s = jobs_of_batch(batch, jobs);
    if (s != FT_OK) return s;
    if (batch->stage_in_bytes && (!batch->stage_in_host || !batch->stage_in_dev))
        return fail(FT_EINVAL, "batch: stage-in buffers missing");
    if (batch->stage_out_bytes && (!batch->stage_out_host || !batch->stage_out_dev))
        return fail(FT_EINVAL, "batch: stage-out buffers missing");
    cudaStream_t st = (cudaStream_t)stream;
    FT_CUDA(cudaSetDevice(ctx->device));
    if (batch->stage_in_bytes) {
        if ((s = order_stream(ctx, st)) != FT_OK) return s;
        FT_CUDA(cudaMemcpyAsync(batch->stage_in_dev, batch->stage_in_host, batch->stage_in_bytes,
                                cudaMemcpyHostToDevice, st));
    }
    if ((s = submit(ctx, st, p, jobs, nullptr, true)) != FT_OK) return s;
    if (batch->stage_out_bytes)
        FT_CUDA(cudaMemcpyAsync(batch->stage_out_host, batch->stage_out_dev, batch->stage_out_bytes,
                                cudaMemcpyDeviceToHost, st));
    return FT_OK;
}

ft_status ft_set_tuning(ft_ctx *ctx, const ft_batch *batch, const ft_tuning *t)
{
    if (!ctx || !batch || !t) return fail(FT_EINVAL, "ft_set_tuning: NULL argument");
    std::vector<Job> jobs;
    ft_status s = jobs_of_batch(batch, jobs);
    if (s != FT_OK) return s;
    ctx->tuning[bucket_of(jobs)] = *t;
    return FT_OK;
}

ft_status ft_get_tuning(ft_ctx *ctx, const ft_batch *batch, ft_tuning *t)
{
    if (!ctx || !batch || !t) return fail(FT_EINVAL, "ft_get_tuning: NULL argument");
    std::vector<Job> jobs;
    ft_status s = jobs_of_batch(batch, jobs);
    if (s != FT_OK) return s;
    auto it = ctx->tuning.find(bucket_of(jobs));
    *t = it != ctx->tuning.end() ? it->second : default_tuning();
    return FT_OK;
}

// The launch shapes both autotuners try: strip rows 16/32/64, search tile
// 256/512/1024, fisheye tile 64/128, every count of CTAs per SM from the
// resident maximum down to one (fewer leave room for a concurrent launch),
// both search staging modes and the search in one pass or two halves.
static std::vector<ft_tuning> tuning_candidates(int occ)
{
    const int strips[] = {16, 32, 64};
    const int tiles[] = {256, 512, 1024};
    const int fish[] = {64, 128};
    std::vector<int> occs;
    for (int o = std::max(1, occ); o >= 1; --o) occs.push_back(o);
    std::vector<ft_tuning> cand;
    for (int a : strips)
        for (int b : tiles)
            for (int c : fish)
                for (int o : occs)
                    for (int st = 0; st < 2; ++st)
                        for (int sp : {1, -1}) {
                            ft_tuning t = default_tuning();
                            t.strip_rows = a;
                            t.search_tile = b;
                            t.fisheye_tile = c;
                            t.ctas_per_sm = o;
                            t.search_stage = st;
                            t.split_search = sp;
                            cand.push_back(t);
                        }
    return cand;
}

ft_status ft_autotune(ft_ctx *ctx, void *stream, const ft_params *params, const ft_batch *batch, int iters,
                      ft_tuning *best)
{
    if (!ctx || !batch) return fail(FT_EINVAL, "ft_autotune: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    std::vector<Job> jobs;
    ft_status s = jobs_of_batch(batch, jobs);
    if (s != FT_OK) return s;
    if (iters < 1) iters = 3;
    cudaStream_t st = (cudaStream_t)stream;
    FT_CUDA(cudaSetDevice(ctx->device));
    // Two rounds: every candidate is timed launch by launch (after one
    // untimed launch) and ranked by its median; the four best are then
    // re-timed in turn, four times as often, so that clock drift and one-off
    // delays do not pick the winner.
    const std::vector<ft_tuning> cand = tuning_candidates(ctx->occ);
    const int slots = 4 * iters;
    std::vector<cudaEvent_t> ev(2 * (size_t)slots, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return fail(FT_ECUDA, "autotune: cannot create events");
        }
    // times n launches of candidate t, one after another; the median in ms
    auto time_one = [&](const ft_tuning &t, int n, float *med) -> ft_status {
        ft_status r;
        for (int i = 0; i < n; ++i) {
            cudaEventRecord(ev[2 * i], st);
            if ((r = submit(ctx, st, p, jobs, &t, false)) != FT_OK) return r;
            cudaEventRecord(ev[2 * i + 1], st);
        }
        if (cudaEventSynchronize(ev[2 * n - 1]) != cudaSuccess) return fail(FT_ECUDA, "autotune: event sync failed");
        std::vector<float> ms((size_t)n);
        for (int i = 0; i < n; ++i) cudaEventElapsedTime(&ms[i], ev[2 * i], ev[2 * i + 1]);
        std::nth_element(ms.begin(), ms.begin() + n / 2, ms.end());
        *med = ms[n / 2];
        return FT_OK;
    };
    std::vector<std::pair<float, int>> score;
    for (size_t k = 0; k < cand.size() && s == FT_OK; ++k) {
        float med = 0;
        if ((s = submit(ctx, st, p, jobs, &cand[k], false)) != FT_OK) break;
        if ((s = time_one(cand[k], iters, &med)) != FT_OK) break;
        score.push_back({med, (int)k});
    }
    if (s == FT_OK) {
        std::sort(score.begin(), score.end());
        const int top = std::min<int>(4, (int)score.size());
        std::vector<std::vector<float>> again((size_t)top);
        for (int round = 0; round < 4 * iters && s == FT_OK; ++round)
            for (int q = 0; q < top && s == FT_OK; ++q) {
                float med = 0;
                if ((s = time_one(cand[score[q].second], 1, &med)) == FT_OK) again[q].push_back(med);
            }
        if (s == FT_OK) {
            int win = 0;
            float win_ms = 1e30f;
            for (int q = 0; q < top; ++q) {
                auto &v = again[q];
                std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
                if (v[v.size() / 2] < win_ms) {
                    win_ms = v[v.size() / 2];
                    win = score[q].second;
                }
            }
            ctx->tuning[bucket_of(jobs)] = cand[win];
            if (best) *best = cand[win];
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return s;
}

ft_status ft_autotune_stream(ft_ctx *const *ctxs, void *const *streams, int n, const ft_params *params,
                             const ft_batch *const *batches, int iters, ft_tuning *best)
{
    if (!ctxs || !streams || !batches || n < 2 || n > 16) return fail(FT_EINVAL, "ft_autotune_stream: bad argument");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !batches[i]) return fail(FT_EINVAL, "ft_autotune_stream: NULL context or batch %d", i);
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(FT_EINVAL, "ft_autotune_stream: contexts on different devices");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(FT_EINVAL, "ft_autotune_stream: context %d given twice", i);
    }
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    std::vector<std::vector<Job>> jobs((size_t)n);
    ft_status s = FT_OK;
    for (int i = 0; i < n && s == FT_OK; ++i) s = jobs_of_batch(batches[i], jobs[(size_t)i]);
    if (s != FT_OK) return s;
    const Bucket bk = bucket_of(jobs[0]);
    int occ = ctxs[0]->occ;
    for (int i = 1; i < n; ++i) {
        const Bucket bi = bucket_of(jobs[(size_t)i]);
        if (bk < bi || bi < bk) return fail(FT_EINVAL, "ft_autotune_stream: batches fall in different buckets");
        occ = std::min(occ, ctxs[i]->occ);
    }
    if (iters < 1) iters = 3;
    FT_CUDA(cudaSetDevice(ctxs[0]->device));
    // the same candidates as ft_autotune; a candidate's score is the time of
    // a run of launches taken by the contexts in turn, divided by the
    // launches (the form where later launches fill earlier ones' tails)
    const std::vector<ft_tuning> cand = tuning_candidates(occ);
    std::vector<cudaEvent_t> ev((size_t)n + 1, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return fail(FT_ECUDA, "autotune: cannot create events");
        }
    cudaStream_t s0 = (cudaStream_t)streams[0];
    auto run = [&](const ft_tuning &t, int launches, float *per_launch_ms) -> ft_status {
        ft_status r;
        if (cudaEventRecord(ev[0], s0) != cudaSuccess) return fail(FT_ECUDA, "autotune: event record failed");
        for (int i = 1; i < n; ++i)
            if (cudaStreamWaitEvent((cudaStream_t)streams[i], ev[0], 0) != cudaSuccess)
                return fail(FT_ECUDA, "autotune: stream wait failed");
        for (int i = 0; i < launches; ++i) {
            const int c = i % n;
            if ((r = submit(ctxs[c], (cudaStream_t)streams[c], p, jobs[(size_t)c], &t, false)) != FT_OK) return r;
        }
        for (int i = 1; i < n; ++i)
            if (cudaEventRecord(ev[(size_t)i], (cudaStream_t)streams[i]) != cudaSuccess ||
                cudaStreamWaitEvent(s0, ev[(size_t)i], 0) != cudaSuccess)
                return fail(FT_ECUDA, "autotune: event record failed");
        if (cudaEventRecord(ev[(size_t)n], s0) != cudaSuccess || cudaEventSynchronize(ev[(size_t)n]) != cudaSuccess)
            return fail(FT_ECUDA, "autotune: event sync failed");
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[(size_t)n]);
        *per_launch_ms = ms / (float)launches;
        return FT_OK;
    };
    std::vector<std::pair<float, int>> score;
    for (size_t k = 0; k < cand.size() && s == FT_OK; ++k) {
        float ms = 0;
        if ((s = run(cand[k], n, &ms)) != FT_OK) break;              // untimed: the first launches of a shape
        if ((s = run(cand[k], 4 * iters * n, &ms)) != FT_OK) break;
        score.push_back({ms, (int)k});
    }
    if (s == FT_OK) {
        // the four best again, in turn, each run four times as long
        std::sort(score.begin(), score.end());
        const int top = std::min<int>(4, (int)score.size());
        std::vector<float> again((size_t)top, 0.0f);
        for (int round = 0; round < 3 && s == FT_OK; ++round)
            for (int q = 0; q < top && s == FT_OK; ++q) {
                float ms = 0;
                if ((s = run(cand[score[q].second], 16 * iters * n, &ms)) == FT_OK) again[q] += ms;
            }
        if (s == FT_OK) {
            int win = score[0].second;
            float win_ms = 1e30f;
            for (int q = 0; q < top; ++q)
                if (again[q] < win_ms) {
                    win_ms = again[q];
                    win = score[q].second;
                }
            for (int i = 0; i < n; ++i) ctxs[i]->tuning[bk] = cand[win];
            if (best) *best = cand[win];
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return s;
}

ft_status ft_save_tuning(ft_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(FT_EINVAL, "ft_save_tuning: NULL argument");
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(FT_EINVAL, "cannot write %s", path);
    std::fprintf(f, "# frames_p2 has_pinhole has_fisheye nl_p2 m_p2 strip_rows search_tile fisheye_tile resolve_tile "
                    "ctas_per_sm search_stage split_search\n");
    for (auto &kv : ctx->tuning) {
        const Bucket &b = kv.first;
        const ft_tuning &t = kv.second;
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d\n", b.frames_p2, b.has_pinhole, b.has_fisheye,
                     b.nl_p2, b.m_p2, t.strip_rows, t.search_tile, t.fisheye_tile, t.resolve_tile, t.ctas_per_sm,
                     t.search_stage, t.split_search);
    }
    std::fclose(f);
    return FT_OK;
}

ft_status ft_load_tuning(ft_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(FT_EINVAL, "ft_load_tuning: NULL argument");
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(FT_EINVAL, "cannot read %s", path);
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        Bucket b{};
        ft_tuning t{};
        // lines without the last columns (search_stage, split_search) come
        // from older tables: 0 for each
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d", &b.frames_p2, &b.has_pinhole,
                                    &b.has_fisheye, &b.nl_p2, &b.m_p2, &t.strip_rows, &t.search_tile,
                                    &t.fisheye_tile, &t.resolve_tile, &t.ctas_per_sm, &t.search_stage,
                                    &t.split_search);
        if (got >= 10 && got <= 12) ctx->tuning[b] = t;
    }
    std::fclose(f);
    return FT_OK;
}

}  // extern "C"
