// ft_noalloc.cu -- pinhole stereo matching of one frame that allocates no
// memory at all: ft_stereo_match_pinhole_noalloc.
//
// Who needs it: callers that must not allocate device memory once they are
// running.  A tracking thread with a hard per-frame deadline cannot afford
// cudaMalloc (it can block and synchronize the device), an embedded
// deployment may reserve all device memory for itself at start-up, and a
// host framework with its own memory manager may forbid allocations behind
// its back.  Such callers cannot create an ft_ctx, because ft_create
// allocates the arena.  This entry point keeps its scratch (the work table,
// the completion counters and the per-frame row sort) in a fixed-size device
// array that is part of the loaded library instead.
//
// The scratch array exists once per device that loads the library and stays
// allocated until the process exits.  All calls share it: a call overwrites
// what the previous call left there, so calls whose GPU work overlaps (for
// example on two streams at once) race and give wrong results; issue them
// on one stream or order them.  The work table, the counters and the status
// word are uploaded zeroed with every call; the row-sort buffers are fully
// rewritten before they are read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "ft_internal.h"

using namespace ft;

namespace {

// Maximum sizes accepted by the allocation-free path.
constexpr int kNoAllocMaxKeypoints = 16384;     // per image (left and right each)
constexpr int kNoAllocMaxRows = kMaxRows;       // level-0 image height
constexpr size_t kNoAllocScratchBytes = (size_t)2 << 20;
constexpr int kMaxDevices = 64;

// The scratch memory: 2 MiB per device, resident from library load to exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int grid = 0;                       // persistent CTAs (SMs x resident CTAs per SM)
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// errors are reported through ft_last_error(), like every other entry point
ft_status fail(ft_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Once per device, with that device current: resolve the array's device
// address (host code cannot use the symbol itself as a device pointer) and
// the launch shape of the fused kernel.
ft_status setup_device(int dev, DeviceSetup **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(FT_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &S = g_setup[dev];
    if (!S.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(FT_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        int per_sm = 0, sms = 0;
        e = fused_occupancy(&per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(FT_ECUDA, "device set-up: %s", cudaGetErrorString(e));
        S.scratch = static_cast<unsigned char *>(ptr);
        S.grid = std::max(1, sms * std::max(1, per_sm));
        S.ready = true;
    }
    *out = &S;
    return FT_OK;
}

}  // namespace

extern "C" {

ft_status ft_stereo_match_pinhole_noalloc(void *stream, const ft_params *params, const ft_pinhole *cam,
                                          const ft_stereo_frame *frame, ft_stereo_out *out,
                                          int32_t *device_status)
{
    if (!cam || !frame || !out) return fail(FT_EINVAL, "ft_stereo_match_pinhole_noalloc: NULL argument");
    ft_params p;
    if (params) p = *params;
    else ft_params_default(&p);
    // the same parameter checks as every context entry point
    const ft_status pst = check_params(p);
    if (pst != FT_OK) return pst;
    const ft_keypoints &L = frame->left, &R = frame->right;
    if (L.n < 0 || R.n < 0) return fail(FT_EINVAL, "negative keypoint count");
    if (L.n > kNoAllocMaxKeypoints || R.n > kNoAllocMaxKeypoints)
        return fail(FT_EINVAL, "%d left / %d right keypoints exceed the allocation-free limit of %d per image",
                    L.n, R.n, kNoAllocMaxKeypoints);
    if (cam->height <= 0 || cam->width <= 0) return fail(FT_EINVAL, "bad image size");
    if (cam->height > kNoAllocMaxRows)
        return fail(FT_EINVAL, "%d rows exceed the allocation-free limit of %d", cam->height, kNoAllocMaxRows);
    if (!(cam->b > 0.0f)) return fail(FT_EINVAL, "baseline must be > 0");
    const ft_keypoints *kk[2] = {&L, &R};
    for (const ft_keypoints *k : kk) {
        if (k->n == 0) continue;
        if (!k->x || !k->y || !k->oct || !k->desc) return fail(FT_EINVAL, "NULL keypoint array");
        if (reinterpret_cast<uintptr_t>(k->desc) & 15u) return fail(FT_EALIGN, "descriptors not 16-byte aligned");
    }
    const ft_pyramid *pp[2] = {&frame->pyr_left, &frame->pyr_right};
    for (const ft_pyramid *py : pp) {
        if (py->nlevels < p.nlevels) return fail(FT_EINVAL, "pyramid has too few levels");
        for (int l = 0; l < p.nlevels; ++l)
            if (!py->data[l] || py->width[l] <= 0 || py->height[l] <= 0 || py->pitch[l] < py->width[l])
                return fail(FT_EINVAL, "pyramid level %d is missing or has a bad size", l);
            else if ((reinterpret_cast<uintptr_t>(py->data[l]) & 15u) || (py->pitch[l] & 15))
                return fail(FT_EALIGN, "pyramid level %d needs a 16-byte aligned pointer and pitch", l);
    }
    if (L.n > 0 && (!out->best_r || !out->dist || !out->sad_shift || !out->sad_best || !out->u_right || !out->depth))
        return fail(FT_EINVAL, "NULL output array");

    // The work table is copied from a stack buffer (pageable memory), which a
    // stream capture cannot record: refuse a capturing stream up front rather
    // than fail in the middle of the caller's capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) return fail(FT_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(FT_EINVAL, "ft_stereo_match_pinhole_noalloc: the stream is capturing");

    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    DeviceSetup *S = nullptr;
    ft_status st = setup_device(dev, &S);
    if (st != FT_OK) return st;

    // Scratch layout: [work table | row pointers | row-sorted keypoints].
    const int H = cam->height;
    size_t off = 0;
    const size_t o_hdr = off;
    off = up256(off + sizeof(BatchHeader));
    const size_t o_queue = off;                         // queue head, trace count, status word
    off = up256(off + 64);
    const size_t o_ctr = off;
    off = up256(off + sizeof(unsigned) * kCounters);
    const size_t o_prefix = off;
    off = up256(off + sizeof(int) * K_KINDS * 2);
    const size_t o_frame = off;
    off = up256(off + sizeof(FrameDev));
    const size_t table_bytes = off;
    const size_t o_rpl = off;
    off = up256(off + sizeof(int) * (size_t)(H + 1));
    const size_t o_rpr = off;
    off = up256(off + sizeof(int) * (size_t)(H + 1));
    const size_t o_lkp = off;
    off = up256(off + sizeof(float4) * (size_t)L.n);
    const size_t o_lds = off;
    off = up256(off + sizeof(uint4) * 2 * (size_t)L.n);
    const size_t o_rkp = off;
    off = up256(off + sizeof(float4) * (size_t)R.n);
    const size_t o_rds = off;
    off = up256(off + sizeof(uint4) * 2 * (size_t)R.n);
    if (off > kNoAllocScratchBytes)
        return fail(FT_EINVAL, "frame needs %zu scratch bytes, more than the %zu available", off, kNoAllocScratchBytes);

    // The table is built on the host stack and copied with one asynchronous
    // copy (from pageable memory the copy consumes the source before it
    // returns, so the stack buffer can go away afterwards).
    alignas(256) unsigned char host[8192];
    static_assert(sizeof(BatchHeader) + sizeof(FrameDev) + 2048 < sizeof(host), "host table buffer too small");
    if (table_bytes > sizeof(host)) return fail(FT_EINVAL, "internal: table does not fit the host buffer");
    std::memset(host, 0, table_bytes);
    unsigned char *d = S->scratch;
    BatchHeader &B = *reinterpret_cast<BatchHeader *>(host + o_hdr);
    B.p = make_dev_params(p);
    B.nframes = 1;
    B.prefix = reinterpret_cast<const int *>(d + o_prefix);
    B.frames = reinterpret_cast<const FrameDev *>(d + o_frame);
    B.queue = reinterpret_cast<unsigned *>(d + o_queue);
    B.status = reinterpret_cast<unsigned *>(d + o_queue + 8);
    B.timeout_ns = 2000000000ull;
    B.trace = nullptr;

    FrameDev &F = *reinterpret_cast<FrameDev *>(host + o_frame);
    F.camera = FT_CAMERA_PINHOLE;
    F.do_stereo = 1;
    F.nl = L.n;
    F.nr = R.n;
    F.lx = L.x;
    F.ly = L.y;
    F.loct = L.oct;
    F.ldesc = reinterpret_cast<const uint4 *>(L.desc);
    F.rx = R.x;
    F.ry = R.y;
    F.roct = R.oct;
    F.rdesc = reinterpret_cast<const uint4 *>(R.desc);
    for (int l = 0; l < p.nlevels; ++l) {
        F.pyrL[l] = frame->pyr_left.data[l];
        F.lw[l] = frame->pyr_left.width[l];
        F.lh[l] = frame->pyr_left.height[l];
        F.lp[l] = frame->pyr_left.pitch[l];
        F.pyrR[l] = frame->pyr_right.data[l];
        F.rw[l] = frame->pyr_right.width[l];
        F.rh[l] = frame->pyr_right.height[l];
        F.rp[l] = frame->pyr_right.pitch[l];
    }
    F.H = H;
    F.b = cam->b;
    F.bf = cam->bf;
    F.best_r = out->best_r;
    F.dist = out->dist;
    F.sad_shift = out->sad_shift;
    F.sad_best = out->sad_best;
    F.u_right = out->u_right;
    F.depth = out->depth;
    F.row_ptr_l = reinterpret_cast<int *>(d + o_rpl);
    F.row_ptr_r = reinterpret_cast<int *>(d + o_rpr);
    F.ls_kp = reinterpret_cast<float4 *>(d + o_lkp);
    F.ls_desc = reinterpret_cast<uint4 *>(d + o_lds);
    F.rs_kp = reinterpret_cast<float4 *>(d + o_rkp);
    F.rs_desc = reinterpret_cast<uint4 *>(d + o_rds);
    // strips of 32 rows (the context's default), shortened by the same rule
    const int sr = stereo_strip_rows(32, H, R.n, B.p.halo);
    F.strip_rows = sr;
    F.n_stereo_items = (H + sr - 1) / sr;
    F.rowsort = kRowSortItems;
    F.n_index_items = kRowSortItems;
    F.ctr = reinterpret_cast<unsigned *>(d + o_ctr);
    int *prefix = reinterpret_cast<int *>(host + o_prefix);
    const int per_kind[K_KINDS] = {kRowSortItems, F.n_stereo_items, 0, 0};
    int total = 0;
    for (int k = 0; k < K_KINDS; ++k) {
        prefix[2 * k] = 0;
        prefix[2 * k + 1] = per_kind[k];
        B.kind_begin[k] = total;
        total += per_kind[k];
    }
    B.kind_begin[K_KINDS] = total;
    B.total_items = total;

    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d, host, table_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_fused(reinterpret_cast<const BatchHeader *>(d + o_hdr), std::min(total, S->grid), s);
    if (e == cudaSuccess && device_status)
        e = cudaMemcpyAsync(device_status, d + o_queue + 8, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(FT_ECUDA, "launch: %s", cudaGetErrorString(e));
    return FT_OK;
}

}  // extern "C"
