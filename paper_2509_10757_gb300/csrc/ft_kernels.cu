// ft_kernels.cu -- the fused, persistent tracking kernel for sm_103a.
//
// Work items (pulled in queue order by every CTA of one launch):
//   K_INDEX    per frame: the row sort of the pinhole stereo step (left and
//              right keypoints bucketed by image row, a counting sort), and
//              per camera the 64x48 keypoint grid of the search step (paper
//              section IV-E; grid reading 64x48), also a counting sort.
//   K_STEREO   pinhole: one horizontal strip of image rows.  The CTA stages
//              the row-sorted right keypoints that can reach the strip in
//              shared memory, then runs three CTA-wide phases so that every
//              memory latency is paid once per phase, not once per keypoint:
//              (1) one thread per left keypoint: band Hamming search over the
//              staged candidates (kernel 1 of section IV-C); (2) the 11x11
//              left patches and 11x21 right strips of all matches gathered
//              into shared memory; (3) one thread per (match, shift): SAD of
//              centre-subtracted patches, then per match the best shift,
//              parabola, disparity and depth (kernel 2 of section IV-C).  The
//              frame's last strip runs the median rejection.
//              fisheye: one tile of left keypoints, one thread each, against
//              the right overlap descriptors staged in shared memory chunks;
//              best/second best kept as packed (distance, index) keys.
//   K_SEARCH   one tile of map points, one thread each: frustum test, FP32
//              projection, predicted level, grid-window gather, top-2 Hamming,
//              ratio test; accepted claims go to an atomicMin per keypoint.
//              A frame whose search is split around its stereo step scans its
//              candidates before waiting for the stereo step and applies the
//              stereo consistency after it, in the same item.
//   K_RESOLVE  one tile: final map-point -> keypoint and keypoint -> map
//              point tables from the per-keypoint winners.
// Floating point runs through __fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn /
// __fsqrt_rn so that no multiply-add is contracted and every operation is
// IEEE-rounded in the order the method defines it.
#include <cuda_runtime.h>

#include <cstdint>

#include "ft_internal.h"

namespace ft {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kNoKey = 0xffffffffu;
constexpr int kW = FT_SAD_W;
constexpr int kL = FT_SAD_L;
constexpr int kStripW = 2 * (kW + kL) + 1;                      // 21
constexpr int kShifts = 2 * kL + 1;                             // 11
constexpr int kBatch = 4;                                       // loads issued ahead per thread
constexpr int kScatter = 3;                                     // keypoints per thread per scatter batch
constexpr int kGridScatter = 2;

// resident CTAs per SM the register budget is sized for
#ifndef FT_MIN_CTAS_PER_SM
#define FT_MIN_CTAS_PER_SM 3
#endif

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ int f2i(float x) { return __float2int_rz(x); }   // C (int) cast

__device__ __forceinline__ int ham8(uint4 a0, uint4 a1, uint4 b0, uint4 b1)
{
    return __popc(a0.x ^ b0.x) + __popc(a0.y ^ b0.y) + __popc(a0.z ^ b0.z) +
           __popc(a0.w ^ b0.w) + __popc(a1.x ^ b1.x) + __popc(a1.y ^ b1.y) +
           __popc(a1.z ^ b1.z) + __popc(a1.w ^ b1.w);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Top-2 of packed (distance << 20 | index) keys: the smallest and the
// smallest of the rest.
__device__ __forceinline__ void top2_push(unsigned key, unsigned &best, unsigned &second)
{
    second = min(second, max(best, key));
    best = min(best, key);
}

// atan2 for y >= 0, x >= 0, from the mathematics: atan2(y, x) = atan(y/x)
// when y <= x, else pi/2 - atan(x/y); atan(t) = pi/4 + atan((t-1)/(t+1)) for
// t > tan(pi/8); below that the Taylor series of atan with terms up to a^17
// (coefficients (-1)^k / (2k+1) divided out in FP32), evaluated by Horner in
// a^2.
__device__ float atan_series(float a)
{
    const float a2 = fmul(a, a);
    float p = fdiv(1.0f, 17.0f);
    p = fadd(-fdiv(1.0f, 15.0f), fmul(a2, p));
    p = fadd(fdiv(1.0f, 13.0f), fmul(a2, p));
    p = fadd(-fdiv(1.0f, 11.0f), fmul(a2, p));
    p = fadd(fdiv(1.0f, 9.0f), fmul(a2, p));
    p = fadd(-fdiv(1.0f, 7.0f), fmul(a2, p));
    p = fadd(fdiv(1.0f, 5.0f), fmul(a2, p));
    p = fadd(-fdiv(1.0f, 3.0f), fmul(a2, p));
    p = fadd(1.0f, fmul(a2, p));
    return fmul(a, p);
}

__device__ float atan_unit(float t)
{
    if (t > 0.41421356237309504880f)
        return fadd(0.78539816339744830962f, atan_series(fdiv(fsub(t, 1.0f), fadd(t, 1.0f))));
    return atan_series(t);
}

__device__ float atan2_pos(float y, float x)
{
    if (y == 0.0f) return 0.0f;
    if (y <= x) return atan_unit(fdiv(y, x));
    return fsub(1.57079632679489661923f, atan_unit(fdiv(x, y)));
}

// Exclusive scan of n ints (in place allowed), block-wide; returns the total.
__device__ int block_scan(const int *in, int *out, int n, int *warp_sums)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int per = (n + kThreads - 1) / kThreads;
    const int b = tid * per;
    int local = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < n) local += in[b + i];
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < kWarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += t;
        }
        if (lane < kWarps) warp_sums[lane] = s;
    }
    __syncthreads();
    int run = v - local + (w > 0 ? warp_sums[w - 1] : 0);
    for (int i = 0; i < per; ++i) {
        if (b + i < n) {
            const int x = in[b + i];
            out[b + i] = run;
            run += x;
        }
    }
    const int total = warp_sums[kWarps - 1];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------- shared memory
// one match waiting for its SAD refinement
struct RefineJob {
    int i, j, d, l, ul, vl, ur0;
    float xi;
};

constexpr int kGroup = 4;                       // lanes per left keypoint in the Hamming phase
constexpr int kGroups = kThreads / kGroup;      // left keypoints in flight per CTA
constexpr int kSadChunk = 64;                   // matches refined per round
constexpr int kChunksL = 2;                     // 16-byte chunks holding a left patch row (11 bytes)
constexpr int kChunksR = 3;                     // chunks holding a right strip row (21 bytes)

// patches of one refinement round as the raw 16-byte chunks of their rows
// (copied asynchronously; a row's bytes start at offset (column & 15))
struct PatchBuf {
    uint4 l[kSadChunk][2 * kW + 1][kChunksL];
    uint4 r[kSadChunk][2 * kW + 1][kChunksR];
};
// left keypoints of a pass (Hamming phase)
struct LeftBuf {
    float4 lkp[kThreads];              // x, y, index, octave
    uint4 ldesc[2 * kThreads];
};

// what the Hamming phase reads: the staged right window and the pass's left
// keypoints
struct StageBuf {
    float4 rkp[kStageCap];             // staged right keypoints sorted by (octave, row)
    uint4 sdesc[2 * kStageCap];        // their descriptors in row order
    LeftBuf left;
};

struct SmemStereo {
    union {                            // the window and the left keypoints are dead once
        StageBuf st;                   // the Hamming phase is over; the patches reuse them
        PatchBuf patch;                // (a strip with a second pass stages its window again)
    } u;
    RefineJob ref[kThreads];
    int gp[kSadChunk];                 // grid record of each match of the round (-1: none)
    int sad[kSadChunk][12];
    int bptr[kOctBuckets * kWinRows + 1];   // start of each (octave, window row) bucket
    int warp_sums[kWarps];
    int nref;
};

constexpr int kSortParts = kRowSortItems / 2;   // work items per side of a frame's row sort

struct SmemRows {
    int cnt[kSortParts][kMaxRows + 1];  // per-part row counts, then this part's write cursors
    int tot[kMaxRows + 1];              // row totals, then row starts
    int warp_sums[kWarps];
};

struct SmemGrid {
    int cnt[kCells];
    int warp_sums[kWarps];
};

constexpr int kFishGroup = 4;                    // lanes sharing one left keypoint (each scans a quarter)
constexpr int kFishSlots = kThreads / kFishGroup; // left keypoints per pass
static_assert(kFishTileMax % kFishSlots == 0, "a fisheye item is a whole number of passes");

struct SmemFish {
    uint4 desc[2 * kFishChunk];
    int idx[kFishChunk];
    int act[kFishTileMax];   // the item's left keypoints inside the overlap
    int count, nact;
};

constexpr int kMedianSmem = 8192;               // left keypoints whose SADs the median keeps on chip

struct SmemMedian {
    int hist[256], hist2[256];          // high bytes; low bytes within the median's high byte
    int count, bin, before;
    int vals[kMedianSmem];
    int gp[kMedianSmem];               // grid record of each left keypoint (searched frames)
};

constexpr int kSearchStage = 1536;              // keypoints of one camera the search keeps on chip

constexpr int kCell16Bytes = (2 * (kCells + 1) + 15) / 16 * 16;   // 16-bit cell starts, whole chunks

// a camera's keypoints in cell order, staged for the search of one tile:
// records (x, y, index | octave << 20 | taken << 28, right coordinate or -1)
// then descriptors, and, when they fit behind them, the 16-bit cell starts
struct SmemSearch {
    float pose[12];
    uint4 buf[kSearchStage * 3];
};

union Smem {
    SmemStereo s;
    SmemRows r;
    SmemGrid g;
    SmemFish f;
    SmemMedian m;
    SmemSearch q;
};
// three CTAs per SM: dynamic + static shared memory + the 1 KB the SM
// reserves per CTA must stay within the SM's 228 KB
static_assert(3 * (sizeof(Smem) + sizeof(BatchHeader) + sizeof(FrameDev) + 256 + 1024) <= 228 * 1024,
              "shared memory above three CTAs per SM");

// ---------------------------------------------------------------- waits and signals
// time this CTA spent in waits during the current item, and phase marks (tracing)
__shared__ unsigned long long s_wait_ns;
__shared__ unsigned long long s_mark[4];

__device__ __forceinline__ void mark(const BatchHeader &B, int k)
{
    if (B.trace != nullptr && threadIdx.x == 0) s_mark[k] = global_ns();
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

// Block-wide wait until *ctr >= target, bounded by the header's timeout.  On
// timeout (or when another CTA already reported one) it records the timeout in
// the status word and returns false.
// A second counter (ctr2 non-null) is polled in the same round trip.
__device__ bool wait_geq(const BatchHeader &B, const unsigned *ctr, unsigned target, int *s_flag,
                         const unsigned *ctr2 = nullptr, unsigned target2 = 0)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        auto ready = [&]() {
            const unsigned a = ld_acquire(ctr);
            const unsigned b = ctr2 ? ld_acquire(ctr2) : target2;
            return a >= target && b >= target2;
        };
        if (!ready()) {
            const unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (!ready()) {
                if ((++spins & 31u) == 0) {
                    if (global_ns() - t0 > B.timeout_ns || (ld_acquire(B.status) & kStatusTimeout)) {
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(256);
            }
            if (!ok) atomicOr(B.status, kStatusTimeout);
            s_wait_ns += global_ns() - t0;
        }
        *s_flag = ok;
    }
    __syncthreads();
    const bool ok = *s_flag != 0;
    __syncthreads();
    return ok;
}

// Publish this CTA's writes and add one to *ctr; returns true in every thread
// of the CTA that brought the counter to `total`.
__device__ bool signal_count(unsigned *ctr, unsigned total, int *s_flag)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(ctr, 1u);
        const int last = (prev + 1u == total);
        if (last) __threadfence();
        *s_flag = last;
    }
    __syncthreads();
    const bool last = *s_flag != 0;
    __syncthreads();
    return last;
}

// ---------------------------------------------------------------- K_INDEX
__device__ __forceinline__ int grid_cell(const CamDev &C, float iw, float ih, float x, float y)
{
    const int cx = f2i(roundf(fmul(fsub(x, C.minx), iw)));
    const int cy = f2i(roundf(fmul(fsub(y, C.miny), ih)));
    if (cx < 0 || cx >= FT_GRID_COLS || cy < 0 || cy >= FT_GRID_ROWS) return -1;
    return cy * FT_GRID_COLS + cx;
}

__device__ void grid_item(const BatchHeader &B, const FrameDev &F, int cam, SmemGrid &G,
                          int *s_flag)
{
    const CamDev &C = F.cam[cam];
    const int tid = threadIdx.x;
    const float iw = fdiv((float)FT_GRID_COLS, fsub(C.maxx, C.minx));
    const float ih = fdiv((float)FT_GRID_ROWS, fsub(C.maxy, C.miny));
    for (int c = tid; c < kCells; c += kThreads) G.cnt[c] = 0;
    __syncthreads();
    for (int base = 0; base < C.nk; base += kBatch * kThreads) {
        float x[kBatch], y[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = base + u * kThreads + tid;
            x[u] = k < C.nk ? __ldg(C.kx + k) : 0.0f;
            y[u] = k < C.nk ? __ldg(C.ky + k) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int c = grid_cell(C, iw, ih, x[u], y[u]);
            if (base + u * kThreads + tid < C.nk && c >= 0) atomicAdd(&G.cnt[c], 1);
        }
    }
    __syncthreads();
    mark(B, 0);
    const int total = block_scan(G.cnt, G.cnt, kCells, G.warp_sums);
    for (int c = tid; c < kCells; c += kThreads) {
        C.cell_ptr[c] = G.cnt[c];
        C.cell16[c] = (uint16_t)G.cnt[c];      // read only for frames of fewer than 65536 keypoints
    }
    if (tid == 0) {
        C.cell_ptr[kCells] = total;
        C.cell16[kCells] = (uint16_t)total;
    }
    __syncthreads();
    mark(B, 1);
    // the record's right coordinate: a stereo step in this launch fills it
    // in later (pinhole frames that wait for their stereo); otherwise it is
    // the caller's u_right input, or -1 (no consistency check)
    const bool ur_in = C.model == FT_CAMERA_PINHOLE && F.u_right_in != nullptr && !F.wait_stereo;
    for (int base = 0; base < C.nk; base += kGridScatter * kThreads) {
        float x[kGridScatter], y[kGridScatter], ur[kGridScatter];
        unsigned oct[kGridScatter], tk[kGridScatter];
        uint4 d0[kGridScatter], d1[kGridScatter];
#pragma unroll
        for (int u = 0; u < kGridScatter; ++u) {
            const int k = min(base + u * kThreads + tid, C.nk - 1);
            x[u] = __ldg(C.kx + k);
            y[u] = __ldg(C.ky + k);
            oct[u] = (unsigned)__ldg(C.koct + k) & 0xffu;
            tk[u] = C.taken ? (__ldg(C.taken + k) != 0) : 0u;
            ur[u] = ur_in ? __ldg(F.u_right_in + k) : -1.0f;
            d0[u] = __ldg(C.kdesc + 2 * k);
            d1[u] = __ldg(C.kdesc + 2 * k + 1);
        }
#pragma unroll
        for (int u = 0; u < kGridScatter; ++u) {
            const int k = base + u * kThreads + tid;
            if (k >= C.nk) continue;
            const int c = grid_cell(C, iw, ih, x[u], y[u]);
            int pos = -1;
            if (c >= 0) {
                pos = atomicAdd(&G.cnt[c], 1);
                C.gkp[pos] = make_float4(x[u], y[u], __uint_as_float((unsigned)k | (oct[u] << 20) | (tk[u] << 28)),
                                         ur[u]);
                C.gdesc[2 * pos] = d0[u];
                C.gdesc[2 * pos + 1] = d1[u];
            }
            C.gpos[k] = pos;
            C.owner[k] = ~0ull;
        }
    }
    mark(B, 2);
    signal_count(&F.ctr[C_GRID_DONE], (unsigned)F.n_grid_items, s_flag);
    mark(B, 3);
}

// ---------------------------------------------------------------- K_INDEX: row sort
__device__ __forceinline__ int floor_row(float y) { return f2i(floorf(y)); }

// Row that owns a keypoint in the row sort (rows outside the image go to the
// edge rows).
__device__ __forceinline__ int own_row(float y, int H)
{
    if (y < 0.0f) return 0;
    return min(f2i(y), H - 1);
}

// Right keypoints are bucketed by floor(y) clamped to the image, left
// keypoints by the row they search, (int)y clamped to the image.  Each side's
// sort is split over kSortParts work items that run side by side: every part
// counts all keypoints per row and per part, and scatters only its own
// contiguous share, starting each row after the parts before it.
__device__ __forceinline__ int sort_row(bool right, float y, int H)
{
    return right ? clampi(floor_row(y), 0, H - 1) : own_row(y, H);
}

__device__ void rowsort_item(const BatchHeader &B, const FrameDev &F, SmemRows &S, bool right, int part,
                             int *s_flag)
{
    const int tid = threadIdx.x, H = F.H;
    const int n = right ? F.nr : F.nl;
    const float *ys = right ? F.ry : F.ly;
    const int share = (n + kSortParts - 1) / kSortParts;
    for (int r = tid; r <= H; r += kThreads)
        for (int p = 0; p < kSortParts; ++p) S.cnt[p][r] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kBatch * kThreads) {
        float y[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads + tid;
            y[u] = i < n ? __ldg(ys + i) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads + tid;
            if (i < n) atomicAdd(&S.cnt[i / share][sort_row(right, y[u], H)], 1);
        }
    }
    __syncthreads();
    mark(B, 0);
    for (int r = tid; r < H; r += kThreads) {
        int t = 0;
        for (int p = 0; p < kSortParts; ++p) t += S.cnt[p][r];
        S.tot[r] = t;
    }
    __syncthreads();
    const int total = block_scan(S.tot, S.tot, H, S.warp_sums);
    // this part's write cursor per row: the row's start plus the earlier parts' counts
    for (int r = tid; r < H; r += kThreads) {
        int c = S.tot[r];
        for (int p = 0; p < part; ++p) c += S.cnt[p][r];
        S.cnt[part][r] = c;
    }
    if (part == 0) {
        int *row_ptr = right ? F.row_ptr_r : F.row_ptr_l;
        for (int r = tid; r < H; r += kThreads) row_ptr[r] = S.tot[r];
        if (tid == 0) row_ptr[H] = total;
    }
    __syncthreads();
    mark(B, 1);
    // the part's share: records (right: x, band rows, row, index | octave;
    // left: x, y, index, octave) and descriptors in row order, so that the
    // stereo strips read them contiguously (all loads of a batch are issued
    // before its shared-memory atomics)
    const int i0 = part * share, i1 = min(n, i0 + share);
    const float *xs = right ? F.rx : F.lx;
    const int8_t *os = right ? F.roct : F.loct;
    const uint4 *ds = right ? F.rdesc : F.ldesc;
    float4 *rec_out = right ? F.rs_kp : F.ls_kp;
    uint4 *desc_out = right ? F.rs_desc : F.ls_desc;
    for (int base = i0; base < i1; base += kScatter * kThreads) {
        float x[kScatter], y[kScatter];
        int oct[kScatter];
        uint4 d0[kScatter], d1[kScatter];
#pragma unroll
        for (int u = 0; u < kScatter; ++u) {
            const int i = min(base + u * kThreads + tid, i1 - 1);
            x[u] = __ldg(xs + i);
            y[u] = __ldg(ys + i);
            oct[u] = __ldg(os + i);
            d0[u] = __ldg(ds + 2 * i);
            d1[u] = __ldg(ds + 2 * i + 1);
        }
#pragma unroll
        for (int u = 0; u < kScatter; ++u) {
            const int i = base + u * kThreads + tid;
            if (i >= i1) continue;
            const int row = sort_row(right, y[u], H);
            const int pos = atomicAdd(&S.cnt[part][row], 1);
            if (right) {
                // the rows this keypoint lists: floor(y - r) .. ceil(y + r), r = 2 scale[oct],
                // clamped to the image (computed once here, tested per candidate later;
                // an empty band stays empty: lo in [0, H], hi in [-1, H - 1])
                const float r = B.p.band_r[clampi(oct[u], 0, B.p.nlevels - 1)];
                const int lo = min(max(f2i(floorf(fsub(y[u], r))), 0), H);
                const int hi = max(min(f2i(ceilf(fadd(y[u], r))), H - 1), -1);
                rec_out[pos] = make_float4(x[u], __int_as_float(lo | (hi << 16)), __int_as_float(row),
                                           __int_as_float(i | ((oct[u] & 0xff) << 20)));
            } else {
                rec_out[pos] = make_float4(x[u], y[u], __int_as_float(i), __int_as_float(oct[u]));
            }
            desc_out[2 * pos] = d0[u];
            desc_out[2 * pos + 1] = d1[u];
        }
    }
    mark(B, 2);
    signal_count(&F.ctr[C_ROWS_DONE], (unsigned)F.rowsort, s_flag);
    mark(B, 3);
}

// ---------------------------------------------------------------- K_STEREO, pinhole
// A row-sorted right keypoint record: x, band rows lo | hi << 16, bucket row,
// index | octave << 20.
__device__ __forceinline__ bool band_has(float packed, int row)
{
    const int b = __float_as_int(packed);
    return (b & 0xffff) <= row && row <= (b >> 16);
}
__device__ __forceinline__ int rec_index(float w) { return __float_as_int(w) & 0xfffff; }
__device__ __forceinline__ int rec_octave(float w) { return (int)(int8_t)((__float_as_int(w) >> 20) & 0xff); }

__device__ __forceinline__ void write_stereo(const FrameDev &F, int i, int best, int dist, int shift,
                                             int sadb, float ur, float dep)
{
    F.best_r[i] = best;
    F.dist[i] = dist;
    F.sad_shift[i] = shift;
    F.sad_best[i] = sadb;
    F.u_right[i] = ur;
    F.depth[i] = dep;
}

// Phase 1: the 8 lanes of a group scan the band candidates of one left
// keypoint (consecutive candidates per lane, conflict-free shared loads) and
// reduce to the smallest (distance, right index); lane 0 of the group queues
// the match for refinement or writes the final "no match" outputs.
__device__ void hamming_phase(const DevParams &P, const FrameDev &F, SmemStereo &S, int npass,
                              bool staged, int w_a, int nrows)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane & (kGroup - 1), gw = lane / kGroup;
    const float disp_hi = fdiv(F.bf, F.b);
    for (int tb = warp * (32 / kGroup); tb < npass; tb += kGroups) {
        const int t = tb + gw;
        const bool have = t < npass;
        unsigned key = kNoKey;
        float xb = 0.0f;
        float xi = 0.0f, yi = 0.0f;
        int oi = 0, i = 0;
        if (have) {
            const float4 L = S.u.st.left.lkp[t];
            xi = L.x;
            yi = L.y;
            i = __float_as_int(L.z);
            oi = __float_as_int(L.w);
            const int row = f2i(yi);
            const float u_lo = fsub(xi, disp_hi);
            const float u_hi = fsub(xi, 0.0f);
            if (!(yi < 0.0f) && row < F.H && !(u_hi < 0.0f)) {
                const uint4 a0 = S.u.st.left.ldesc[2 * t], a1 = S.u.st.left.ldesc[2 * t + 1];
                if (staged) {
                    // candidate octaves oi-1 .. oi+1, each over the rows its band can reach
                    const int olo = max(oi - 1, 0), ohi = min(oi + 1, kOctBuckets - 1);
                    for (int o = olo; o <= ohi; ++o) {
                        const int h = P.halo_c[o];
                        const int ra = max(row - h, w_a) - w_a;
                        const int rb = min(row + h, w_a + nrows - 1) - w_a;
                        const int e1 = S.bptr[o * nrows + rb + 1];
                        for (int e = S.bptr[o * nrows + ra] + sub; e < e1; e += kGroup) {
                            const float4 g = S.u.st.rkp[e];
                            const int oj = rec_octave(g.w);
                            if (oj < oi - 1 || oj > oi + 1) continue;
                            if (!band_has(g.y, row)) continue;
                            if (g.x < u_lo || g.x > u_hi) continue;
                            const int at = __float_as_int(g.z);
                            const unsigned k = ((unsigned)ham8(a0, a1, S.u.st.sdesc[2 * at], S.u.st.sdesc[2 * at + 1]) << 20) |
                                               (unsigned)rec_index(g.w);
                            if (k < key) {
                                key = k;
                                xb = g.x;
                            }
                        }
                    }
                } else {
                    const int h = (oi >= 0 && oi < P.nlevels) ? P.halo_oct[oi] : P.halo;
                    const int e0 = __ldcg(F.row_ptr_r + max(row - h, 0));
                    const int e1 = __ldcg(F.row_ptr_r + min(row + h, F.H - 1) + 1);
                    for (int e = e0 + sub; e < e1; e += kGroup) {
                        const float4 g = __ldcg(F.rs_kp + e);
                        const int oj = rec_octave(g.w);
                        if (oj < oi - 1 || oj > oi + 1) continue;
                        if (!band_has(g.y, row)) continue;
                        if (g.x < u_lo || g.x > u_hi) continue;
                        const unsigned k = ((unsigned)ham8(a0, a1, __ldcg(F.rs_desc + 2 * e),
                                                           __ldcg(F.rs_desc + 2 * e + 1)) << 20) |
                                           (unsigned)rec_index(g.w);
                        if (k < key) {
                            key = k;
                            xb = g.x;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) {
            const unsigned k2 = __shfl_xor_sync(kFull, key, o);
            const float x2 = __shfl_xor_sync(kFull, xb, o);
            if (k2 < key) {
                key = k2;
                xb = x2;
            }
        }
        // every lane of the group holds the reduced key
        if (have) {
            int best = -1, dist = -1;
            if (key != kNoKey) {
                dist = (int)(key >> 20);
                if (dist < P.th_stereo) best = (int)(key & 0xfffffu);
            }
            bool queued = false;
            if (best >= 0) {
                const int l = clampi(oi, 0, P.nlevels - 1);
                const int ul = f2i(roundf(fmul(xi, P.isc[l])));
                const int vl = f2i(roundf(fmul(yi, P.isc[l])));
                const int ur0 = f2i(roundf(fmul(xb, P.isc[l])));
                // windows inside both level images.  ul, vl and ur0 saturate at
                // INT_MAX / INT_MIN for coordinates of 2^31 and more (or +-inf), so
                // they are compared with the bounds and never offset: ul + kW would
                // wrap negative and let a window 2 GB past the level through.
                const bool inside = vl >= kW && vl <= F.lh[l] - 1 - kW && vl <= F.rh[l] - 1 - kW &&
                                    ul >= kW && ul <= F.lw[l] - 1 - kW &&
                                    ur0 >= kL + kW && ur0 <= F.rw[l] - 1 - kL - kW;
                if (inside) {
                    // the lanes ask L2 for the patch rows now, so that the
                    // refinement's copies find them there
                    for (int rr = sub; rr < 2 * kW + 1; rr += kGroup) {
                        const uint8_t *pl = F.pyrL[l] + (size_t)(vl - kW + rr) * F.lp[l] + (ul - kW);
                        const uint8_t *pr = F.pyrR[l] + (size_t)(vl - kW + rr) * F.rp[l] + (ur0 - kL - kW);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(pl));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(pr));
                        if (((reinterpret_cast<uintptr_t>(pr) & 127u) + kStripW - 1) >= 128u)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + kStripW - 1));
                        if (((reinterpret_cast<uintptr_t>(pl) & 127u) + 2 * kW) >= 128u)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + 2 * kW));
                    }
                    if (sub == 0) {
                        const int slot = atomicAdd(&S.nref, 1);
                        S.ref[slot] = RefineJob{i, best, dist, l, ul, vl, ur0, xi};
                    }
                    queued = true;
                }
            }
            if (!queued && sub == 0) write_stereo(F, i, best, dist, FT_NO_SHIFT, -1, -1.0f, -1.0f);
        }
    }
}

// Phases 2-3 for refine jobs [r0, r0 + nc), nc <= kSadChunk:
// (2) one warp per match copies its 11 left patch rows and 11 right strip
//     rows into shared memory, lanes on consecutive bytes (coalesced);
// (3) one thread per (match, patch row) reads its rows as words and adds the
//     row's part of the 11 SADs of centre-subtracted patches; then per match
//     the first strict minimum over the shifts, the parabola, disparity and
//     depth.
__device__ void refine_round(const DevParams &P, const FrameDev &F, SmemStereo &S, int r0, int nc, bool rec)
{
    const int tid = threadIdx.x;
    constexpr int kRows = 2 * kW + 1;
    for (int q = tid; q < nc * kShifts; q += kThreads) S.sad[q / kShifts][q % kShifts] = 0;
    // asynchronous copies of the 16-byte chunks holding every patch row; a
    // match has five chunk slots (two of a left row, three of a right row)
    // and one thread per slot walks the 11 rows.  Level pointers and pitches
    // are 16-byte aligned (checked on the host): a row's chunks start at its
    // column rounded down to a multiple of 16 and end within the row's pitch.
    constexpr int kSlots = kChunksL + kChunksR;
    for (int q = tid; q < nc * kSlots; q += kThreads) {
        const int mm = q / kSlots, w = q - mm * kSlots;
        const bool right = w >= kChunksL;
        const int k = right ? w - kChunksL : w;
        const RefineJob &J = S.ref[r0 + mm];
        const int col = right ? J.ur0 - kL - kW : J.ul - kW;
        const int len = right ? kStripW : 2 * kW + 1;
        if (k > (((col & 15) + len - 1) >> 4)) continue;    // the chunk holds none of the row's bytes
        const int pitch = right ? F.rp[J.l] : F.lp[J.l];
        const uint8_t *src = (right ? F.pyrR[J.l] : F.pyrL[J.l]) + (size_t)(J.vl - kW) * pitch + (col & ~15) + 16 * k;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(right ? &S.u.patch.r[mm][0][k]
                                                                       : &S.u.patch.l[mm][0][k]);
        const unsigned dstep = 16u * (right ? kChunksR : kChunksL);
#pragma unroll
        for (int row = 0; row < kRows; ++row)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + row * dstep),
                         "l"(src + (size_t)row * pitch)
                         : "memory");
    }
    // the grid record of each match (the search reads the right coordinate there)
    if (rec && tid < nc) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&S.gp[tid]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(F.cam[0].gpos + S.ref[r0 + tid].i)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int q = tid; q < nc * kRows; q += kThreads) {
        const int dy = q / nc, m = q - dy * nc;
        const RefineJob &J = S.ref[r0 + m];
        const int ol = (J.ul - kW) & 15, orr = (J.ur0 - kL - kW) & 15;
        // the rows as 32-bit words; byte b of a row is byte (o + b) of its chunks
        const unsigned *ql = reinterpret_cast<const unsigned *>(S.u.patch.l[m][dy]) + (ol >> 2);
        const unsigned *qr = reinterpret_cast<const unsigned *>(S.u.patch.r[m][dy]) + (orr >> 2);
        const unsigned *qc = reinterpret_cast<const unsigned *>(S.u.patch.r[m][kW]) + (orr >> 2);
        const unsigned *qlc = reinterpret_cast<const unsigned *>(S.u.patch.l[m][kW]) + (ol >> 2);
        const int sl = 8 * (ol & 3), sr = 8 * (orr & 3);
        // realigned words: byte b of the row is byte b & 3 of word b >> 2
        unsigned wl[3], wr[6], wc[4];
#pragma unroll
        for (int k = 0; k < 3; ++k) wl[k] = __funnelshift_r(ql[k], ql[k + 1], sl);
#pragma unroll
        for (int k = 0; k < 6; ++k) wr[k] = __funnelshift_r(qr[k], qr[k + 1], sr);
#pragma unroll
        for (int k = 1; k < 4; ++k) wc[k] = __funnelshift_r(qc[k], qc[k + 1], sr);
        // left row minus the left centre, right row, and the centres of the
        // 11 right patches (bytes 5..15 of the right centre row)
        const int cl = (int)((__funnelshift_r(qlc[1], qlc[2], sl) >> 8) & 0xff);
        int lc[2 * kW + 1], rv[kStripW], cr[kShifts];
#pragma unroll
        for (int b = 0; b < 2 * kW + 1; ++b) lc[b] = (int)((wl[b >> 2] >> (8 * (b & 3))) & 0xff) - cl;
#pragma unroll
        for (int b = 0; b < kStripW; ++b) rv[b] = (wr[b >> 2] >> (8 * (b & 3))) & 0xff;
#pragma unroll
        for (int k = 0; k < kShifts; ++k) cr[k] = (wc[(k + kW) >> 2] >> (8 * ((k + kW) & 3))) & 0xff;
#pragma unroll
        for (int k = 0; k < kShifts; ++k) {
            int s = 0;
#pragma unroll
            for (int dx = 0; dx < 2 * kW + 1; ++dx) s = __sad(lc[dx] + cr[k], rv[k + dx], s);
            atomicAdd(&S.sad[m][k], s);
        }
    }
    __syncthreads();
    for (int m = tid; m < nc; m += kThreads) {
        const RefineJob &J = S.ref[r0 + m];
        const int *sad = S.sad[m];
        int kb = 0;
        for (int k = 1; k < kShifts; ++k)
            if (sad[k] < sad[kb]) kb = k;
        const int shift = kb - kL;
        int sadb = -1;
        float ur = -1.0f, dep = -1.0f;
        if (kb != 0 && kb != 2 * kL) {
            const float d1 = (float)sad[kb - 1], d2 = (float)sad[kb], d3 = (float)sad[kb + 1];
            const float delta = fdiv(fsub(d1, d3), fmul(2.0f, fsub(fadd(d1, d3), fmul(2.0f, d2))));
            if (!(delta < -1.0f || delta > 1.0f)) {
                float ur_sub = fmul(P.sc[J.l], fadd(fadd((float)J.ur0, (float)shift), delta));
                float disparity = fsub(J.xi, ur_sub);
                const float disp_hi = fdiv(F.bf, F.b);
                if (disparity >= 0.0f && disparity < disp_hi) {
                    if (disparity <= 0.0f) {
                        disparity = 0.01f;
                        ur_sub = fsub(J.xi, 0.01f);
                    }
                    dep = fdiv(F.bf, disparity);
                    ur = ur_sub;
                    sadb = sad[kb];
                }
            }
        }
        write_stereo(F, J.i, J.j, J.d, shift, sadb, ur, dep);
        if (rec && sadb >= 0 && S.gp[m] >= 0) reinterpret_cast<float *>(F.cam[0].gkp + S.gp[m])[3] = ur;
    }
    __syncthreads();
}

// warp 0: bin of the k-th smallest value (0-based) of a 256-bin histogram
__device__ void select_bin(const int *hist, int k, int *bin, int *before)
{
    const int lane = threadIdx.x & 31;
    int s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += hist[lane * 8 + j];
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - s;
    const unsigned m = __ballot_sync(kFull, excl <= k && k < incl);
    if (lane == __ffs(m) - 1) {
        int c = excl;
        for (int j = 0; j < 8; ++j) {
            const int h = hist[lane * 8 + j];
            if (k < c + h) {
                *bin = lane * 8 + j;
                *before = c;
                break;
            }
            c += h;
        }
    }
}

// a5: median of the frame's accepted SAD minima (radix select on 2 x 8 bits),
// then drop matches with SAD >= factor * median.  Frames of up to
// kMedianSmem left keypoints load the values once into shared memory;
// larger frames read them three times.
__device__ __forceinline__ int median_value(const FrameDev &F, const SmemMedian &M, bool on_chip, int i)
{
    return on_chip ? M.vals[i] : __ldcg(F.sad_best + i);
}

constexpr int kMedianBatch = 8;   // values a thread loads at once in the median's first pass

__device__ void median_reject(const BatchHeader &B, const FrameDev &F, SmemMedian &M, bool grid_ok)
{
    const DevParams &P = B.p;
    const int tid = threadIdx.x;
    // a search in this launch reads the final right coordinates from the
    // grid records (the strip waited for the grid step): a rejected match
    // takes its coordinate back there too
    const bool rec = F.wait_stereo && F.u_right_in != nullptr && grid_ok;
    const bool on_chip = F.nl <= kMedianSmem;
    for (int b = tid; b < 256; b += kThreads) M.hist[b] = M.hist2[b] = 0;
    if (tid == 0) M.count = 0;
    __syncthreads();
    // one pass over the values (kept on chip with each keypoint's grid
    // record when they fit): the count and the histogram of the high bytes;
    // a thread loads kMedianBatch values before it stores or counts any
    int local = 0;
    for (int i0 = tid; i0 < F.nl; i0 += kThreads * kMedianBatch) {
        int xv[kMedianBatch], gv[kMedianBatch];
#pragma unroll
        for (int u = 0; u < kMedianBatch; ++u) {
            const int i = i0 + u * kThreads;
            xv[u] = i < F.nl ? __ldcg(F.sad_best + i) : -1;
            gv[u] = on_chip && rec && i < F.nl ? __ldcg(F.cam[0].gpos + i) : -1;
        }
#pragma unroll
        for (int u = 0; u < kMedianBatch; ++u) {
            const int i = i0 + u * kThreads;
            if (i >= F.nl) continue;
            if (on_chip) {
                M.vals[i] = xv[u];
                if (rec) M.gp[i] = gv[u];
            }
            if (xv[u] >= 0) {
                atomicAdd(&M.hist[(xv[u] >> 8) & 255], 1);
                ++local;
            }
        }
    }
    local = __reduce_add_sync(kFull, local);
    if ((tid & 31) == 0 && local) atomicAdd(&M.count, local);
    __syncthreads();
    const int n = M.count;
    if (n == 0) return;
    const int k = n / 2;
    if (tid < 32) select_bin(M.hist, k, &M.bin, &M.before);
    __syncthreads();
    const int hi = M.bin;
    const int k2 = k - M.before;
    for (int i = tid; i < F.nl; i += kThreads) {
        const int x = median_value(F, M, on_chip, i);
        if (x >= 0 && ((x >> 8) & 255) == hi) atomicAdd(&M.hist2[x & 255], 1);
    }
    __syncthreads();
    if (tid < 32) select_bin(M.hist2, k2, &M.bin, &M.before);
    __syncthreads();
    const int median = (hi << 8) | M.bin;
    const float th = fmul(P.median_factor, (float)median);
    const CamDev &C = F.cam[0];
    for (int i = tid; i < F.nl; i += kThreads) {
        const int x = median_value(F, M, on_chip, i);
        if (x < 0) continue;
        if ((float)x >= th) {
            F.u_right[i] = -1.0f;
            F.depth[i] = -1.0f;
            if (rec) {
                const int pos = on_chip ? M.gp[i] : __ldcg(C.gpos + i);
                if (pos >= 0) reinterpret_cast<float *>(C.gkp + pos)[3] = -1.0f;
            }
        }
    }
}

// Stage the row-sorted right keypoints of window rows [w_a, w_a + nrows)
// in shared memory, re-bucketed by (octave, row) so that a left keypoint
// visits only its octaves; their descriptors keep row order (a staged record
// carries its row-order position) and arrive by asynchronous copies that the
// caller waits for.
__device__ __forceinline__ void stage_window(const FrameDev &F, SmemStereo &S, int w_a, int nrows, int e_base,
                                             int n_st)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < 2 * n_st; e += kThreads) cp_async16(&S.u.st.sdesc[e], F.rs_desc + 2 * e_base + e);
    constexpr int Q = kStageCap / kThreads;
    const int nb = kOctBuckets * nrows;
    for (int b = tid; b <= nb; b += kThreads) S.bptr[b] = 0;
    __syncthreads();
    float4 g[Q];
    int bucket[Q], rank[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int e = q * kThreads + tid;
        if (e < n_st) {
            g[q] = __ldcg(F.rs_kp + e_base + e);
            bucket[q] = clampi(rec_octave(g[q].w), 0, kOctBuckets - 1) * nrows + (__float_as_int(g[q].z) - w_a);
            rank[q] = atomicAdd(&S.bptr[bucket[q]], 1);
        }
    }
    __syncthreads();
    block_scan(S.bptr, S.bptr, nb + 1, S.warp_sums);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int e = q * kThreads + tid;
        if (e < n_st) {
            g[q].z = __int_as_float(e);          // row-order position: its descriptor
            S.u.st.rkp[S.bptr[bucket[q]] + rank[q]] = g[q];
        }
    }
}

__device__ void stereo_pinhole_item(const BatchHeader &B, const FrameDev &F, int strip, Smem &U,
                                    int *s_flag)
{
    SmemStereo &S = U.s;
    const DevParams &P = B.p;
    const int tid = threadIdx.x;
    // a search in this launch reads each refined match's right coordinate
    // from the grid record, written once the grid step is done
    const bool rec = F.wait_stereo && F.u_right_in != nullptr;
    bool ready = wait_geq(B, &F.ctr[C_ROWS_DONE], (unsigned)F.rowsort, s_flag);
    if (ready) {
        const int H = F.H;
        const int r_lo = strip * F.strip_rows;
        const int r_hi = min(H, r_lo + F.strip_rows);
        // the window of right keypoint rows [w_a, w_b] the strip's bands can reach
        const int w_a = max(r_lo - P.halo, 0);
        const int w_b = min(r_hi - 1 + P.halo, H - 1);
        const int nrows = w_b - w_a + 1;
        const int e_base = __ldcg(F.row_ptr_r + w_a);
        const int e_end = __ldcg(F.row_ptr_r + w_b + 1);
        const int l_lo = __ldcg(F.row_ptr_l + r_lo), l_hi = __ldcg(F.row_ptr_l + r_hi);
        const int n_st = e_end - e_base;
        const bool staged = n_st <= kStageCap && nrows <= kWinRows && P.nlevels <= kOctBuckets;
        if (tid == 0) S.nref = 0;
        for (int pass = l_lo; pass < l_hi; pass += kThreads) {
            // the pass's left keypoints arrive by asynchronous copies while the
            // window is staged (again for a later pass: the previous pass's
            // patches overwrote it)
            const int npass = min(kThreads, l_hi - pass);
            if (tid < npass) {
                cp_async16(&S.u.st.left.lkp[tid], F.ls_kp + pass + tid);
                cp_async16(&S.u.st.left.ldesc[2 * tid], F.ls_desc + 2 * (pass + tid));
                cp_async16(&S.u.st.left.ldesc[2 * tid + 1], F.ls_desc + 2 * (pass + tid) + 1);
            }
            if (staged) stage_window(F, S, w_a, nrows, e_base, n_st);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            mark(B, 0);
            hamming_phase(P, F, S, npass, staged, w_a, nrows);
            // the refinement writes the grid records: the grid step must be done
            if (rec && pass == l_lo) ready = wait_geq(B, &F.ctr[C_GRID_DONE], (unsigned)F.n_grid_items, s_flag);
            else __syncthreads();
            mark(B, 1);
            const int nref = S.nref;
            for (int r0 = 0; r0 < nref; r0 += kSadChunk)
                refine_round(P, F, S, r0, min(kSadChunk, nref - r0), rec && ready);
            if (tid == 0) S.nref = 0;
            __syncthreads();
            mark(B, 2);
        }
    }
    if (signal_count(&F.ctr[C_STEREO_DONE], (unsigned)F.n_stereo_items, s_flag)) {
        // the rejection writes grid records too (this strip may have had no
        // keypoints to refine, so it has not waited for the grid step yet)
        if (rec && ready) ready = wait_geq(B, &F.ctr[C_GRID_DONE], (unsigned)F.n_grid_items, s_flag);
        median_reject(B, F, U.m, ready);
        __threadfence();
        __syncthreads();
        mark(B, 3);
        if (tid == 0 && !(B.debug_flags & kDebugWithholdStereoReady))
            atomicExch(&F.ctr[C_STEREO_READY], 1u);
    }
}

// ---------------------------------------------------------------- f1: fisheye triangulation
// sin and cos by their Taylor series (to t^13 and t^14; |t| <= 2 keeps the
// remainder under 2e-8), Horner in t^2, every operation explicitly rounded
__device__ __forceinline__ float sin_series(float t)
{
    const float t2 = fmul(t, t);
    float s = 1.60590444e-10f;               //  1/13!
    s = fadd(-2.50521079e-08f, fmul(t2, s)); // -1/11!
    s = fadd(2.75573188e-06f, fmul(t2, s));  //  1/9!
    s = fadd(-1.98412701e-04f, fmul(t2, s)); // -1/7!
    s = fadd(8.33333377e-03f, fmul(t2, s));  //  1/5!
    s = fadd(-1.66666672e-01f, fmul(t2, s)); // -1/3!
    s = fadd(1.0f, fmul(t2, s));
    return fmul(t, s);
}

__device__ __forceinline__ float cos_series(float t)
{
    const float t2 = fmul(t, t);
    float c = -1.14707454e-11f;              // -1/14!
    c = fadd(2.08767559e-09f, fmul(t2, c));  //  1/12!
    c = fadd(-2.75573200e-07f, fmul(t2, c)); // -1/10!
    c = fadd(2.48015876e-05f, fmul(t2, c));  //  1/8!
    c = fadd(-1.38888892e-03f, fmul(t2, c)); // -1/6!
    c = fadd(4.16666679e-02f, fmul(t2, c));  //  1/4!
    c = fadd(-0.5f, fmul(t2, c));            // -1/2!
    return fadd(1.0f, fmul(t2, c));
}

// Ray of a Kannala-Brandt pixel (kb = fx, fy, cx, cy, k1..k4): theta solves
// theta * (1 + k1 t + k2 t^2 + k3 t^3 + k4 t^4) = |m| (t = theta^2) by
// `iters` Newton steps from theta = |m|; false if the residual stays above
// 2e-6 rad, the model no longer rises there, or theta leaves [0, 2].
__device__ bool unproject_kb8(const float *kb, int iters, float u, float v, float *ray)
{
    const float mx = fdiv(fsub(u, kb[2]), kb[0]);
    const float my = fdiv(fsub(v, kb[3]), kb[1]);
    const float thd = fsqrt(fadd(fmul(mx, mx), fmul(my, my)));
    if (thd == 0.0f) {
        ray[0] = 0.0f;
        ray[1] = 0.0f;
        ray[2] = 1.0f;
        return true;
    }
    float th = thd, f = 0.0f, dp = 1.0f;
    for (int it = 0; it <= iters; ++it) {
        const float t2 = fmul(th, th);
        float poly = kb[7];
        poly = fadd(kb[6], fmul(t2, poly));
        poly = fadd(kb[5], fmul(t2, poly));
        poly = fadd(kb[4], fmul(t2, poly));
        poly = fadd(1.0f, fmul(t2, poly));
        f = fsub(fmul(th, poly), thd);
        dp = fmul(9.0f, kb[7]);
        dp = fadd(fmul(7.0f, kb[6]), fmul(t2, dp));
        dp = fadd(fmul(5.0f, kb[5]), fmul(t2, dp));
        dp = fadd(fmul(3.0f, kb[4]), fmul(t2, dp));
        dp = fadd(1.0f, fmul(t2, dp));
        if (it == iters) break;             // the last pass only measures the residual
        th = fsub(th, fdiv(f, dp));
    }
    if (!(fabsf(f) <= 2e-6f && dp > 0.0f && th >= 0.0f && th <= 2.0f)) return false;
    const float sn = fdiv(sin_series(th), thd);
    ray[0] = fmul(mx, sn);
    ray[1] = fmul(my, sn);
    ray[2] = cos_series(th);
    return true;
}

__device__ __forceinline__ float dot3f(const float *a, const float *b)
{
    return fadd(fadd(fmul(a[0], b[0]), fmul(a[1], b[1])), fmul(a[2], b[2]));
}

__device__ __forceinline__ void cross3f(const float *a, const float *b, float *c)
{
    c[0] = fsub(fmul(a[1], b[2]), fmul(a[2], b[1]));
    c[1] = fsub(fmul(a[2], b[0]), fmul(a[0], b[2]));
    c[2] = fsub(fmul(a[0], b[1]), fmul(a[1], b[0]));
}

// Midpoint of the common perpendicular of the left ray l (from the left
// centre) and the right ray r (right camera coordinates; X_r = R_rl X_l +
// t_rl), in left-camera coordinates: with C = -R^T t, d = R^T r and
// n = l x d, s = ((C x d).n)/(n.n), t = ((C x l).n)/(n.n).  Kept if the rays
// are not parallel, both parameters are positive and the depth exceeds
// min_depth.
__device__ bool triangulate(const float *l, const float *r, const float *R, const float *t, float min_depth,
                            float *X)
{
    float C[3], d[3], n[3], cd[3], cl[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        C[i] = -fadd(fadd(fmul(R[i], t[0]), fmul(R[3 + i], t[1])), fmul(R[6 + i], t[2]));
        d[i] = fadd(fadd(fmul(R[i], r[0]), fmul(R[3 + i], r[1])), fmul(R[6 + i], r[2]));
    }
    cross3f(l, d, n);
    const float nn = dot3f(n, n);
    if (!(nn > fmul(1e-10f, fmul(dot3f(l, l), dot3f(d, d))))) return false;
    cross3f(C, d, cd);
    cross3f(C, l, cl);
    const float s = fdiv(dot3f(cd, n), nn);
    const float tt = fdiv(dot3f(cl, n), nn);
    if (!(s > 0.0f && tt > 0.0f)) return false;
#pragma unroll
    for (int i = 0; i < 3; ++i) X[i] = fmul(0.5f, fadd(fmul(s, l[i]), fadd(C[i], fmul(tt, d[i]))));
    return X[2] > min_depth;
}

// f1 for left keypoint i with accepted right keypoint j (j < 0: none)
__device__ void triangulate_match(const DevParams &P, const FrameDev &F, int i, int j)
{
    float X[3] = {0.0f, 0.0f, 0.0f}, rl[3], rr[3];
    bool ok = false;
    if (j >= 0 && unproject_kb8(F.kbl, P.kb_iters, __ldg(F.lx + i), __ldg(F.ly + i), rl) &&
        unproject_kb8(F.kbr, P.kb_iters, __ldg(F.rx + j), __ldg(F.ry + j), rr))
        ok = triangulate(rl, rr, F.R_rl, F.t_rl, P.min_depth, X);
    F.fdepth[i] = ok ? X[2] : -1.0f;
    if (F.fxyz) F.fxyz[i] = ok ? make_float4(X[0], X[1], X[2], 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- K_STEREO, fisheye
__device__ void stereo_fisheye_item(const BatchHeader &B, const FrameDev &F, int tile, Smem &U,
                                    int *s_flag)
{
    // The item's left keypoints inside the overlap are compacted into a list;
    // kFishGroup lanes share each one, lane g comparing it with the staged
    // right overlap descriptors g, g + kFishGroup, ...; the lanes' top-2 keys
    // (distance << 20 | right index, all distinct) merge by shuffles into the
    // top-2 of the whole scan.
    SmemFish &S = U.f;
    const DevParams &P = B.p;
    const int tid = threadIdx.x;
    const int g = tid & (kFishGroup - 1), slot = tid / kFishGroup;
    const int i0 = tile * F.fisheye_tile, i1 = min(F.nl, i0 + F.fisheye_tile);
    if (tid == 0) S.nact = 0;
    __syncthreads();
    for (int i = i0 + tid; i < i1; i += kThreads) {
        const float x = __ldg(F.lx + i);
        if (x >= F.lap_l0 && x <= F.lap_l1) S.act[atomicAdd(&S.nact, 1)] = i;
    }
    __syncthreads();
    const int nact = S.nact;
    constexpr int Q = kFishTileMax / kFishSlots;    // passes: left keypoints per lane group
    int idx[Q];
    uint4 a0[Q], a1[Q];
    unsigned best[Q], second[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int a = q * kFishSlots + slot;
        idx[q] = a < nact ? S.act[a] : -1;
        best[q] = second[q] = kNoKey;
        if (idx[q] >= 0) {
            a0[q] = __ldg(F.ldesc + 2 * idx[q]);
            a1[q] = __ldg(F.ldesc + 2 * idx[q] + 1);
        }
    }
    if (nact > 0) {
        for (int c0 = 0; c0 < F.nr; c0 += kFishChunk) {
            if (tid == 0) S.count = 0;
            __syncthreads();
            const int c1 = min(F.nr, c0 + kFishChunk);
            for (int j = c0 + tid; j < c1; j += kThreads) {
                const float x = __ldg(F.rx + j);
                if (x >= F.lap_r0 && x <= F.lap_r1) {
                    const int pos = atomicAdd(&S.count, 1);
                    S.idx[pos] = j;
                    S.desc[2 * pos] = __ldg(F.rdesc + 2 * j);
                    S.desc[2 * pos + 1] = __ldg(F.rdesc + 2 * j + 1);
                }
            }
            __syncthreads();
            const int cnt = S.count;
            if (idx[0] >= 0) {
                for (int e = g; e < cnt; e += kFishGroup) {
                    const uint4 b0 = S.desc[2 * e], b1 = S.desc[2 * e + 1];
                    const unsigned j = (unsigned)S.idx[e];
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        if (idx[q] >= 0) top2_push(((unsigned)ham8(a0[q], a1[q], b0, b1) << 20) | j, best[q], second[q]);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int off = 1; off < kFishGroup; off <<= 1) {
            const unsigned ob = __shfl_xor_sync(kFull, best[q], off), os = __shfl_xor_sync(kFull, second[q], off);
            second[q] = min(min(second[q], os), max(best[q], ob));
            best[q] = min(best[q], ob);
        }
        if (idx[q] >= 0 && g == 0) {
            int r = -1, d2 = 256;
            const int d1 = best[q] != kNoKey ? (int)(best[q] >> 20) : -1;
            if (best[q] != kNoKey) {
                d2 = second[q] != kNoKey ? (int)(second[q] >> 20) : 256;
                if ((float)d1 < fmul(P.fisheye_ratio, (float)d2)) r = (int)(best[q] & 0xfffffu);
            } else {
                d2 = -1;
            }
            F.r_idx[idx[q]] = r;
            F.fd1[idx[q]] = d1;
            F.fd2[idx[q]] = d2;
            if (F.fdepth) triangulate_match(P, F, idx[q], r);
        }
    }
    // the item's keypoints outside the overlap: no match
    for (int i = i0 + tid; i < i1; i += kThreads) {
        const float x = __ldg(F.lx + i);
        if (x >= F.lap_l0 && x <= F.lap_l1) continue;
        F.r_idx[i] = -1;
        F.fd1[i] = -1;
        F.fd2[i] = -1;
        if (F.fdepth) triangulate_match(P, F, i, -1);
    }
    if (signal_count(&F.ctr[C_STEREO_DONE], (unsigned)F.n_stereo_items, s_flag)) {
        if (tid == 0 && !(B.debug_flags & kDebugWithholdStereoReady))
            atomicExch(&F.ctr[C_STEREO_READY], 1u);
    }
}

// ---------------------------------------------------------------- K_SEARCH
__device__ void resolve_range(const CamDev &C, int nm, int i0, int i1);

__device__ __forceinline__ void transform(const float *pose, float4 p, float &x, float &y, float &z)
{
    x = fadd(fadd(fadd(fmul(pose[0], p.x), fmul(pose[1], p.y)), fmul(pose[2], p.z)), pose[9]);
    y = fadd(fadd(fadd(fmul(pose[3], p.x), fmul(pose[4], p.y)), fmul(pose[5], p.z)), pose[10]);
    z = fadd(fadd(fadd(fmul(pose[6], p.x), fmul(pose[7], p.y)), fmul(pose[8], p.z)), pose[11]);
}

// distance window, viewing cosine, predicted level
__device__ __forceinline__ bool distance_scale(const DevParams &P, const float *O, float4 pos,
                                               float4 nrm, float &vc, int &level)
{
    const float px = fsub(pos.x, O[0]), py = fsub(pos.y, O[1]), pz = fsub(pos.z, O[2]);
    const float dist = fsqrt(fadd(fadd(fmul(px, px), fmul(py, py)), fmul(pz, pz)));
    const float d_far = fmul(P.dist_hi, nrm.w);
    const float d_near = fmul(P.dist_lo, pos.w);
    if (dist < d_near || dist > d_far) return false;
    vc = fdiv(fadd(fadd(fmul(px, nrm.x), fmul(py, nrm.y)), fmul(pz, nrm.z)), dist);
    if (vc < P.view_cos_min) return false;
    const float ratio = fdiv(nrm.w, dist);
    level = P.nlevels - 1;
    for (int l = 0; l < P.nlevels; ++l) {
        if (P.sc[l] >= ratio) {
            level = l;
            break;
        }
    }
    return true;
}

// a8 without the distance and viewing tests: camera z > 0 and the
// projection inside the image bounds
__device__ bool project_uv(const CamDev &C, const float *pose, float4 pos, float &u, float &v, float &ur)
{
    float x, y, z;
    transform(pose, pos, x, y, z);
    if (!(z > 0.0f)) return false;
    if (C.model == FT_CAMERA_PINHOLE) {
        const float invz = fdiv(1.0f, z);
        u = fadd(fmul(fmul(C.fx, x), invz), C.cx);
        v = fadd(fmul(fmul(C.fy, y), invz), C.cy);
        if (u < C.minx || u > C.maxx) return false;
        if (v < C.miny || v > C.maxy) return false;
        ur = fsub(u, fmul(C.bf, invz));
    } else {
        const float rho = fsqrt(fadd(fmul(x, x), fmul(y, y)));
        if (rho == 0.0f) {
            u = C.cx;
            v = C.cy;
        } else {
            const float theta = atan2_pos(rho, z);
            const float t2 = fmul(theta, theta);
            float poly = C.k[3];
            poly = fadd(C.k[2], fmul(t2, poly));
            poly = fadd(C.k[1], fmul(t2, poly));
            poly = fadd(C.k[0], fmul(t2, poly));
            poly = fadd(1.0f, fmul(t2, poly));
            const float thetad = fmul(theta, poly);
            u = fadd(fdiv(fmul(fmul(C.fx, thetad), x), rho), C.cx);
            v = fadd(fdiv(fmul(fmul(C.fy, thetad), y), rho), C.cy);
        }
        if (u < C.minx || u > C.maxx) return false;
        if (v < C.miny || v > C.maxy) return false;
        ur = -1.0f;
    }
    return true;
}

__device__ bool project(const DevParams &P, const CamDev &C, const float *pose, float4 pos,
                        float4 nrm, float &u, float &v, float &ur, float &vc, int &level)
{
    return project_uv(C, pose, pos, u, v, ur) && distance_scale(P, C.O, pos, nrm, vc, level);
}

// One map point against the keypoints of its search window.  kStaged: the
// camera's cell-ordered records and descriptors sit in shared memory.
// motion: for a last-frame search, +1 / -1 / 0 for a camera that moved
// forward / backward / neither along its viewing axis (f2).
// kScan: the first half of a search split around the stereo step.  Every
// test but the stereo consistency is applied; the four smallest keys
// (distance << 20 | keypoint) that pass, their octaves, the number that
// passed and the projection's right coordinate and radius go to C.scan for
// finish_point, which applies the consistency once the stereo step is done.
// The consistency test drops candidates and keys are unique, so the two
// smallest consistent keys among the four smallest candidates are the two
// smallest consistent candidates, unless fewer than two of the four are
// consistent while more than four passed: only then is the point searched
// again.
template <bool kStaged, bool kScan = false>
__device__ void search_point(const DevParams &P, const FrameDev &F, const CamDev &C, const SmemSearch &Q,
                             const uint16_t *scell, float iw, float ih, int m, int motion)
{
    const float *pose = Q.pose;
    const float4 *srec = reinterpret_cast<const float4 *>(Q.buf);
    const uint4 *sdesc = Q.buf + C.nk;
    const bool last = F.search_mode != 0;
    int lvl = -1, d1 = -1, d2 = -1, kp = -1;
    float4 pj = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned sk[4] = {kNoKey, kNoKey, kNoKey, kNoKey};   // kScan: four smallest keys, ascending
    unsigned soct = 0, scount = 0;                          // their octaves (a byte each), how many passed
    float sr = 0.0f, sur = 0.0f;
    const int loct = last ? (int)__ldg(F.last_oct + m) : 0;
    const bool skipped = (F.skip != nullptr && __ldg(F.skip + m) != 0) || (last && (loct < 0 || loct >= P.nlevels));
    if (!skipped) {
        const float4 pos = __ldg(F.pos + m);
        float u, v, ur, vc = 0.0f;
        int level = loct;
        const bool in_view = last ? project_uv(C, pose, pos, u, v, ur)
                                  : project(P, C, pose, pos, __ldg(F.nrm + m), u, v, ur, vc, level);
        if (in_view) {
            lvl = level;
            pj = make_float4(u, v, ur, vc);
            float r;
            int min_oct = level - 1, max_oct = level;
            if (last) {
                // f2: radius of the last octave, octave window by the motion
                r = fmul(P.th_last, P.sc[level]);
                min_oct = motion > 0 ? level : (motion < 0 ? 0 : level - 1);
                max_oct = motion > 0 ? P.nlevels - 1 : (motion < 0 ? level : level + 1);
            } else {
                r = (vc > P.view_cos_narrow) ? P.radius_narrow : P.radius_wide;
                r = fmul(r, P.search_th);
                r = fmul(r, P.sc[level]);
            }
            const float du = fsub(u, C.minx), dv = fsub(v, C.miny);
            const int x0 = max(f2i(floorf(fmul(fsub(du, r), iw))), 0);
            const int x1 = min(f2i(ceilf(fmul(fadd(du, r), iw))), FT_GRID_COLS - 1);
            const int y0 = max(f2i(floorf(fmul(fsub(dv, r), ih))), 0);
            const int y1 = min(f2i(ceilf(fmul(fadd(dv, r), ih))), FT_GRID_ROWS - 1);
            sr = r;
            sur = ur;
            if (!(x0 >= FT_GRID_COLS || x1 < 0 || y0 >= FT_GRID_ROWS || y1 < 0)) {
                const uint4 q0 = __ldg(F.mdesc + 2 * m), q1 = __ldg(F.mdesc + 2 * m + 1);
                const bool check_ur = C.model == FT_CAMERA_PINHOLE;
                unsigned best = kNoKey, second = kNoKey;
                int oct1 = -1, oct2 = -1;
                for (int cy = y0; cy <= y1; ++cy) {
                    int e0, e1;
                    if (kStaged && scell != nullptr) {
                        e0 = scell[cy * FT_GRID_COLS + x0];
                        e1 = scell[cy * FT_GRID_COLS + x1 + 1];
                    } else {
                        e0 = __ldcg(C.cell_ptr + cy * FT_GRID_COLS + x0);
                        e1 = __ldcg(C.cell_ptr + cy * FT_GRID_COLS + x1 + 1);
                    }
                    // records in device memory arrive kBatchRec at a time (one
                    // round trip), the descriptors of those that pass the tests after
                    constexpr int kBatchRec = kStaged ? 1 : 4;
                    for (int eb = e0; eb < e1; eb += kBatchRec) {
                        float4 gb[kBatchRec];
#pragma unroll
                        for (int q = 0; q < kBatchRec; ++q) {
                            if (kStaged) gb[q] = srec[eb + q];
                            else gb[q] = eb + q < e1 ? __ldcg(C.gkp + eb + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < kBatchRec; ++q) {
                            const int e = eb + q;
                            if (e >= e1) break;
                            const float4 g = gb[q];
                            const unsigned z = __float_as_uint(g.z);
                            const int k = (int)(z & 0xfffffu);
                            const int oct = (int)(int8_t)((z >> 20) & 0xffu);
                            if (oct < min_oct || oct > max_oct) continue;
                            const float distx = fsub(g.x, u), disty = fsub(g.y, v);
                            if (!(fabsf(distx) < r && fabsf(disty) < r)) continue;
                            if (z >> 28) continue;                         // taken
                            if (!kScan && check_ur && g.w > 0.0f && fabsf(fsub(ur, g.w)) > r) continue;
                            const uint4 b0 = kStaged ? sdesc[2 * e] : __ldcg(C.gdesc + 2 * e);
                            const uint4 b1 = kStaged ? sdesc[2 * e + 1] : __ldcg(C.gdesc + 2 * e + 1);
                            const unsigned key = ((unsigned)ham8(q0, q1, b0, b1) << 20) | (unsigned)k;
                            if (kScan) {
                                scount = min(scount + 1u, 255u);
                                const unsigned ob = (unsigned)oct & 0xffu;
                                if (key < sk[3]) {
                                    if (key < sk[2]) {
                                        sk[3] = sk[2];
                                        if (key < sk[1]) {
                                            sk[2] = sk[1];
                                            if (key < sk[0]) {
                                                sk[1] = sk[0];
                                                sk[0] = key;
                                                soct = (soct << 8) | ob;
                                            } else {
                                                sk[1] = key;
                                                soct = (soct & 0xffu) | ((soct << 8) & 0xff0000u) |
                                                       ((soct << 8) & 0xff000000u) | ob << 8;
                                            }
                                        } else {
                                            sk[2] = key;
                                            soct = (soct & 0xffffu) | ((soct << 8) & 0xff000000u) | ob << 16;
                                        }
                                    } else {
                                        sk[3] = key;
                                        soct = (soct & 0xffffffu) | ob << 24;
                                    }
                                }
                                continue;
                            }
                            if (key < best) {
                                second = best;
                                oct2 = oct1;
                                best = key;
                                oct1 = oct;
                            } else if (key < second) {
                                second = key;
                                oct2 = oct;
                            }
                        }
                    }
                }
                if (best != kNoKey) {
                    d1 = (int)(best >> 20);
                    d2 = second != kNoKey ? (int)(second >> 20) : 256;
                    if (d1 <= P.th_search) {
                        const int k1 = (int)(best & 0xfffffu);
                        const bool ratio = !last && (P.ratio_any_octave || oct1 == oct2);
                        if (!(ratio && (float)d1 > fmul(P.nn_ratio, (float)d2))) {
                            atomicMin(C.owner + k1, ((unsigned long long)d1 << 32) | (unsigned)m);
                            kp = k1;
                        }
                    }
                }
            }
        }
    }
    C.level[m] = (int8_t)lvl;
    if (C.proj) C.proj[m] = pj;
    if (kScan) {
        C.scan[2 * m] = make_uint4(sk[0], sk[1], sk[2], sk[3]);
        C.scan[2 * m + 1] = make_uint4(__float_as_uint(sur), __float_as_uint(sr), soct, scount);
        return;
    }
    C.mp_d1[m] = d1;
    C.mp_d2[m] = d2;
    C.mp_kp[m] = kp;
}

// The second half of a split search (see search_point): the stereo
// consistency applied to the four smallest candidates of map point m, then
// the top-2 rules and the claim, exactly as the unsplit search takes them.
// A point that needs more than its four smallest candidates is searched
// again from the device-memory records (whose right coordinates are final).
__device__ void finish_point(const DevParams &P, const FrameDev &F, const CamDev &C, const SmemSearch &Q, float iw,
                             float ih, int m, int motion)
{
    const uint4 ks = __ldcg(C.scan + 2 * m), aux = __ldcg(C.scan + 2 * m + 1);
    const unsigned sk[4] = {ks.x, ks.y, ks.z, ks.w};
    const float ur = __uint_as_float(aux.x), r = __uint_as_float(aux.y);
    const unsigned count = aux.w;
    const bool check_ur = C.model == FT_CAMERA_PINHOLE;
    const bool last = F.search_mode != 0;
    unsigned best = kNoKey, second = kNoKey;
    int oct1 = -1, oct2 = -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if ((unsigned)q >= count) break;
        const unsigned key = sk[q];
        const int k = (int)(key & 0xfffffu);
        if (k >= C.nk) continue;                     // never: keys name keypoints of the window
        if (check_ur) {
            const int e = __ldcg(C.gpos + k);
            if (e < 0) continue;                     // never: window keypoints lie in the grid
            const float w = __ldcg(&C.gkp[e].w);
            if (w > 0.0f && fabsf(fsub(ur, w)) > r) continue;
        }
        const int oct = (int)(int8_t)((aux.z >> (8 * q)) & 0xffu);
        if (best == kNoKey) {
            best = key;
            oct1 = oct;
        } else {
            second = key;
            oct2 = oct;
            break;
        }
    }
    if (count > 4u && second == kNoKey) {
        search_point<false>(P, F, C, Q, nullptr, iw, ih, m, motion);
        return;
    }
    int d1 = -1, d2 = -1, kp = -1;
    if (best != kNoKey) {
        d1 = (int)(best >> 20);
        d2 = second != kNoKey ? (int)(second >> 20) : 256;
        if (d1 <= P.th_search) {
            const int k1 = (int)(best & 0xfffffu);
            const bool ratio = !last && (P.ratio_any_octave || oct1 == oct2);
            if (!(ratio && (float)d1 > fmul(P.nn_ratio, (float)d2))) {
                atomicMin(C.owner + k1, ((unsigned long long)d1 << 32) | (unsigned)m);
                kp = k1;
            }
        }
    }
    C.mp_d1[m] = d1;
    C.mp_d2[m] = d2;
    C.mp_kp[m] = kp;
}

// The camera pose of a search item in shared memory (the right fisheye
// camera's composed from the rig), the grid scale and the last-frame motion.
__device__ void search_setup(const FrameDev &F, int cam, SmemSearch &Q, float &iw, float &ih, int &motion)
{
    const CamDev &C = F.cam[cam];
    const int tid = threadIdx.x;
    if (tid < 12) {
        const CamDev &L = F.cam[0];
        float v;
        if (cam == 0 || F.camera == FT_CAMERA_PINHOLE) {
            v = tid < 9 ? L.R[tid] : L.t[tid - 9];
        } else if (tid < 9) {      // right camera: R_rw = R_rl * R_lw
            const int i = tid / 3, j = tid % 3;
            v = fadd(fadd(fmul(F.R_rl[3 * i], L.R[j]), fmul(F.R_rl[3 * i + 1], L.R[3 + j])),
                     fmul(F.R_rl[3 * i + 2], L.R[6 + j]));
        } else {                   // t_rw = R_rl * t_lw + t_rl
            const int i = tid - 9;
            v = fadd(fadd(fadd(fmul(F.R_rl[3 * i], L.t[0]), fmul(F.R_rl[3 * i + 1], L.t[1])),
                          fmul(F.R_rl[3 * i + 2], L.t[2])),
                     F.t_rl[i]);
        }
        Q.pose[tid] = v;
    }
    iw = fdiv((float)FT_GRID_COLS, fsub(C.maxx, C.minx));
    ih = fdiv((float)FT_GRID_ROWS, fsub(C.maxy, C.miny));
    motion = 0;
    if (F.search_mode != 0) {
        // the current (left) camera centre in the last frame's camera
        // coordinates; its z against the baseline (f2)
        const float *O = F.cam[0].O;
        const float cz = fadd(fadd(fadd(fmul(F.last_R[6], O[0]), fmul(F.last_R[7], O[1])), fmul(F.last_R[8], O[2])),
                              F.last_t[2]);
        motion = cz > F.base ? 1 : (-cz > F.base ? -1 : 0);
    }
}

// Defined outputs of map points [m0, m1) after a wait ran out (reported in
// the status word).
__device__ void search_abandon(const CamDev &C, int m0, int m1)
{
    for (int m = m0 + (int)threadIdx.x; m < m1; m += kThreads) {
        C.level[m] = -1;
        if (C.proj) C.proj[m] = make_float4(0.f, 0.f, 0.f, 0.f);
        C.mp_d1[m] = -1;
        C.mp_d2[m] = -1;
        C.mp_kp[m] = -1;
    }
}

// A tile of map points.  A frame whose search is split around its stereo
// step (split_search) runs the first half of every point without waiting
// for the stereo step, then waits for it and finishes the points: the first
// half overlaps the wait.
__device__ void search_item(const BatchHeader &B, const FrameDev &F, int tile, Smem &U, int *s_flag)
{
    const int cam = tile < F.n_search_items[0] ? 0 : 1;
    const int t = cam ? tile - F.n_search_items[0] : tile;
    const bool split = F.split_search != 0;
    const int m0 = t * F.search_tile;
    const int m1 = min(F.nm, m0 + F.search_tile);
    // the tile's map point records do not depend on the stereo step: ask L2
    // for them before waiting for it
    for (int m = m0 + (int)threadIdx.x; m < m1; m += kThreads) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(F.pos + m));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(F.mdesc + 2 * m));
        if (F.search_mode == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(F.nrm + m));
    }
    bool ok = true;
    if (F.wait_stereo && !split) ok = wait_geq(B, &F.ctr[C_STEREO_READY], 1u, s_flag);
    if (ok) ok = wait_geq(B, &F.ctr[C_GRID_DONE], (unsigned)F.n_grid_items, s_flag);
    const CamDev &C = F.cam[cam];
    if (ok) {
        SmemSearch &Q = U.q;
        const int tid = threadIdx.x;
        float iw, ih;
        int motion;
        search_setup(F, cam, Q, iw, ih, motion);
        // stage the camera's cell-ordered keypoint records and descriptors
        // by asynchronous copies when they fit (the tail past the placed
        // records is copied but never read)
        const int nk = C.nk;
        const bool staged = F.search_stage == 0 && nk <= kSearchStage;
        // the 16-bit cell starts too when they fit behind the descriptors
        const bool cells = staged && 48 * nk + kCell16Bytes <= (int)sizeof(Q.buf);
        const uint16_t *scell = cells ? reinterpret_cast<const uint16_t *>(Q.buf + 3 * nk) : nullptr;
        if (staged) {
            for (int e = tid; e < nk; e += kThreads) cp_async16(Q.buf + e, C.gkp + e);
            for (int e = tid; e < 2 * nk; e += kThreads) cp_async16(Q.buf + nk + e, C.gdesc + e);
            if (cells)
                for (int c = tid; c < kCell16Bytes / 16; c += kThreads)
                    cp_async16(Q.buf + 3 * nk + c, reinterpret_cast<const uint4 *>(C.cell16) + c);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();
        mark(B, 0);
        if (split) {
            // first halves (the staged records' right coordinates are not
            // read: they may not be final yet), then the stereo step, then
            // the second halves; each thread finishes the points it scanned
            if (staged) {
                for (int m = m0 + tid; m < m1; m += kThreads)
                    search_point<true, true>(B.p, F, C, Q, scell, iw, ih, m, motion);
            } else {
                for (int m = m0 + tid; m < m1; m += kThreads)
                    search_point<false, true>(B.p, F, C, Q, nullptr, iw, ih, m, motion);
            }
            mark(B, 1);
            if (wait_geq(B, &F.ctr[C_STEREO_READY], 1u, s_flag)) {
                for (int m = m0 + tid; m < m1; m += kThreads) finish_point(B.p, F, C, Q, iw, ih, m, motion);
            } else {
                search_abandon(C, m0, m1);
            }
            mark(B, 2);
        } else if (staged) {
            for (int m = m0 + tid; m < m1; m += kThreads) search_point<true>(B.p, F, C, Q, scell, iw, ih, m, motion);
            mark(B, 1);
        } else {
            for (int m = m0 + tid; m < m1; m += kThreads)
                search_point<false>(B.p, F, C, Q, nullptr, iw, ih, m, motion);
            mark(B, 1);
        }
    } else {
        search_abandon(C, m0, m1);
    }
    if (signal_count(&F.ctr[C_SEARCH_DONE0 + cam], (unsigned)F.n_search_items[cam], s_flag) &&
        F.fold_resolve) {
        // the last search item of this camera also writes the final tables
        // (small frames: no separate resolve items wait for the search)
        resolve_range(F.cam[cam], F.nm, 0, max(F.nm, F.cam[cam].nk));
    }
}

// ---------------------------------------------------------------- K_RESOLVE
// Final tables for entries [i0, i1): a map point keeps its keypoint only if
// it owns it; a keypoint gets its owner (or -1).  A thread takes kResolveBatch
// entries at a time and issues all their loads before any store, so a
// range's dependent reads (map point -> keypoint -> owner) cost two L2 round
// trips per batch rather than per entry.
constexpr int kResolveBatch = 8;

__device__ void resolve_range(const CamDev &C, int nm, int i0, int i1)
{
    const int me = min(i1, nm), ke = min(i1, C.nk);
    for (int m0 = i0 + (int)threadIdx.x; m0 < me; m0 += kThreads * kResolveBatch) {
        int kk[kResolveBatch];
#pragma unroll
        for (int u = 0; u < kResolveBatch; ++u) {
            const int m = m0 + u * kThreads;
            kk[u] = m < me ? __ldcg(C.mp_kp + m) : -1;
        }
        unsigned own[kResolveBatch];
#pragma unroll
        for (int u = 0; u < kResolveBatch; ++u)
            own[u] = kk[u] >= 0 && kk[u] < C.nk ? (unsigned)(__ldcg(C.owner + kk[u]) & 0xffffffffull) : 0u;
#pragma unroll
        for (int u = 0; u < kResolveBatch; ++u) {
            const int m = m0 + u * kThreads;
            if (m >= me || kk[u] < 0) continue;
            if (kk[u] >= C.nk || own[u] != (unsigned)m) C.mp_kp[m] = -1;   // never written / not the owner
        }
    }
    for (int k0 = i0 + (int)threadIdx.x; k0 < ke; k0 += kThreads * kResolveBatch) {
        unsigned long long own[kResolveBatch];
#pragma unroll
        for (int u = 0; u < kResolveBatch; ++u) {
            const int k = k0 + u * kThreads;
            own[u] = k < ke ? __ldcg(C.owner + k) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < kResolveBatch; ++u) {
            const int k = k0 + u * kThreads;
            if (k < ke) C.kp_mp[k] = own[u] == ~0ull ? -1 : (int)(own[u] & 0xffffffffull);
        }
    }
}

__device__ void resolve_item(const BatchHeader &B, const FrameDev &F, int tile, int *s_flag)
{
    const int cam = tile < F.n_resolve_items[0] ? 0 : 1;
    const int t = cam ? tile - F.n_resolve_items[0] : tile;
    // the grid build initialises the owners (a frame without map points has no
    // search item to order the two)
    const CamDev &C = F.cam[cam];
    const int i0 = t * F.resolve_tile, i1 = i0 + F.resolve_tile;
    if (!wait_geq(B, &F.ctr[C_GRID_DONE], (unsigned)F.n_grid_items, s_flag) ||
        !wait_geq(B, &F.ctr[C_SEARCH_DONE0 + cam], (unsigned)F.n_search_items[cam], s_flag)) {
        // the wait ran out (reported in the status word): leave defined outputs
        for (int m = i0 + threadIdx.x; m < min(i1, F.nm); m += kThreads) C.mp_kp[m] = -1;
        for (int k = i0 + threadIdx.x; k < min(i1, C.nk); k += kThreads) C.kp_mp[k] = -1;
        return;
    }
    resolve_range(C, F.nm, i0, i1);
}

// ---------------------------------------------------------------- the kernel
__device__ __forceinline__ void copy_words(void *dst, const void *src, size_t bytes)
{
    const unsigned *a = reinterpret_cast<const unsigned *>(src);
    unsigned *b = reinterpret_cast<unsigned *>(dst);
    for (size_t i = threadIdx.x; i < bytes / 4; i += kThreads) b[i] = __ldg(a + i);
}

__global__ void __launch_bounds__(kThreads, FT_MIN_CTAS_PER_SM) ft_fused_kernel(const BatchHeader *__restrict__ hdr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &U = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ int s_item;
    __shared__ int s_flag;
    // the launch header and the current frame's descriptor live in shared
    // memory: their many indexed fields (level sizes, pitches, scales) are
    // then shared-memory loads instead of dependent global loads
    __shared__ __align__(16) BatchHeader sB;
    __shared__ __align__(16) FrameDev sF;
    copy_words(&sB, hdr, sizeof(BatchHeader));
    __syncthreads();
    const BatchHeader &B = sB;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(B.queue, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= B.total_items) break;
        int kind = 0;
        while (kind < K_KINDS - 1 && item >= B.kind_begin[kind + 1]) ++kind;
        const int local = item - B.kind_begin[kind];
        const int *pre = B.prefix + kind * (B.nframes + 1);
        int lo = 0, hi = B.nframes - 1;          // last frame f with pre[f] <= local
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= local) lo = mid;
            else hi = mid - 1;
        }
        copy_words(&sF, B.frames + lo, sizeof(FrameDev));
        __syncthreads();
        const FrameDev &F = sF;
        const int tile = local - pre[lo];
        unsigned long long t_start = 0;
        if (B.trace != nullptr && threadIdx.x == 0) {
            t_start = global_ns();
            s_wait_ns = 0;
            s_mark[0] = s_mark[1] = s_mark[2] = s_mark[3] = 0;
        }
        switch (kind) {
        case K_INDEX:
            if (tile < F.rowsort) {
                rowsort_item(B, F, U.r, tile >= kSortParts, tile % kSortParts, &s_flag);
            } else {
                grid_item(B, F, tile - F.rowsort, U.g, &s_flag);
            }
            break;
        case K_STEREO:
            if (F.camera == FT_CAMERA_PINHOLE) stereo_pinhole_item(B, F, tile, U, &s_flag);
            else stereo_fisheye_item(B, F, tile, U, &s_flag);
            break;
        case K_SEARCH: search_item(B, F, tile, U, &s_flag); break;
        default: resolve_item(B, F, tile, &s_flag); break;
        }
        if (B.trace != nullptr && threadIdx.x == 0) {
            const unsigned slot = atomicAdd(B.queue + 1, 1u);
            if (slot < (unsigned)B.trace_cap) {
                unsigned sm;
                asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
                ft_trace_record r;
                r.item = item;
                r.kind = kind;
                r.frame = lo;
                r.sm = (int)sm;
                r.t_start = t_start;
                r.t_end = global_ns();
                r.wait_ns = s_wait_ns;
                for (int q = 0; q < 4; ++q) r.mark[q] = s_mark[q];
                B.trace[slot] = r;
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- f4: pose optimization
// The refinement of the camera pose with all the map points the search found
// in the frame (paper section II-D; FastTrack switches it off, section
// IV-F), as the algorithm family's motion-only optimization (a reading):
// observations are the matched keypoints (x, y) and, where stereo gave one,
// u_right; weight 1/scale[oct]^2; po_rounds rounds of po_iters Gauss-Newton
// steps over the inliers with Huber weights, the update exp(d) multiplied on
// the left of the pose; every observation reclassified by its chi2 after
// each round.  FP32.  A kernel of its own, after the fused kernel on the
// same stream (the matches are final by then): one block of kPoseThreads
// per frame.  Every thread accumulates the normal equations of its
// observations, each warp reduce-scatters its 27 sums (lane q ends with sum
// q), warp 0 adds the warps in a fixed order and lane 0 solves the 6x6
// system (Cholesky) and updates the pose.  The observations stay in shared
// memory when they fit; they are read at every step.
namespace {

constexpr int kPoseThreads = 512;
constexpr int kPoseWarps = kPoseThreads / 32;
constexpr int kPoseStage = 2048;                 // observations kept on chip
constexpr int kPoseSmem = 2 * kPoseStage * (int)sizeof(float4);

struct PoseShared {
    float part[kPoseWarps][32];
    float tot[32];
    float Rt[12];
    int warp_sums[kPoseWarps];
    int n_in, ok, total;
};

// observation (a, b) at pose Rt: residual, chi2 and Jacobian rows (rotation
// then translation of the left perturbation); false if not in front
struct PoseObs {
    float e[3], J[3][6], chi2;
    bool stereo;
};

__device__ __forceinline__ bool pose_obs(const CamDev &C, const float *Rt, float4 a, float4 b, PoseObs &o)
{
    const float x = Rt[0] * a.x + Rt[1] * a.y + Rt[2] * a.z + Rt[9];
    const float y = Rt[3] * a.x + Rt[4] * a.y + Rt[5] * a.z + Rt[10];
    const float z = Rt[6] * a.x + Rt[7] * a.y + Rt[8] * a.z + Rt[11];
    if (!(z > 0.0f)) return false;
    const float iz = 1.0f / z, iz2 = iz * iz;
    const float u = C.fx * x * iz + C.cx, v = C.fy * y * iz + C.cy;
    o.stereo = b.z >= 0.0f;
    o.e[0] = b.x - u;
    o.e[1] = b.y - v;
    o.e[2] = o.stereo ? b.z - (u - C.bf * iz) : 0.0f;
    o.chi2 = a.w * (o.e[0] * o.e[0] + o.e[1] * o.e[1] + o.e[2] * o.e[2]);
    // d projection / d Pc, times d Pc / d (w, v) = [ -[Pc]x | I ]
    const float D[3][3] = {{C.fx * iz, 0.0f, -C.fx * x * iz2},
                           {0.0f, C.fy * iz, -C.fy * y * iz2},
                           {C.fx * iz, 0.0f, -C.fx * x * iz2 + C.bf * iz2}};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        o.J[r][0] = -D[r][1] * z + D[r][2] * y;
        o.J[r][1] = D[r][0] * z - D[r][2] * x;
        o.J[r][2] = -D[r][0] * y + D[r][1] * x;
        o.J[r][3] = D[r][0];
        o.J[r][4] = D[r][1];
        o.J[r][5] = D[r][2];
    }
    return true;
}

// lane 0 of warp 0: solve H d = g (H as its upper triangle, row by row, in
// tot[0..20], g in tot[21..26]) by Cholesky with one reciprocal per column,
// then (R, t) <- exp(d) (R, t); ok = 0 if H is not positive definite
__device__ void pose_step(PoseShared &S)
{
    float H[6][6], L[6][6], inv[6], y[6], d[6];
    int q = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) H[i][j] = H[j][i] = S.tot[q++];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float s = H[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0f)) {
            S.ok = 0;
            return;
        }
        L[j][j] = sqrtf(s);
        inv[j] = 1.0f / L[j][j];
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            float t = H[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t * inv[j];
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float s = S.tot[21 + i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s * inv[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        float s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * d[k];
        d[i] = s * inv[i];
    }
    // exp of the twist d = (w, v): R_d = I + a [w]x + b [w]x^2,
    // V = I + b [w]x + c [w]x^2 (series of a, b, c below theta = 0.01)
    const float th2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float th = sqrtf(th2);
    float a, b, c;
    if (th < 0.01f) {
        a = 1.0f - th2 / 6.0f;
        b = 0.5f - th2 / 24.0f;
        c = 1.0f / 6.0f - th2 / 120.0f;
    } else {
        const float sn = sinf(th), cs = cosf(th);
        a = sn / th;
        b = (1.0f - cs) / th2;
        c = (th - sn) / (th2 * th);
    }
    const float W[9] = {0.0f, -d[2], d[1], d[2], 0.0f, -d[0], -d[1], d[0], 0.0f};
    float W2[9], Rd[9], V[9], Rn[12];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            W2[3 * i + j] = W[3 * i] * W[j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float id = (i % 4 == 0) ? 1.0f : 0.0f;
        Rd[i] = id + a * W[i] + b * W2[i];
        V[i] = id + b * W[i] + c * W2[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rn[3 * i + j] = Rd[3 * i] * S.Rt[j] + Rd[3 * i + 1] * S.Rt[3 + j] + Rd[3 * i + 2] * S.Rt[6 + j];
        Rn[9 + i] = Rd[3 * i] * S.Rt[9] + Rd[3 * i + 1] * S.Rt[10] + Rd[3 * i + 2] * S.Rt[11] +
                    V[3 * i] * d[3] + V[3 * i + 1] * d[4] + V[3 * i + 2] * d[5];
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) S.Rt[i] = Rn[i];
}

// block-wide sum of one int per thread (all threads get it)
__device__ int pose_block_sum(int v, PoseShared &S)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_add_sync(kFull, v);
    if (lane == 0) S.warp_sums[w] = v;
    __syncthreads();
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kPoseWarps; ++i) sum += S.warp_sums[i];
    __syncthreads();
    return sum;
}

__global__ void __launch_bounds__(kPoseThreads, 1) ft_pose_kernel(const BatchHeader *__restrict__ hdr)
{
    extern __shared__ __align__(16) float4 pose_stage[];
    __shared__ PoseShared S;
    __shared__ __align__(16) DevParams sP;
    __shared__ __align__(16) FrameDev sF;
    const int f = blockIdx.x;
    if (f >= hdr->nframes || !hdr->frames[f].do_pose) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const unsigned *a = reinterpret_cast<const unsigned *>(hdr->frames + f);
        unsigned *b = reinterpret_cast<unsigned *>(&sF);
        for (int i = tid; i < (int)(sizeof(FrameDev) / 4); i += kPoseThreads) b[i] = __ldg(a + i);
        const unsigned *pa = reinterpret_cast<const unsigned *>(&hdr->p);
        unsigned *pb = reinterpret_cast<unsigned *>(&sP);
        for (int i = tid; i < (int)(sizeof(DevParams) / 4); i += kPoseThreads) pb[i] = __ldg(pa + i);
    }
    __syncthreads();
    const FrameDev &F = sF;
    const DevParams &P = sP;
    const CamDev &C = F.cam[0];
    const int M = F.nm;
    if (tid < 9) S.Rt[tid] = C.R[tid];
    else if (tid < 12) S.Rt[tid] = C.t[tid - 9];
    // observations in map-point order: thread tid takes a contiguous chunk of
    // map points, counts its matches, and writes them after the chunks before
    const int per = (M + kPoseThreads - 1) / kPoseThreads;
    const int m0 = min(M, tid * per), m1 = min(M, m0 + per);
    int cnt = 0;
    for (int m = m0; m < m1; ++m) {
        const int k = __ldg(F.po_mp_kp + m);
        cnt += (k >= 0 && k < C.nk) ? 1 : 0;
    }
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) S.warp_sums[warp] = x;
    __syncthreads();
    int pos = x - cnt, total = 0;
#pragma unroll
    for (int i = 0; i < kPoseWarps; ++i) {
        const int ws = S.warp_sums[i];
        pos += i < warp ? ws : 0;
        total += ws;
    }
    __syncthreads();
    float4 *list = total <= kPoseStage ? pose_stage : F.po_list;
    for (int m = m0; m < m1; ++m) {
        const int k = __ldg(F.po_mp_kp + m);
        const bool valid = k >= 0 && k < C.nk;
        F.po_inlier[m] = valid ? 1 : -1;
        if (!valid) continue;
        const float4 Pw = __ldg(F.pos + m);
        const int oct = __ldg(C.koct + k);
        const float sc = (oct >= 0 && oct < P.nlevels) ? P.sc[oct] : 1.0f;
        const float ur = F.u_right_in ? __ldg(F.u_right_in + k) : -1.0f;
        list[2 * pos] = make_float4(Pw.x, Pw.y, Pw.z, 1.0f / (sc * sc));
        list[2 * pos + 1] = make_float4(__ldg(C.kx + k), __ldg(C.ky + k), ur >= 0.0f ? ur : -1.0f,
                                        __int_as_float(m | (int)0x80000000));
        ++pos;
    }
    if (tid == 0) {
        S.n_in = total;
        S.ok = 1;
    }
    __syncthreads();
    const float th_mono = P.po_chi2_mono, th_stereo = P.po_chi2_stereo;
    for (int round = 0; round < P.po_rounds; ++round) {
        if (S.n_in < 3) break;
        for (int it = 0; it < P.po_iters; ++it) {
            float acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
            for (int e = tid; e < total; e += kPoseThreads) {
                const float4 a = list[2 * e], b = list[2 * e + 1];
                if (__float_as_int(b.w) >= 0) continue;            // outlier
                PoseObs o;
                if (!pose_obs(C, S.Rt, a, b, o)) continue;
                const float th = o.stereo ? th_stereo : th_mono;
                const float h = (!P.po_huber || o.chi2 <= th) ? 1.0f : sqrtf(th / o.chi2);
                const float hw = h * a.w;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (r == 2 && !o.stereo) break;
                    int q = 0;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const float wi = hw * o.J[r][i];
#pragma unroll
                        for (int j = i; j < 6; ++j) acc[q++] += wi * o.J[r][j];
                        acc[21 + i] += wi * o.e[r];
                    }
                }
            }
            // reduce-scatter: after the five butterfly stages lane q holds
            // the warp's sum of entry q
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const bool upper = (lane & s) != 0;
#pragma unroll
                for (int i = 0; i < s; ++i) {
                    const float send = upper ? acc[i] : acc[i + s];
                    const float keep = upper ? acc[i + s] : acc[i];
                    acc[i] = keep + __shfl_xor_sync(kFull, send, s);
                }
            }
            S.part[warp][lane] = acc[0];
            __syncthreads();
            if (warp == 0) {
                float v = 0.0f;
#pragma unroll
                for (int w = 0; w < kPoseWarps; ++w) v += S.part[w][lane];
                S.tot[lane] = v;
                __syncwarp();
                if (lane == 0) pose_step(S);
            }
            __syncthreads();
            if (!S.ok) break;
        }
        // classify every observation at the new pose
        int n_in = 0;
        for (int e = tid; e < total; e += kPoseThreads) {
            const float4 a = list[2 * e];
            float4 b = list[2 * e + 1];
            PoseObs o;
            bool in = pose_obs(C, S.Rt, a, b, o);
            if (in) in = !(o.chi2 > (o.stereo ? th_stereo : th_mono));
            const int m = __float_as_int(b.w) & 0x7fffffff;
            b.w = __int_as_float(in ? (m | (int)0x80000000) : m);
            list[2 * e + 1] = b;
            n_in += in ? 1 : 0;
        }
        const int all = pose_block_sum(n_in, S);
        if (tid == 0) S.n_in = all;
        __syncthreads();
        if (!S.ok) break;
    }
    for (int e = tid; e < total; e += kPoseThreads) {
        const int w = __float_as_int(list[2 * e + 1].w);
        F.po_inlier[w & 0x7fffffff] = w < 0 ? 1 : 0;
    }
    if (tid < 12) F.po_Rt[tid] = S.Rt[tid];
    if (tid == 0) *F.po_n = S.n_in;
}

}  // namespace

int fused_smem_bytes() { return (int)sizeof(Smem); }

const void *fused_kernel_ptr() { return (const void *)ft_fused_kernel; }

cudaError_t fused_occupancy(int *ctas_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(ft_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ft_pose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPoseSmem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, ft_fused_kernel, kThreads,
                                                         sizeof(Smem));
}

cudaError_t launch_fused(const BatchHeader *dev_hdr, int grid, cudaStream_t stream)
{
    ft_fused_kernel<<<grid, kThreads, sizeof(Smem), stream>>>(dev_hdr);
    return cudaGetLastError();
}

cudaError_t launch_pose(const BatchHeader *dev_hdr, int nframes, cudaStream_t stream)
{
    if (nframes <= 0) return cudaSuccess;
    ft_pose_kernel<<<nframes, kPoseThreads, kPoseSmem, stream>>>(dev_hdr);
    return cudaGetLastError();
}

}  // namespace ft
