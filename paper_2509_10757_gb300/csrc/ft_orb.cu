// ft_orb.cu -- keypoint detection and description on the pyramid levels
// (next row f3).  The paper's ORB extraction builds the image pyramid, finds
// keypoints on every level, describes each one and filters them (section
// II-A); FastTrack reuses an existing GPU extractor (section IV-B) and
// prints none of its steps.  This file implements the reading stated in the
// public header: FAST-9 corners with the maximum-threshold score, 3x3
// non-maximum suppression (ties: the earlier raster position), the best
// max_kp[l] corners per level by (score descending, y, x) in fixed slots,
// intensity-centroid orientation over the radius-15 disk, and 256 steered
// tests on the level smoothed by the 5x5 binomial filter.
//
// Three launches per call, each over every image of the call:
//   detect    one block of 256 threads per 32x32 tile of a level: the tile
//             and a 4-pixel halo in shared memory as two planes of packed
//             pixel pairs, the FAST score of every pixel of the tile and its
//             one-pixel ring (two pixels per step in 16-bit lanes, both
//             polarities by three-input packed min/max), a 16-bit
//             suppression key per pixel that orders score and raster
//             position at once, suppression as one comparison with the
//             eight neighbours' largest key, the kept corners appended as
//             keys (255 - score) << 24 | y << 12 | x (one atomic per warp),
//             and the smoothed level written from the same tile (separable,
//             two pixels per word);
//   select    one block per (image, level): the max_kp-th smallest key by an
//             exact 4 x 8-bit radix select over the level's corners, the
//             keys up to it gathered and sorted (bitonic) in shared memory;
//   describe  one warp per output slot: the keypoint's two neighbourhoods
//             (level and smoothed level) copied to shared memory in one
//             round trip of 16-byte asynchronous copies, the moments over
//             the disk (integer warp sums), the orientation, and lane b
//             computes descriptor byte b (tests 8b .. 8b+7).
// Integer work is exact; the orientation and the rotated test positions use
// IEEE-rounded FP32 in the order the reading gives (the moment magnitude,
// a double square root rounded to float in the reading, is the same value
// from an FP32 square root settled by integer comparisons: ft_sqrt.h), so
// results equal the oracle's bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "ft_internal.h"
#include "ft_sqrt.h"

namespace ft {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDetThreads = 256;
constexpr int kTileW = kOrbTile + 2 * kOrbHalo;     // tile + halo: 40 columns and rows
constexpr int kHalfW = kTileW / 2;                  // words per row of a pixel-pair plane
constexpr int kRing = kOrbTile + 2;                 // tile + suppression ring
constexpr int kPairs = kRing / 2;                   // pixel pairs per ring row (= words per key row)
constexpr int kHsW = kOrbTile / 2 + 1;              // words per row of horizontal sums (+1: no bank conflicts)
constexpr int kDescribeWarps = 8;
static_assert(kDetThreads == 8 * kOrbTile, "suppression: 16 pairs x 2 rows per warp, 2 steps");

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Offsets of the 16 pixels of the radius-3 circle, clockwise from (0, -3):
// x offsets 0 1 2 3 3 3 2 1 0 -1 -2 -3 -3 -3 -2 -1, stored + 3 as 4-bit
// nibbles of one constant; the y offset of pixel i is the x offset of pixel
// i + 12.
__device__ __forceinline__ int circle_dx(int i)
{
    constexpr unsigned long long kPacked = 0x2100012345666543ull;
    return (int)((kPacked >> (4 * i)) & 15ull) - 3;
}
__device__ __forceinline__ int circle_dy(int i) { return circle_dx((i + 12) & 15); }

// lane-wise minimum / maximum of two pixel pairs (16-bit lanes)
__device__ __forceinline__ unsigned vmin2(unsigned a, unsigned b) { return __vminu2(a, b); }
__device__ __forceinline__ unsigned vmax2(unsigned a, unsigned b) { return __vmaxu2(a, b); }

// The best arc of a pixel pair's 16 circle values v (one pixel per 16-bit
// lane): for kBright the largest, over the 16 arcs of 9 contiguous circle
// pixels, of the arc's smallest value; otherwise the smallest of the arcs'
// largest values.  Three-input packed min/max: the extremes of the 16 arcs
// of 3, those of the arcs of 9 as three arcs of 3 (i, i + 3, i + 6), then
// the best of the 16 in a tree (40 operations per polarity; the form with
// running extremes over blocks of 9, 57 two-input operations, measured 3 %
// slower over the whole extraction).
template <bool kBright>
__device__ __forceinline__ unsigned best_arc(const unsigned (&v)[16])
{
    auto in3 = [](unsigned a, unsigned b, unsigned c) { return kBright ? __vimin3_u16x2(a, b, c) : __vimax3_u16x2(a, b, c); };
    auto out3 = [](unsigned a, unsigned b, unsigned c) { return kBright ? __vimax3_u16x2(a, b, c) : __vimin3_u16x2(a, b, c); };
    unsigned w3[16], w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w3[i] = in3(v[i], v[(i + 1) & 15], v[(i + 2) & 15]);
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = in3(w3[i], w3[(i + 3) & 15], w3[(i + 6) & 15]);
    const unsigned r0 = out3(w[0], w[1], w[2]), r1 = out3(w[3], w[4], w[5]), r2 = out3(w[6], w[7], w[8]);
    const unsigned r3 = out3(w[9], w[10], w[11]), r4 = out3(w[12], w[13], w[14]);
    const unsigned q0 = out3(r0, r1, r2), q1 = out3(r3, r4, w[15]);
    return kBright ? vmax2(q0, q1) : vmin2(q0, q1);
}

// One block per 32 x 32 tile of a level.  The tile and its 4-pixel halo are
// held as two planes of pixel pairs: pe[r][k] packs the pixels of halo
// columns 2k and 2k + 1 of halo row r in its low and high 16-bit lanes,
// po[r][k] those of columns 2k + 1 and 2k + 2.  Any two horizontally adjacent
// pixels are then one word, and a warp's pixel pairs read consecutive words.
// Every pixel of the tile and of its one-pixel ring gets a suppression key:
// 0 where it is not a corner, else (FAST score + 1) << 8 | (255 - g) with
// g = 3 * ring row + ring column.  Between 8-neighbours, 3 * dy + dx orders
// the earlier raster position first, so "the neighbour's score is larger,
// or equal and the neighbour comes first" is "the neighbour's key is larger"
// and a corner survives suppression when its key exceeds its 8 neighbours'.
__global__ void __launch_bounds__(kDetThreads, 5) orb_detect_kernel(const OrbHeader *__restrict__ hdr)
{
    __shared__ __align__(16) unsigned pe[kTileW][kHalfW];
    __shared__ __align__(16) unsigned po[kTileW][kHalfW];
    __shared__ unsigned key[kRing][kPairs];             // two 16-bit keys per word
    __shared__ unsigned hs[kOrbTile + 4][kHsW];         // horizontal binomial sums of rows -2 .. T+1, two per word
    const OrbHeader &H = *hdr;
    const OrbImage &I = H.images[blockIdx.y];
    const int tile = blockIdx.x;
    if (tile >= I.tiles) return;
    int l = 0;
    for (int k = 1; k < H.nlevels; ++k)
        if (I.lv[k].tile0 <= tile) l = k;
    const OrbLevel &L = I.lv[l];
    const int t = tile - L.tile0;
    const int x0 = (t % L.tiles_x) * kOrbTile, y0 = (t / L.tiles_x) * kOrbTile;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tile == 0 && tid == 0) I.n_level[H.nlevels] = 0;     // the select blocks add to it
    // the tile and its halo; coordinates are clamped to the level (the
    // smoothing replicates the border; FAST only runs where its circle is
    // inside).  Tiles whose halo lies inside the level read whole words
    // (level rows are 16-byte aligned: checked on the host).
    if (x0 >= kOrbHalo && y0 >= kOrbHalo && x0 + kOrbTile + kOrbHalo <= L.w && y0 + kOrbTile + kOrbHalo <= L.h) {
        constexpr int kWords = kTileW / 4;
        for (int i = tid; i < kTileW * kWords; i += kDetThreads) {
            const int r = i / kWords, m = i - r * kWords;
            const unsigned *row =
                reinterpret_cast<const unsigned *>(L.img + (size_t)(y0 - kOrbHalo + r) * L.pitch + x0 - kOrbHalo);
            const unsigned a = __ldg(row + m), b = m + 1 < kWords ? __ldg(row + m + 1) : 0u;
            *reinterpret_cast<uint2 *>(&pe[r][2 * m]) = make_uint2(__byte_perm(a, 0u, 0x4140), __byte_perm(a, 0u, 0x4342));
            *reinterpret_cast<uint2 *>(&po[r][2 * m]) =
                make_uint2(__byte_perm(a, 0u, 0x4241), __byte_perm(__funnelshift_r(a, b, 24), 0u, 0x4140));
        }
    } else {
        for (int i = tid; i < kTileW * kHalfW; i += kDetThreads) {
            const int r = i / kHalfW, k = i - r * kHalfW;
            const uint8_t *row = L.img + (size_t)clampi(y0 - kOrbHalo + r, 0, L.h - 1) * L.pitch;
            const int xa = x0 - kOrbHalo + 2 * k;
            const unsigned a = row[clampi(xa, 0, L.w - 1)], b = row[clampi(xa + 1, 0, L.w - 1)],
                           c = row[clampi(xa + 2, 0, L.w - 1)];
            pe[r][k] = a | (b << 16);
            po[r][k] = b | (c << 16);
        }
    }
    __syncthreads();
    // keys of the tile and its ring, two adjacent pixels (ring columns 2h,
    // 2h + 1) per step; the pair's centre is po[ry + 3][h + 1]
    const int E = H.edge, th = H.fast_th;
    const bool ring_in = x0 - 1 >= E && x0 + kOrbTile < L.w - E && y0 - 1 >= E && y0 + kOrbTile < L.h - E;
    for (int q = tid; q < kRing * kPairs; q += kDetThreads) {
        const int ry = q / kPairs, h = q - ry * kPairs;
        // pixels closer than E to a border (or outside the level) are not
        // corners; a pair with neither pixel inside is not scored (a warp of
        // such pairs, as on a tile that overhangs the level, skips the work)
        bool in0 = true, in1 = true;
        if (!ring_in) {
            const int px = x0 - 1 + 2 * h, py = y0 - 1 + ry;
            const bool rows_in = py >= E && py < L.h - E;
            in0 = rows_in && px >= E && px < L.w - E;
            in1 = rows_in && px + 1 >= E && px + 1 < L.w - E;
        }
        unsigned k0 = 0u, k1 = 0u;
        if (in0 || in1) {
            const unsigned c = po[ry + 3][h + 1];
            unsigned v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int dx = circle_dx(i), dy = circle_dy(i);     // halo column of the pair: 2h + 3 + dx
                v[i] = (dx & 1) ? pe[ry + 3 + dy][h + ((3 + dx) >> 1)] : po[ry + 3 + dy][h + 1 + (dx >> 1)];
            }
            // the best arc's smallest difference, over both polarities, + 256
            // in each lane (bright: arc minimum - centre, dark: centre - arc
            // maximum; the lanes stay in [1, 511])
            const unsigned e = vmax2(best_arc<true>(v) + 0x01000100u - c, c + 0x01000100u - best_arc<false>(v));
            const int b0 = (int)(e & 0xffffu) - 256, b1 = (int)(e >> 16) - 256;
            const unsigned g = 3u * (unsigned)ry + 2u * (unsigned)h;
            if (in0 && b0 > th) k0 = ((unsigned)b0 << 8) | (255u - g);
            if (in1 && b1 > th) k1 = ((unsigned)b1 << 8) | (254u - g);
        }
        key[ry][h] = k0 | (k1 << 16);
    }
    // horizontal binomial sums (1 4 6 4 1) of halo rows 2 .. 37, output
    // columns 2k and 2k + 1 (taps at halo columns 2k + 2 .. 2k + 7)
    for (int q = (tid + kDetThreads / 2) % kDetThreads; q < (kOrbTile + 4) * (kOrbTile / 2); q += kDetThreads) {
        const int r = q / (kOrbTile / 2), k = q % (kOrbTile / 2);
        const unsigned *e = pe[r + 2], *o = po[r + 2];
        hs[r][k] = e[k + 1] + 4u * o[k + 1] + 6u * e[k + 2] + 4u * o[k + 2] + e[k + 3];
    }
    __syncthreads();
    // suppression and smoothing: thread (h, row) owns tile pixels (2h, iy)
    // and (2h + 1, iy) for iy = row, row + 8 (a warp: 16 pairs of rows 16
    // apart, so its key and sum words fall in distinct banks)
    const int h = tid & 15;
    const int row0 = (tid >> 5) + 16 * ((tid >> 4) & 1);
    unsigned kv[4];
    bool kf[4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int iy = row0 + 8 * s;
        const unsigned a0 = key[iy][h], a1 = key[iy][h + 1];
        const unsigned b0 = key[iy + 1][h], b1 = key[iy + 1][h + 1];
        const unsigned c0 = key[iy + 2][h], c1 = key[iy + 2][h + 1];
        const unsigned mid = __byte_perm(b0, b1, 0x5432);      // ring columns 2h + 1, 2h + 2 of ring row iy + 1
        const unsigned up = vmax2(vmax2(a0, a1), __byte_perm(a0, a1, 0x5432));
        const unsigned dn = vmax2(vmax2(c0, c1), __byte_perm(c0, c1, 0x5432));
        const unsigned m = vmax2(vmax2(up, dn), vmax2(b0, b1));
        const int py = y0 + iy, px = x0 + 2 * h;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const unsigned kp = j ? mid >> 16 : mid & 0xffffu, km = j ? m >> 16 : m & 0xffffu;
            kf[2 * s + j] = kp > km;
            kv[2 * s + j] = ((256u - (kp >> 8)) << 24) | ((unsigned)py << 12) | (unsigned)(px + j);
        }
        if (py < L.h && px < L.w) {
            const unsigned acc =
                hs[iy][h] + 4u * hs[iy + 1][h] + 6u * hs[iy + 2][h] + 4u * hs[iy + 3][h] + hs[iy + 4][h] + 0x00800080u;
            uint8_t *o = L.smooth + (size_t)py * L.spitch + px;
            const unsigned sv = __byte_perm(acc, 0u, 0x4431);       // the two lanes' bits 8-15
            if (px + 1 < L.w) *reinterpret_cast<uint16_t *>(o) = (uint16_t)sv;
            else o[0] = (uint8_t)sv;
        }
    }
    // one atomic per warp reserves the warp's corners
    const int nkeep = (int)kf[0] + (int)kf[1] + (int)kf[2] + (int)kf[3];
    int incl = nkeep;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(&I.cnt[l], (unsigned)total);
    base = __shfl_sync(kFull, base, 31);
    int at = (int)base + incl - nkeep;
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (kf[s]) {
            if (at < L.cand_cap) L.cand[at] = kv[s];
            ++at;
        }
}

__global__ void __launch_bounds__(kOrbSelectThreads) orb_select_kernel(const OrbHeader *__restrict__ hdr)
{
    __shared__ unsigned keys[kOrbMaxSlots];
    __shared__ int hist[256];
    __shared__ unsigned s_prefix;
    __shared__ int s_rank, s_n;
    const OrbHeader &H = *hdr;
    const int l = blockIdx.x;
    if (l >= H.nlevels) return;
    const OrbImage &I = H.images[blockIdx.y];
    const OrbLevel &L = I.lv[l];
    const int tid = threadIdx.x;
    const int c = min((int)I.cnt[l], L.cand_cap);
    const int K = L.max_kp;
    unsigned kth = 0xffffffffu;
    if (c > K && K > 0) {
        // the K-th smallest key (keys are distinct): one byte per pass
        unsigned prefix = 0, mask = 0;
        int rank = K;
        for (int b = 3; b >= 0; --b) {
            if (tid < 256) hist[tid] = 0;
            __syncthreads();
            for (int i = tid; i < c; i += kOrbSelectThreads) {
                const unsigned k = L.cand[i];
                if ((k & mask) == prefix) atomicAdd(&hist[(k >> (8 * b)) & 255u], 1);
            }
            __syncthreads();
            if (tid < 32) {
                // the first bin whose running count reaches the rank: lane t
                // sums bins 8t .. 8t + 7, a warp scan finds the lane
                int s8 = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) s8 += hist[8 * tid + q];
                int incl = s8;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(kFull, incl, o);
                    if (tid >= o) incl += v;
                }
                const unsigned hit = __ballot_sync(kFull, incl >= rank);
                if (tid == __ffs(hit) - 1) {
                    int cum = incl - s8;
                    for (int q = 0; q < 8; ++q) {
                        const int bin = 8 * tid + q;
                        if (cum + hist[bin] >= rank) {
                            s_prefix = prefix | ((unsigned)bin << (8 * b));
                            s_rank = rank - cum;
                            break;
                        }
                        cum += hist[bin];
                    }
                }
            }
            __syncthreads();
            prefix = s_prefix;
            rank = s_rank;
            mask |= 255u << (8 * b);
            __syncthreads();
        }
        kth = prefix;
    }
    if (tid == 0) s_n = 0;
    __syncthreads();
    for (int i = tid; i < c; i += kOrbSelectThreads) {
        const unsigned k = L.cand[i];
        if (k <= kth) {
            const int at = atomicAdd(&s_n, 1);
            if (at < kOrbMaxSlots) keys[at] = k;
        }
    }
    __syncthreads();
    const int n = min(s_n, K);
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + tid; i < P; i += kOrbSelectThreads) keys[i] = 0xffffffffu;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += kOrbSelectThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned a = keys[i], b = keys[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < n; i += kOrbSelectThreads) I.sel[L.slot0 + i] = keys[i];
    if (tid == 0) {
        I.n_level[l] = n;
        atomicAdd(&I.n_level[H.nlevels], n);
    }
}

// Staged neighbourhoods of one keypoint (one warp): rows y - 15 .. y + 15 of
// the level for the moments and rows y - 18 .. y + 18 of the smoothed level
// for the tests (rotated pattern points within [-13, 13]^2 land within
// round(13 sqrt 2) = 18 pixels), each row copied from the 16-byte boundary at
// or before its first column.
constexpr int kMomR = 15, kTestR = 18;
constexpr int kMomRows = 2 * kMomR + 1, kTestRows = 2 * kTestR + 1;
constexpr int kMomChunks = 3, kTestChunks = 4;      // 16-byte chunks per staged row (31 + 15, 37 + 15 bytes)
constexpr int kMomStride = 16 * kMomChunks, kTestStride = 16 * kTestChunks;
constexpr int kStageCopies = kMomRows * kMomChunks + kTestRows * kTestChunks;

__device__ __forceinline__ void copy16_async(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

__global__ void __launch_bounds__(32 * kDescribeWarps, 7) orb_describe_kernel(const OrbHeader *__restrict__ hdr)
{
    __shared__ __align__(16) uint8_t mom[kDescribeWarps][kMomRows * kMomStride];
    __shared__ __align__(16) uint8_t tst[kDescribeWarps][kTestRows * kTestStride];
    const OrbHeader &H = *hdr;
    const OrbImage &I = H.images[blockIdx.y];
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int slot = blockIdx.x * kDescribeWarps + wv;
    if (slot >= I.nslots) return;
    int l = 0;
    for (int k = 0; k < H.nlevels; ++k)
        if (slot >= I.lv[k].slot0 && slot < I.lv[k].slot0 + I.lv[k].max_kp) l = k;
    const OrbLevel &L = I.lv[l];
    const int i = slot - L.slot0;
    if (i >= I.n_level[l]) {
        // a slot without a keypoint
        if (lane == 0) {
            I.x[slot] = -1.0e9f;
            I.y[slot] = -1.0e9f;
            I.oct[slot] = 0;
            I.score[slot] = -1;
            I.cs[2 * slot] = 1.0f;
            I.cs[2 * slot + 1] = 0.0f;
        }
        I.desc[(size_t)slot * 32 + lane] = 0;
        return;
    }
    const unsigned key = I.sel[slot];
    const int x = (int)(key & 4095u), y = (int)((key >> 12) & 4095u);
    // both neighbourhoods in one round trip; keypoints lie at least 19
    // pixels inside the level, and a chunk that holds a column of a row
    // lies inside the row's 16-byte padded pitch
    const int a1 = (x - kMomR) & ~15, n1 = ((x + kMomR) >> 4) - (a1 >> 4) + 1;
    const int a0 = (x - kTestR) & ~15, n0 = ((x + kTestR) >> 4) - (a0 >> 4) + 1;
    for (int j = lane; j < kStageCopies; j += 32) {
        if (j < kMomRows * kMomChunks) {
            const int r = j / kMomChunks, ch = j - r * kMomChunks;
            if (ch < n1)
                copy16_async(&mom[wv][r * kMomStride + 16 * ch],
                             L.img + (size_t)(y - kMomR + r) * L.pitch + a1 + 16 * ch);
        } else {
            const int jt = j - kMomRows * kMomChunks, r = jt / kTestChunks, ch = jt - r * kTestChunks;
            if (ch < n0)
                copy16_async(&tst[wv][r * kTestStride + 16 * ch],
                             L.smooth + (size_t)(y - kTestR + r) * L.spitch + a0 + 16 * ch);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
    // intensity centroid over the disk u^2 + v^2 <= 225 (exact integer
    // sums): lane u + 15 walks column u (lane 31 idles)
    int m10 = 0, m01 = 0;
    if (lane < kMomRows) {
        const int u = lane - kMomR;
        const uint8_t *col = &mom[wv][x - a1 + u];          // row v + 15 at col[(v + 15) * stride]
        int sum = 0;
#pragma unroll
        for (int v = -kMomR; v <= kMomR; ++v)
            if (u * u <= kMomR * kMomR - v * v) {
                const int p = col[(v + kMomR) * kMomStride];
                sum += p;
                m01 += v * p;
            }
        m10 = u * sum;
    }
    m10 = __reduce_add_sync(kFull, m10);
    m01 = __reduce_add_sync(kFull, m01);
    float c = 1.0f, s = 0.0f;
    if (m10 != 0 || m01 != 0) {
        // |m| = sqrt(m10^2 + m01^2) as the double square root rounded to
        // float, which for these integers is the correctly rounded FP32
        // square root (ft_sqrt.h)
        const float nm = float_sqrt_rn((uint64_t)((long long)m10 * m10 + (long long)m01 * m01));
        c = __fdiv_rn((float)m10, nm);
        s = __fdiv_rn((float)m01, nm);
    }
    // byte `lane` of the descriptor: tests 8 lane .. 8 lane + 7 (their 32
    // pattern coordinates in two 16-byte loads)
    const uint8_t *tp = &tst[wv][kTestR * kTestStride + (x - a0)];
    const uint4 *pw = reinterpret_cast<const uint4 *>(H.pattern) + 2 * lane;
    const uint4 pa = __ldg(pw), pb = __ldg(pw + 1);
    const unsigned pws[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
    unsigned byte = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int val[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // test point q: bytes 2q (x) and 2q + 1 (y) of the test's word, signed
            const int xi = (int)(pws[k] << (24 - 16 * q)) >> 24, yi = (int)(pws[k] << (16 - 16 * q)) >> 24;
            const float px = (float)xi, py = (float)yi;
            const int u = (int)roundf(__fsub_rn(__fmul_rn(c, px), __fmul_rn(s, py)));
            const int v = (int)roundf(__fadd_rn(__fmul_rn(s, px), __fmul_rn(c, py)));
            val[q] = tp[v * kTestStride + u];
        }
        byte |= (val[0] < val[1] ? 1u : 0u) << k;
    }
    I.desc[(size_t)slot * 32 + lane] = (uint8_t)byte;
    if (lane == 0) {
        I.x[slot] = __fmul_rn((float)x, H.sc[l]);
        I.y[slot] = __fmul_rn((float)y, H.sc[l]);
        I.oct[slot] = (int8_t)l;
        I.score[slot] = 255 - (int)(key >> 24);
        I.cs[2 * slot] = c;
        I.cs[2 * slot + 1] = s;
    }
}

}  // namespace

cudaError_t launch_orb(const OrbHeader *dev_hdr, int nimages, int nlevels, int max_tiles, int max_slots,
                       cudaStream_t stream)
{
    if (nimages <= 0) return cudaSuccess;
    orb_detect_kernel<<<dim3((unsigned)max(max_tiles, 1), (unsigned)nimages), kDetThreads, 0, stream>>>(
        dev_hdr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    orb_select_kernel<<<dim3((unsigned)nlevels, (unsigned)nimages), kOrbSelectThreads, 0, stream>>>(dev_hdr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((max(max_slots, 1) + kDescribeWarps - 1) / kDescribeWarps);
    orb_describe_kernel<<<dim3(blocks, (unsigned)nimages), 32 * kDescribeWarps, 0, stream>>>(dev_hdr);
    return cudaGetLastError();
}

}  // namespace ft
