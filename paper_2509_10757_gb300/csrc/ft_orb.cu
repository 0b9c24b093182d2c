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
//             and a 4-pixel halo in shared memory, the FAST score of every
//             pixel of the tile and its one-pixel ring (two pixels per step
//             in packed 16-bit lanes), suppression against the eight
//             neighbours, the kept corners appended as keys
//             (255 - score) << 24 | y << 12 | x (one atomic per warp), and
//             the smoothed level written from the same tile (separable);
//   select    one block per (image, level): the max_kp-th smallest key by an
//             exact 4 x 8-bit radix select over the level's corners, the
//             keys up to it gathered and sorted (bitonic) in shared memory;
//   describe  one warp per output slot: the moments over the disk (lanes
//             stride over it, integer warp sums), the orientation, and lane b
//             computes descriptor byte b (tests 8b .. 8b+7).
// Integer work is exact; the orientation and the rotated test positions use
// IEEE-rounded FP32 (and one double square root) in the order the reading
// gives, so results equal the oracle's bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "ft_internal.h"

namespace ft {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDetThreads = 256;
constexpr int kTileW = kOrbTile + 2 * kOrbHalo;     // tile + halo
constexpr int kRing = kOrbTile + 2;                 // tile + suppression ring
constexpr int kRows = kOrbTile / (kDetThreads / kOrbTile);   // output rows per thread
constexpr int kDescribeWarps = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
__device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

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

// binomial weights 1 4 6 4 1
__device__ __forceinline__ int binomial5(int j) { return j == 2 ? 6 : ((j & 1) ? 4 : 1); }

// FAST-9 scores of the horizontally adjacent pixels (cx, cy) and (cx + 1, cy)
// of the shared tile, -1 where a pixel is not a corner at t.  The score is
// the best arc's smallest difference minus one, over both polarities.  The
// pair's 16 circle differences travel as biased 16-bit lanes (v - c + 256 in
// [1, 511], the first pixel in the low lane): minima (bright) and maxima
// (dark) over windows of 3, then of 9, by three-input packed min/max, then
// the best window.  Every pixel gets its score (no branch on the segment
// test): a corner is a pixel whose best arc exceeds t.
__device__ __forceinline__ void fast_score2(const uint8_t (*raw)[kTileW], int cx, int cy, int t, int &s0, int &s1)
{
    const unsigned c = (unsigned)raw[cy][cx] | ((unsigned)raw[cy][cx + 1] << 16);
    unsigned b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int yy = cy + circle_dy(i), xx = cx + circle_dx(i);
        b[i] = ((unsigned)raw[yy][xx] | ((unsigned)raw[yy][xx + 1] << 16)) + 0x01000100u - c;
    }
    unsigned lo3[22], hi3[22];
#pragma unroll
    for (int i = 0; i < 22; ++i) {
        lo3[i] = __vimin3_u16x2(b[i & 15], b[(i + 1) & 15], b[(i + 2) & 15]);
        hi3[i] = __vimax3_u16x2(b[i & 15], b[(i + 1) & 15], b[(i + 2) & 15]);
    }
    unsigned best_lo = 0u, least_hi = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const unsigned m = __vimin3_u16x2(lo3[i], lo3[i + 3], lo3[i + 6]);
        const unsigned M = __vimax3_u16x2(hi3[i], hi3[i + 3], hi3[i + 6]);
        best_lo = __vimax3_u16x2(best_lo, m, m);
        least_hi = __vimin3_u16x2(least_hi, M, M);
    }
    const int b0 = imax((int)(best_lo & 0xffffu) - 256, 256 - (int)(least_hi & 0xffffu));
    const int b1 = imax((int)(best_lo >> 16) - 256, 256 - (int)(least_hi >> 16));
    s0 = b0 > t ? b0 - 1 : -1;
    s1 = b1 > t ? b1 - 1 : -1;
}

__global__ void __launch_bounds__(kDetThreads) orb_detect_kernel(const OrbHeader *__restrict__ hdr)
{
    __shared__ uint8_t raw[kTileW][kTileW];
    __shared__ short sco[kRing][kRing];
    __shared__ short hs[kOrbTile + 4][kOrbTile];      // horizontal binomial sums of rows -2 .. T+1
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
    // the tile and its halo, coordinates clamped to the level (the smoothing
    // replicates the border; FAST only runs where its circle is inside)
    for (int i = tid; i < kTileW * kTileW; i += kDetThreads) {
        const int yy = clampi(y0 - kOrbHalo + i / kTileW, 0, L.h - 1);
        const int xx = clampi(x0 - kOrbHalo + i % kTileW, 0, L.w - 1);
        raw[i / kTileW][i % kTileW] = L.img[(size_t)yy * L.pitch + xx];
    }
    __syncthreads();
    // scores of the tile and its one-pixel ring, two adjacent pixels per step
    const int E = H.edge;
    constexpr int kPairs = kRing / 2;
    for (int q = tid; q < kRing * kPairs; q += kDetThreads) {
        const int ry = q / kPairs, rx = 2 * (q % kPairs);
        int s0, s1;
        fast_score2(raw, rx + 3, ry + 3, H.fast_th, s0, s1);
        const int px = x0 - 1 + rx, py = y0 - 1 + ry;
        const bool rows_in = py >= E && py < L.h - E;
        sco[ry][rx] = (short)((rows_in && px >= E && px < L.w - E) ? s0 : -1);
        sco[ry][rx + 1] = (short)((rows_in && px + 1 >= E && px + 1 < L.w - E) ? s1 : -1);
    }
    for (int q = tid; q < (kOrbTile + 4) * kOrbTile; q += kDetThreads) {
        const int r = q / kOrbTile, x = q % kOrbTile;
        int a = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) a += binomial5(i) * (int)raw[r + kOrbHalo - 2][x + kOrbHalo - 2 + i];
        hs[r][x] = (short)a;
    }
    __syncthreads();
    // suppression: thread (ix, iy) owns the pixels of column ix, rows iy + k * (T / kRows)
    const int ix = tid % kOrbTile, iy0 = tid / kOrbTile;
    unsigned keys[kRows];
    int nkeep = 0;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int iy = iy0 + k * (kDetThreads / kOrbTile);
        const int sp = sco[iy + 1][ix + 1];
        bool keep = sp >= 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int q = sco[iy + 1 + dy][ix + 1 + dx];
                const bool earlier = dy < 0 || (dy == 0 && dx < 0);
                if (q >= 0 && (q > sp || (q == sp && earlier))) keep = false;
            }
        if (keep) keys[nkeep++] = ((unsigned)(255 - sp) << 24) | ((unsigned)(y0 + iy) << 12) | (unsigned)(x0 + ix);
        const int px = x0 + ix, py = y0 + iy;
        if (px < L.w && py < L.h) {
            int acc = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc += binomial5(j) * (int)hs[iy + j][ix];
            L.smooth[(size_t)py * L.w + px] = (uint8_t)((acc + 128) >> 8);
        }
    }
    // one atomic per warp reserves the warp's corners
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
    for (int k = 0; k < nkeep; ++k, ++at)
        if (at < L.cand_cap) L.cand[at] = keys[k];
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
    if (c > K) {
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
            if (tid == 0) {
                int cum = 0;
                for (int bin = 0; bin < 256; ++bin) {
                    if (cum + hist[bin] >= rank) {
                        s_prefix = prefix | ((unsigned)bin << (8 * b));
                        s_rank = rank - cum;
                        break;
                    }
                    cum += hist[bin];
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

__global__ void __launch_bounds__(32 * kDescribeWarps) orb_describe_kernel(const OrbHeader *__restrict__ hdr)
{
    const OrbHeader &H = *hdr;
    const OrbImage &I = H.images[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * kDescribeWarps + (threadIdx.x >> 5);
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
    // intensity centroid over the disk u^2 + v^2 <= 225 (exact integer sums)
    // all 31 loads of a lane are issued before any is used (unrolled)
    int m10 = 0, m01 = 0;
    int pix[31];
#pragma unroll
    for (int r = 0; r < 31; ++r) {
        const int q = lane + 32 * r;
        const int u = q % 31 - 15, v = q / 31 - 15;
        pix[r] = (q < 31 * 31 && u * u + v * v <= 225) ? (int)L.img[(size_t)(y + v) * L.pitch + (x + u)] : 0;
    }
#pragma unroll
    for (int r = 0; r < 31; ++r) {
        const int q = lane + 32 * r;
        m10 += (q % 31 - 15) * pix[r];
        m01 += (q / 31 - 15) * pix[r];
    }
    m10 = __reduce_add_sync(kFull, m10);
    m01 = __reduce_add_sync(kFull, m01);
    float c = 1.0f, s = 0.0f;
    if (m10 != 0 || m01 != 0) {
        const double n2 = __dadd_rn(__dmul_rn((double)m10, (double)m10), __dmul_rn((double)m01, (double)m01));
        const float nm = __double2float_rn(__dsqrt_rn(n2));
        c = __fdiv_rn((float)m10, nm);
        s = __fdiv_rn((float)m01, nm);
    }
    // byte `lane` of the descriptor: tests 8 lane .. 8 lane + 7
    unsigned byte = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int8_t *pt = H.pattern + 4 * (8 * lane + k);
        int val[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float px = (float)pt[2 * q], py = (float)pt[2 * q + 1];
            const int u = (int)roundf(__fsub_rn(__fmul_rn(c, px), __fmul_rn(s, py)));
            const int v = (int)roundf(__fadd_rn(__fmul_rn(s, px), __fmul_rn(c, py)));
            val[q] = L.smooth[(size_t)(y + v) * L.w + (x + u)];
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
