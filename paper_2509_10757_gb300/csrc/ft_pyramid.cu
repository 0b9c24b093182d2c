// ft_pyramid.cu -- levels 1.. of an image pyramid resampled from level 0 on
// the device (next row f3, the pyramid part).  The paper builds the pyramid
// on the GPU as part of its ORB extraction so that it never crosses the bus
// (section IV-B) and prints no resampling; the library's reading: level l is
// round(W / sc[l]) x round(H / sc[l]); pixel (x, y) samples level 0 at
// xs = (x + 0.5) * (W / w) - 0.5 (ys likewise), clamped to the image,
// bilinear in FP32 in the order top = I00 (1 - fx) + I01 fx, bottom
// likewise, value = top (1 - fy) + bottom fy, rounded half to even.  Every
// level comes straight from level 0.
//
// One block per tile of level 0: kPyrTileRows source rows (plus the next
// row) by kPyrTileCols source columns (plus the next 16).  The block
//   1. reads the tile with 16-byte loads and stores it in shared memory as
//      floats (each source byte is converted once, for every level);
//   2. finds, for every level, the output rows whose upper source row y0
//      and the output columns whose left source column c0 lie in the tile
//      (searches over the same FP32 operations as the formula, one lane of
//      the last warp per level while the tile loads are in flight; y0 and
//      c0 never decrease along a level), and tabulates those rows'
//      source-row offsets and vertical weights;
//   3. gives each thread kPyrCols output columns (x, x + 32, ...) of one
//      level at a time (all levels' columns in one list, so few threads
//      idle) and walks those columns' rows in the tile, keeping the
//      horizontal interpolations of the last bottom source row for the next
//      output row when it is the next row's top.  The lanes of a warp take
//      32 neighbouring columns, so the byte stores of a row coalesce.
// The image's last column and row are repeated past the tile's staged ones
// where the tile reaches the image's edge, so the formula's clamped c1 and y1
// are always the staged c0 + 1 and y0 + 1.
// Every tile is independent: no block waits for another.
//
// A byte b becomes the float b exactly by placing it in the mantissa of 2^23
// and subtracting 2^23.  Products and sums are single FP32 operations with
// explicit rounding (a multiply feeding an add is never contracted into a
// fused multiply-add).  The value v lies in [0, 255] up to rounding (a
// convex combination of bytes), so adding 1.5 * 2^23 rounds it to the
// nearest integer, ties to even, and the low mantissa byte is the result.
// Levels therefore equal the per-pixel formula bit for bit.
#include "ft_internal.h"

#ifndef FT_PYR_COLS
#define FT_PYR_COLS 4
#endif

namespace ft {
namespace {

constexpr int kPyrCols = FT_PYR_COLS;        // output columns per thread (32 apart)

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ int f2i(float x) { return __float2int_rz(x); }   // C (int) cast

typedef unsigned long long f32x2;        // lane 0 in the low 32 bits

__device__ __forceinline__ f32x2 f2_pack(unsigned lo, unsigned hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 a, unsigned &lo, unsigned &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(a));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

constexpr unsigned kExp23 = 0x4B000000u;     // bits of 2^23
constexpr float kTwo23 = 8388608.0f;         // 2^23
constexpr float kRound23 = 12582912.0f;      // 1.5 * 2^23

// Upper source row (or left source column) of output coordinate y of a level
// with scale s = (source size) / (level size): the formula's operations.
__device__ __forceinline__ float pyr_src(int y, float s, int n)
{
    const float ys = fsub(fmul(fadd((float)y, 0.5f), s), 0.5f);
    return fminf(fmaxf(ys, 0.0f), (float)(n - 1));
}
__device__ __forceinline__ int pyr_floor(int y, float s, int n) { return f2i(floorf(pyr_src(y, s, n))); }

// First output coordinate in [0, m] whose floor source coordinate is >= t
// (m if none); the floor never decreases with the coordinate.  Starts from
// the real-valued solution of (y + 0.5) s - 0.5 = t and steps to the exact
// answer (one or two steps: the estimate is off by less than one).
__device__ int pyr_first_at_least(int t, float s, int n, int m)
{
    int y = (int)ceilf(fsub(fdiv(fadd((float)t, 0.5f), s), 0.5f));
    y = min(max(y, 0), m);
    while (y > 0 && pyr_floor(y - 1, s, n) >= t) --y;
    while (y < m && pyr_floor(y, s, n) < t) ++y;
    return y;
}

// Per level of the tile: output rows [ylo, ylo + nrows), output columns
// [xlo, xlo + ncols) (the columns from the level's width to its width
// rounded up to 4 get zeros), and the level's first unit.  A unit is one
// thread's kPyrCols columns x, x + 32, ... of a group of 32 kPyrCols
// columns, so a warp (32 units) covers one group of one level.
struct PyrLevelInfo {
    int ylo, nrows, xlo, ncols, wreal, unit0, dp;
    float sx;
    uint8_t *dst;
};

// A tile's output row of a level in the row table: its upper source row r0
// (offset in floats of the staged tile; the lower one is the next staged
// row), weights fy and 1 - fy, and the row's byte offset in the level.
struct alignas(16) PyrRow {
    unsigned r0;
    float fy, gy;
    unsigned doff;
};

__global__ void __launch_bounds__(kPyrThreads, 4) ft_pyramid_kernel(const BatchHeader *__restrict__ hdr)
{
    extern __shared__ float4 pyr_smem[];
    float *tile = reinterpret_cast<float *>(pyr_smem);                       // [kPyrTileRows + 1][kPyrStride]
    PyrRow *tab = reinterpret_cast<PyrRow *>(tile + (kPyrTileRows + 1) * kPyrStride);   // [levels][kPyrRowsPerLevel]
    __shared__ PyrLevelInfo info[FT_MAX_LEVELS + 1];

    const int f = (int)(blockIdx.y >> 1), side = (int)(blockIdx.y & 1);
    if (f >= hdr->nframes) return;
    const FrameDev &F = hdr->frames[f];
    if (!(F.build_pyr & (1 << side))) return;
    const int nl = hdr->p.nlevels;
    const uint8_t *src = side ? F.pyrR[0] : F.pyrL[0];
    const int *lw = side ? F.rw : F.lw, *lh = side ? F.rh : F.lh, *lp = side ? F.rp : F.lp;
    const int W = lw[0], H = lh[0], sp = lp[0];
    const int ntx = (W + kPyrTileCols - 1) / kPyrTileCols;
    if ((int)blockIdx.x >= pyr_tiles(W, H)) return;
    const int Y0 = ((int)blockIdx.x / ntx) * kPyrTileRows, X0 = ((int)blockIdx.x % ntx) * kPyrTileCols;
    const int tid = (int)threadIdx.x;

    // 1. the tile as floats: source rows Y0 .. Y0 + nr - 1, bytes X0 .. X0 +
    // nb - 1 (16-byte chunks; W rounded up to 16 is within the pitch)
    const int nr = min(kPyrTileRows + 1, H - Y0);
    const int nch = min(kPyrStride, ((W + 15) & ~15) - X0) >> 4;
    for (int k = tid; k < nr * nch; k += kPyrThreads) {
        const int r = k / nch, c = k - r * nch;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + (size_t)(Y0 + r) * sp + X0 + 16 * c));
        float4 *d = reinterpret_cast<float4 *>(tile + r * kPyrStride + 16 * c);
        const unsigned wd[4] = {v.x, v.y, v.z, v.w};
        const f32x2 neg = f2_pack(__float_as_uint(-kTwo23), __float_as_uint(-kTwo23));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            unsigned a, b, c2, e;
            f2_unpack(f2_add(f2_pack(__byte_perm(wd[j], kExp23, 0x7440), __byte_perm(wd[j], kExp23, 0x7441)), neg),
                      a, b);
            f2_unpack(f2_add(f2_pack(__byte_perm(wd[j], kExp23, 0x7442), __byte_perm(wd[j], kExp23, 0x7443)), neg),
                      c2, e);
            d[j] = make_float4(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c2), __uint_as_float(e));
        }
    }
    // 2. the rows and columns of every level whose source lies in the tile:
    // lane l - 1 of the last warp takes level l (nlevels <= 16 <= 32), while
    // the other warps' tile loads are in flight
    if (tid >= kPyrThreads - 32) {
        const int lane = tid - (kPyrThreads - 32), l = 1 + lane;
        int units = 0;
        if (l < nl) {
            const int w = lw[l], h = lh[l];
            const float sx = fdiv((float)W, (float)w), sy = fdiv((float)H, (float)h);
            const int ylo = pyr_first_at_least(Y0, sy, H, h);
            const int yhi = pyr_first_at_least(Y0 + kPyrTileRows, sy, H, h);
            const int xlo = pyr_first_at_least(X0, sx, W, w);
            int xhi = pyr_first_at_least(X0 + kPyrTileCols, sx, W, w);
            if (xhi == w) xhi = (w + 3) & ~3;         // zeros up to w rounded to 4
            PyrLevelInfo &I = info[l];
            I.ylo = ylo;
            // scale_factor >= 1 makes H / h >= 1, so at most two consecutive
            // output rows share an upper source row: a tile holds at most
            // 2 x kPyrTileRows rows of a level (the bound keeps the table safe)
            I.nrows = min(yhi - ylo, kPyrRowsPerLevel);
            I.xlo = xlo;
            I.ncols = xhi - xlo;
            I.wreal = w;
            I.dp = lp[l];
            I.sx = sx;
            I.dst = const_cast<uint8_t *>(side ? F.pyrR[l] : F.pyrL[l]);
            units = 32 * ((I.ncols + 32 * kPyrCols - 1) / (32 * kPyrCols));
        }
        int end = units;                              // inclusive prefix sum over the levels
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, end, d);
            if (lane >= d) end += o;
        }
        if (l < nl) info[l].unit0 = end - units;
        if (l == nl - 1 || (nl <= 1 && lane == 0)) info[nl].unit0 = nl <= 1 ? 0 : end;   // end of the unit list
    }
    __syncthreads();
    // the image's last column and row repeated past the tile's last staged
    // ones where the tile reaches the image's edge, so that the source
    // column c0 + 1 and row y0 + 1 always hold the formula's c1 and y1
    // (both clamped to the image)
    const int cl = W - 1 - X0;                       // last column, tile-local (< kPyrTileCols if owned)
    if (cl < kPyrTileCols)
        for (int r = tid; r < nr; r += kPyrThreads) tile[r * kPyrStride + cl + 1] = tile[r * kPyrStride + cl];
    if (nr <= kPyrTileRows)                          // the tile holds the image's last row, nr - 1
        for (int c = tid; c < kPyrStride; c += kPyrThreads)
            tile[nr * kPyrStride + c] = tile[(nr - 1) * kPyrStride + (cl < kPyrTileCols ? min(c, cl) : c)];
    for (int k = tid; k < (nl - 1) * kPyrRowsPerLevel; k += kPyrThreads) {
        const int l = 1 + k / kPyrRowsPerLevel, i = k - (l - 1) * kPyrRowsPerLevel;
        if (i >= info[l].nrows) continue;
        const int y = info[l].ylo + i;
        const float ys = pyr_src(y, fdiv((float)H, (float)lh[l]), H);
        const int y0 = f2i(floorf(ys));
        PyrRow e;
        e.r0 = (unsigned)((y0 - Y0) * kPyrStride);
        e.fy = fsub(ys, (float)y0);
        e.gy = fsub(1.0f, e.fy);
        e.doff = (unsigned)(y * info[l].dp);
        tab[k] = e;
    }
    __syncthreads();
    // 3. one unit (kPyrCols output columns 32 apart) of one level per thread
    // at a time, down the level's rows in this tile
    const int units = info[nl].unit0;
    int l = 1;
    for (int u = tid; u < units; u += kPyrThreads) {
        while (u >= info[l + 1].unit0) ++l;          // units are in level order; u only grows
        const int k = u - info[l].unit0;
        const int x0 = info[l].xlo + 32 * kPyrCols * (k >> 5) + (k & 31);
        const int xend = info[l].xlo + info[l].ncols, w = info[l].wreal;
        const int n = info[l].nrows;
        uint8_t *out = info[l].dst;
        const PyrRow *T = tab + (l - 1) * kPyrRowsPerLevel;
        // columns from the width to the width rounded up to 4 get zeros
#pragma unroll
        for (int j = 0; j < kPyrCols; ++j) {
            const int x = x0 + 32 * j;
            if (x >= w && x < xend)
                for (int i = 0; i < n; ++i) out[T[i].doff + x] = 0;
        }
        // sampled columns: below the width and owned by this tile (the last
        // group of a level may run past both); an unsampled column repeats
        // the first one's arithmetic and stores nothing
        const int xs_end = min(w, xend);
        if (x0 >= xs_end) continue;
        const float sx = info[l].sx;
        bool st[kPyrCols];
        const float *P[kPyrCols];
        float fx[kPyrCols], gx[kPyrCols], hb[kPyrCols], ht[kPyrCols];
#pragma unroll
        for (int j = 0; j < kPyrCols; ++j) {
            st[j] = x0 + 32 * j < xs_end;
            const float xs = pyr_src(st[j] ? x0 + 32 * j : x0, sx, W);
            const int c0 = f2i(floorf(xs));
            fx[j] = fsub(xs, (float)c0);
            gx[j] = fsub(1.0f, fx[j]);
            // source columns c0 and c0 + 1; the next row lies kPyrStride floats further
            P[j] = tile + (c0 - X0);
            hb[j] = 0.0f;
        }
        uint8_t *o0 = out + x0;
        unsigned cr1 = 0xffffffffu;
        for (int i = 0; i < n; ++i) {
            const PyrRow e = T[i];
            if (e.r0 != cr1) {                        // else the previous bottom row is this top row
#pragma unroll
                for (int j = 0; j < kPyrCols; ++j) {
                    const float *a = P[j] + e.r0;
                    hb[j] = fadd(fmul(a[0], gx[j]), fmul(a[1], fx[j]));
                }
            }
#pragma unroll
            for (int j = 0; j < kPyrCols; ++j) {
                const float *a = P[j] + e.r0 + kPyrStride;
                ht[j] = hb[j];
                hb[j] = fadd(fmul(a[0], gx[j]), fmul(a[1], fx[j]));
            }
            cr1 = e.r0 + kPyrStride;
            uint8_t *o = o0 + e.doff;
#pragma unroll
            for (int j = 0; j < kPyrCols; ++j) {
                const float v = fadd(fmul(ht[j], e.gy), fmul(hb[j], e.fy));
                if (st[j]) o[32 * j] = (uint8_t)__float_as_uint(fadd(v, kRound23));
            }
        }
    }
}

// Dynamic shared memory of the pyramid kernel for nlevels levels.
size_t pyr_smem_bytes(int nlevels)
{
    return sizeof(float) * (kPyrTileRows + 1) * kPyrStride +
           sizeof(PyrRow) * (size_t)(nlevels > 1 ? nlevels - 1 : 1) * kPyrRowsPerLevel;
}

}  // namespace

cudaError_t pyramid_setup()
{
    return cudaFuncSetAttribute(ft_pyramid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pyr_smem_bytes(FT_MAX_LEVELS));
}

cudaError_t launch_pyramids(const BatchHeader *dev_hdr, int nframes, int nlevels, int tiles_per_image,
                            cudaStream_t stream)
{
    if (nframes <= 0) return cudaSuccess;
    const dim3 grid((unsigned)(tiles_per_image > 0 ? tiles_per_image : 1), (unsigned)(nframes * 2));
    ft_pyramid_kernel<<<grid, kPyrThreads, pyr_smem_bytes(nlevels), stream>>>(dev_hdr);
    return cudaGetLastError();
}

}  // namespace ft
