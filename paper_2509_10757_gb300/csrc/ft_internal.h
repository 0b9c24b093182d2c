// ft_internal.h -- structures shared by the library's host and device code.
//
// One persistent kernel runs every entry point.  The host writes a "batch
// table" (header, per-frame descriptors, per-kind work prefixes, zeroed
// counters) into pinned memory and copies it into the context's arena with
// one cudaMemcpyAsync; the kernel's CTAs then pull work items from a queue
// (an atomic head counter) in a fixed order: grid builds, stereo items,
// search items, resolve items.  An item waits only on items that sit before
// it in the queue, so the queue drains without deadlock whatever the number
// of resident CTAs.
#pragma once

#include <cstddef>
#include <cstdint>

#include "fasttrack.h"

#include <cuda_runtime.h>

namespace ft {

constexpr int kThreads = 256;                       // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kCells = FT_GRID_COLS * FT_GRID_ROWS; // 3072 grid cells
constexpr int kStageCap = 512;                      // right keypoints staged per stereo item
constexpr int kMaxRows = 4096;                      // image rows the row sort handles
constexpr int kWinRows = 192;                       // rows of a stereo item's staged window
constexpr int kOctBuckets = 8;                      // octaves a staged window separates
constexpr int kRefineChunk = 64;                    // matches refined per SAD round
constexpr int kFishChunk = 512;                     // right descriptors staged per chunk
constexpr int kFishTileMax = 128;                   // left keypoints per fisheye item, at most
constexpr int kFoldResolveMax = 8192;               // frames up to this size resolve in their last search item
constexpr int kCounters = 8;                        // per-frame counters (u32)
constexpr int kRowSortItems = 4;                    // row-sort work items per pinhole frame (2 per side)
constexpr int kPyrThreads = 256;                    // threads per pyramid block
constexpr int kPyrTileRows = 16;                    // source rows a pyramid block owns
constexpr int kPyrTileCols = 752;                   // source columns a pyramid block owns (a multiple of 16)
constexpr int kPyrStride = kPyrTileCols + 16;       // floats per staged row (owned columns + 16)
constexpr int kPyrRowsPerLevel = 2 * kPyrTileRows;  // output rows of one level in a tile, at most

// Tiles of a pyramid's level 0 (one pyramid block each).
__host__ __device__ inline int pyr_tiles(int W, int H)
{
    return ((H + kPyrTileRows - 1) / kPyrTileRows) * ((W + kPyrTileCols - 1) / kPyrTileCols);
}
// Byte offsets within one pyramid image are 32-bit in the pyramid kernel.
constexpr long long kPyrMaxLevelBytes = 1ll << 31;

// work item kinds, in queue order
enum Kind { K_INDEX = 0, K_STEREO = 1, K_SEARCH = 2, K_RESOLVE = 3, K_KINDS = 4 };

// per-frame counter slots
enum Ctr { C_GRID_DONE = 0, C_STEREO_DONE = 1, C_STEREO_READY = 2, C_SEARCH_DONE0 = 3,
           C_SEARCH_DONE1 = 4, C_ROWS_DONE = 5 };

// device status bits (ORed into the context's status word)
constexpr unsigned kStatusTimeout = 1u;

// debug flags of the batch header
constexpr unsigned kDebugWithholdStereoReady = 1u;   // never publish stereo-ready

struct DevParams {
    int nlevels, th_stereo, th_search, ratio_any_octave;
    float sc[FT_MAX_LEVELS], isc[FT_MAX_LEVELS], band_r[FT_MAX_LEVELS];
    float median_factor, fisheye_ratio, nn_ratio, search_th;
    float view_cos_min, view_cos_narrow, radius_narrow, radius_wide, dist_lo, dist_hi;
    float th_last;
    int kb_iters;
    float min_depth;
    int po_rounds, po_iters, po_huber;
    float po_chi2_mono, po_chi2_stereo;
    int halo;            // rows a right keypoint's band can reach beyond floor(y), any octave
    int halo_oct[FT_MAX_LEVELS];   // same for the octave window of a left keypoint of octave o
    int halo_c[FT_MAX_LEVELS];     // same for a right keypoint of octave o
};

// One camera of the search step (pinhole: the left camera only).
struct CamDev {
    int model;           // ft_camera_model
    int nk;
    float fx, fy, cx, cy, bf;
    float k[4];
    float minx, maxx, miny, maxy;
    float iw, ih;        // grid cells per pixel (computed on the device)
    float R[9], t[3], O[3];
    const float *kx, *ky;
    const int8_t *koct;
    const uint4 *kdesc;
    const uint8_t *taken;
    int8_t *level;
    float4 *proj;
    int *mp_kp, *mp_d1, *mp_d2, *kp_mp;
    int *cell_ptr;                 // [kCells + 1]
    uint16_t *cell16;              // [kCells + 1] the same starts in 16 bits (nk < 65536), 16-byte aligned
    float4 *gkp;                   // [nk] keypoints in cell order: x, y,
                                   // index | octave << 20 | taken << 28, right coordinate (or -1)
    uint4 *gdesc;                  // [2 * nk]
    int *gpos;                     // [nk] cell-order position of keypoint k (-1: outside the grid)
    unsigned long long *owner;     // [nk] (distance << 32) | map index
    uint4 *scan;                   // [2 * nm] split search: per map point its four smallest candidate keys,
                                   // then (right coordinate, radius, their octaves, how many passed)
};

struct FrameDev {
    int camera, do_stereo, do_search, wait_stereo;
    int nl, nr, nm, ncam;
    // stereo inputs
    const float *lx, *ly, *rx, *ry;
    const int8_t *loct, *roct;
    const uint4 *ldesc, *rdesc;
    const uint8_t *pyrL[FT_MAX_LEVELS], *pyrR[FT_MAX_LEVELS];
    int lw[FT_MAX_LEVELS], lh[FT_MAX_LEVELS], lp[FT_MAX_LEVELS];
    int rw[FT_MAX_LEVELS], rh[FT_MAX_LEVELS], rp[FT_MAX_LEVELS];
    int H;
    float b, bf;
    float lap_l0, lap_l1, lap_r0, lap_r1;
    // row sort of the pinhole stereo step (scratch): keypoints bucketed by row
    int *row_ptr_l, *row_ptr_r;    // [H + 1]
    float4 *ls_kp;                 // [nl] left x, y, index, octave in row order
    uint4 *ls_desc;                // [2 * nl]
    float4 *rs_kp;                 // [nr] right x, band rows lo | hi << 16, row, index | octave << 20
    uint4 *rs_desc;                // [2 * nr]
    // stereo outputs (pinhole)
    int *best_r, *dist, *sad_shift, *sad_best;
    float *u_right, *depth;
    // stereo outputs (fisheye)
    int *r_idx, *fd1, *fd2;
    float *fdepth;                 // triangulated depth per left keypoint (NULL: no triangulation)
    float4 *fxyz;                  // triangulated point (may be NULL)
    float kbl[8], kbr[8];          // fx, fy, cx, cy, k1..k4 of the left and right fisheye cameras
    // search
    const float *u_right_in;       // stereo consistency input (NULL: none)
    int build_pyr;                 // levels 1.. built from level 0 before the launch: bit 0 left, bit 1 right
    int search_mode;               // 0: local map; 1: the last frame's points
    const int8_t *last_oct;        // last mode: octave of each point's last observation
    float last_R[9], last_t[3];    // last mode: the last frame's pose
    float base;                    // stereo baseline (the motion test of the last mode)
    float R_rl[9], t_rl[3];        // fisheye rig (right camera pose is composed on the device)
    CamDev cam[2];
    const float4 *pos, *nrm;
    const uint4 *mdesc;
    const uint8_t *skip;
    // work decomposition
    int strip_rows, n_stereo_items, fisheye_tile;
    int search_tile, resolve_tile;
    int search_stage;              // 0: stage the camera's records on chip when they fit; 1: read from L2
    int rowsort;                   // row-sort index items (kRowSortItems: the first half the left
                                   // keypoints, the second half the right ones), 0 without stereo
    int fold_resolve;              // 1: the last search item of a camera writes the final tables
    int split_search;              // 1: search items scan their candidates before waiting for the stereo
                                   // step and apply the stereo consistency after it
    int n_grid_items, n_index_items, n_search_items[2], n_resolve_items[2];
    unsigned *ctr;                 // [kCounters]
    // pose optimization (next row f4): the pose kernel, launched after the
    // fused kernel, takes one block per frame with do_pose (pinhole frames)
    int do_pose;
    const int *po_mp_kp;           // [nm] matches: map point -> keypoint (cam[0])
    float *po_Rt;                  // [12] out: R row-major, t
    int8_t *po_inlier;             // [nm] out: 1 inlier, 0 outlier, -1 unmatched
    int *po_n;                     // [1] out: inliers
    float4 *po_list;               // [2 * nm] scratch: observations in map-point order
};

struct BatchHeader {
    DevParams p;
    int nframes, total_items;
    int kind_begin[K_KINDS + 1];
    unsigned debug_flags;
    const int *prefix;             // [K_KINDS][nframes + 1]
    const FrameDev *frames;
    unsigned *queue;               // [0]: next item, [1]: trace records written
    unsigned *status;              // context status word (persistent, not in the table)
    unsigned long long timeout_ns; // bound of every device-side wait
    ft_trace_record *trace;        // NULL: tracing off
    int trace_cap;
    int pad_;
};

// ---------------------------------------------------------------- f3: keypoint extraction
constexpr int kOrbTile = 32;            // detection tile: 32 x 32 pixels, 4 per thread
constexpr int kOrbHalo = 4;             // FAST circle (3) + suppression neighbours (1)
constexpr int kOrbMaxDim = 4096;        // level sizes the 12-bit key coordinates allow
constexpr int kOrbMaxSlots = 4096;      // slots per level (sorted in shared memory)
constexpr int kOrbSelectThreads = 1024;

// One pyramid level of an image being described.
struct OrbLevel {
    const uint8_t *img;                 // level image
    int w, h, pitch;
    uint8_t *smooth;                    // [h][spitch] binomial-smoothed level (scratch)
    int spitch;                         // its row pitch: w rounded up to 16 bytes
    unsigned *cand;                     // [cand_cap] suppressed corners as keys (scratch)
    int cand_cap;
    int tiles_x, tile0;                 // tiles per row, first tile of the level in the image
    int slot0, max_kp;                  // first output slot of the level and its slots
};

struct OrbImage {
    OrbLevel lv[FT_MAX_LEVELS];
    int tiles, nslots;
    float *x, *y;                       // outputs, [nslots] each
    int8_t *oct;
    int *score;
    float *cs;                          // [nslots][2]
    uint8_t *desc;                      // [nslots][32]
    int *n_level;                       // [nlevels + 1]
    unsigned *sel;                      // [nslots] selected keys in slot order (scratch)
    unsigned *cnt;                      // [nlevels] candidate counters (zeroed by the table copy)
};

struct OrbHeader {
    int nimages, nlevels, fast_th, edge, max_tiles, max_slots;
    float sc[FT_MAX_LEVELS];
    alignas(16) int8_t pattern[256 * 4];      // test i: x1, y1, x2, y2 at 4 i (16-byte aligned: vector loads)
    const OrbImage *images;
};

}  // namespace ft

// Launch helpers implemented in ft_kernels.cu (host-callable).
namespace ft {
cudaError_t launch_fused(const BatchHeader *dev_hdr, int grid, cudaStream_t stream);
// pose optimization of the frames with do_pose (one block per frame of the
// first nframes; after the fused kernel on the same stream)
cudaError_t launch_pose(const BatchHeader *dev_hdr, int nframes, cudaStream_t stream);
// levels 1.. of the pyramids of the frames that build them (before the fused
// launch); blocks_per_image blocks stride over each image's virtual blocks
cudaError_t launch_pyramids(const BatchHeader *dev_hdr, int nframes, int nlevels, int tiles_per_image,
                            cudaStream_t stream);
cudaError_t pyramid_setup();   // the pyramid kernel's shared-memory attribute (once per context)
int fused_smem_bytes();
// device set-up of the fused and pose kernels (shared-memory attributes),
// then the fused kernel's resident CTAs per SM
cudaError_t fused_occupancy(int *ctas_per_sm);
const void *fused_kernel_ptr();
// keypoint extraction of the images of an OrbHeader (ft_orb.cu): detection,
// selection and description, three launches on the stream
cudaError_t launch_orb(const OrbHeader *dev_hdr, int nimages, int nlevels, int max_tiles, int max_slots,
                       cudaStream_t stream);
// set the text ft_last_error() returns on this thread (ft_api.cu)
void set_last_error(const char *msg);
// host checks and derived tables shared by the entry points (ft_api.cu)
ft_status check_params(const ft_params &p);   // FT_EINVAL + ft_last_error() text on a bad field
DevParams make_dev_params(const ft_params &p);
int stereo_strip_rows(int want, int H, int nr, int halo);
}  // namespace ft
