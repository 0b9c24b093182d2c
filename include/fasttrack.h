/*
 * fasttrack.h -- C ABI of libfasttrack.so: the data-parallel core of visual
 * SLAM tracking from "FastTrack: GPU-Accelerated Tracking for Visual SLAM",
 * as hand-written CUDA for GB300 (sm_103a).
 *
 * Two operations of the tracking thread run here:
 *   - stereo matching (sections II-B and IV-C): for every left keypoint, the
 *     best right keypoint.  Pinhole cameras search a band along the epipolar
 *     row, then refine the match over nearby pixels (SAD + parabola) and drop
 *     outliers against the frame's median SAD.  Fisheye cameras brute-force
 *     the right keypoints of the left/right overlap region.
 *   - search of local map points by projection (sections II-D and IV-E):
 *     every local map point is projected into the frame independently and
 *     matched to the keypoints near its projection.
 *
 * Conventions for every entry point:
 *   - Pointers inside the view structs are DEVICE pointers (unless a call
 *     says otherwise) owned by the caller; the library never frees them.
 *     Outputs are written in full (every element gets a value).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL is the legacy default stream).  FT_OK means "enqueued".
 *   - All argument checks (NULL pointers, sizes, 16-byte alignment, level
 *     sizes) run on the host before anything is enqueued; a failed check
 *     returns its code, enqueues nothing and sets ft_last_error().
 *   - Failures found on the device (a bounded wait that ran out) are ORed
 *     into the context's device status word, read with ft_sync_status().
 *     No call aborts the process and no call traps on the device.
 *   - Keypoint octaves must lie in [0, nlevels); coordinates must be finite.
 *     Inputs outside that are not detected; results for them are unspecified
 *     but every memory access stays in bounds.
 *   - A context (ft_ctx) owns its preallocated device arena, pinned staging
 *     buffers, CUDA graphs and tuning table.  Its calls reuse the same
 *     scratch, so one context serves one stream at a time; calls on another
 *     stream are ordered after the previous call by an event.
 */
#ifndef FASTTRACK_H
#define FASTTRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FT_DESC_BYTES 32        /* 256-bit ORB descriptor, rows of [n][32] uint8 */
#define FT_MAX_LEVELS 16        /* pyramid levels */
#define FT_GRID_COLS 64         /* keypoint grid of the search step */
#define FT_GRID_ROWS 48
#define FT_SAD_W 5              /* SAD half window: 11x11 patches */
#define FT_SAD_L 5              /* SAD shifts k in [-5, 5] */
#define FT_NO_SHIFT (-128)      /* sad_shift when the SAD windows left the image */
#define FT_MAX_KEYPOINTS (1 << 20)   /* per image; indices travel in 20 bits */
#define FT_MAX_MAP_POINTS (1 << 30)

typedef enum {
    FT_OK = 0,
    FT_EINVAL = 1,     /* bad argument (NULL, size, range) */
    FT_EALIGN = 2,     /* descriptor or map record not 16-byte aligned */
    FT_ENOMEM = 3,     /* the context's arena cannot hold this call */
    FT_EBUSY = 4,      /* admission refused (server) */
    FT_ECUDA = 5,      /* a CUDA runtime call failed */
    FT_ETIMEOUT = 6    /* a bounded device wait ran out (device status) */
} ft_status;

typedef enum { FT_CAMERA_PINHOLE = 0, FT_CAMERA_FISHEYE = 1 } ft_camera_model;

/* Constants the paper does not print; each default is a reading of the
 * algorithm family (fill with ft_params_default). */
typedef struct {
    int   nlevels;          /* S pyramid levels (8) */
    float scale_factor;     /* s level scale (1.2); scale[l] = scale[l-1]*s in FP32 */
    int   th_stereo;        /* stereo: accept best Hamming distance d < 75 */
    float median_factor;    /* stereo: drop SAD >= factor * median (1.5f*1.4f) */
    float fisheye_ratio;    /* fisheye: accept d1 < 0.7 * d2 */
    int   th_search;        /* search: accept d1 <= 100 */
    float nn_ratio;         /* search: reject d1 > 0.8 * d2 ... */
    int   ratio_any_octave; /* ... always (1) or only if both share an octave (0) */
    float search_th;        /* search radius factor th (1.0) */
    float view_cos_min;     /* reject viewing cosine < 0.5 */
    float view_cos_narrow;  /* narrow radius if viewing cosine > 0.998 */
    float radius_narrow;    /* 2.5 px at level 0 */
    float radius_wide;      /* 4.0 px at level 0 */
    float dist_lo;          /* in view if dist >= 0.8 * dmin ... */
    float dist_hi;          /* ... and dist <= 1.2 * dmax */
    float th_last;          /* last-frame search: radius = 7 * scale[last octave] */
    int   kb_iters;         /* fisheye triangulation: Newton steps of the
                               Kannala-Brandt unprojection (10), in [1, 64] */
    float min_depth;        /* fisheye triangulation: keep depth > 1e-4 m */
    int   po_rounds;        /* pose optimization: classification rounds (4), in [1, 16] */
    int   po_iters;         /* pose optimization: Gauss-Newton steps per round (10), in [1, 64] */
    float po_chi2_mono;     /* pose optimization: outlier above this chi2, 2 residuals (5.991) */
    float po_chi2_stereo;   /* pose optimization: outlier above this chi2, 3 residuals (7.815) */
    int   po_huber;         /* pose optimization: Huber weights (1) or plain least squares (0) */
} ft_params;

/* Keypoints of one image (level-0 pixel coordinates).  desc is [n][32]
 * uint8 and must be 16-byte aligned.  n in [0, FT_MAX_KEYPOINTS). */
typedef struct {
    int n;
    const float *x, *y;
    const int8_t *oct;
    const uint8_t *desc;
} ft_keypoints;

/* Image pyramid: level l is width[l] x height[l] uint8 with row pitch[l]
 * bytes (pitch >= width); the buffer of a level spans height x pitch bytes
 * (rows are read in aligned 4- and 16-byte words up to the pitch).  Every
 * level pointer must be 16-byte aligned and every pitch a multiple of 16
 * (patch rows are copied in 16-byte chunks; FT_EALIGN otherwise). */
typedef struct {
    int nlevels;
    const uint8_t *data[FT_MAX_LEVELS];
    int width[FT_MAX_LEVELS], height[FT_MAX_LEVELS], pitch[FT_MAX_LEVELS];
} ft_pyramid;

/* Rectified pinhole stereo camera.  bf = b * fx.  [min_x, max_x] x
 * [min_y, max_y] bounds the image for the frustum test and the grid. */
typedef struct {
    float fx, fy, cx, cy, b, bf;
    int width, height;
    float min_x, max_x, min_y, max_y;
} ft_pinhole;

/* Kannala-Brandt fisheye camera (equidistant with k1..k4). */
typedef struct {
    float fx, fy, cx, cy, k[4];
    int width, height;
    float min_x, max_x, min_y, max_y;
} ft_kb8;

/* Fisheye stereo rig: right <- left transform (row-major R_rl, t_rl) and the
 * overlap x-ranges of the two images. */
typedef struct {
    ft_kb8 left, right;
    float R_rl[9], t_rl[3];
    float b;
    float lap_l0, lap_l1, lap_r0, lap_r1;
} ft_fisheye_rig;

/* Camera pose: world -> camera rotation (row-major) and translation, and the
 * camera centre in world coordinates. */
typedef struct {
    float R[9], t[3], O[3];
} ft_pose;

/* Local map points, structure of arrays (the paper splits the map-point
 * record into fine-grained parts, section IV-E).  pos is [n][4] floats
 * (x, y, z, dmin), nrm is [n][4] (mean viewing direction nx, ny, nz, dmax),
 * desc [n][32]; pos, nrm and desc 16-byte aligned.  skip[m] != 0 leaves a
 * point out of the search (may be NULL). */
typedef struct {
    int n;
    const float *pos;
    const float *nrm;
    const uint8_t *desc;
    const uint8_t *skip;
} ft_map_view;

/* One stereo frame (pinhole: both pyramids are needed for the refinement). */
typedef struct {
    ft_keypoints left, right;
    ft_pyramid pyr_left, pyr_right;
} ft_stereo_frame;

/* Pinhole stereo output, one entry per left keypoint:
 *   best_r     right index of the best Hamming match if d < th_stereo, else -1
 *   dist       smallest Hamming distance over the candidates (-1: none)
 *   sad_shift  best SAD shift in [-5, 5] (FT_NO_SHIFT: windows left the image
 *              or no match)
 *   sad_best   SAD at the best shift for matches that passed the parabola and
 *              disparity checks (before median rejection), else -1
 *   u_right    right x coordinate (level 0) of the final match, else -1
 *   depth      bf / disparity of the final match, else -1 */
typedef struct {
    int32_t *best_r, *dist, *sad_shift, *sad_best;
    float *u_right, *depth;
} ft_stereo_out;

/* Fisheye stereo output per left keypoint: r_idx (accepted right index or
 * -1), d1 / d2 (smallest and second smallest Hamming distance over the
 * overlap candidates; d2 = 256 with a single candidate; both -1 outside the
 * overlap or with no candidate).
 * Triangulation of the accepted matches (the paper matches stereo keypoints
 * to obtain depth, section II-B; the method is a reading): each pixel is
 * unprojected through its Kannala-Brandt model (kb_iters Newton steps on
 * theta, kept if the residual is at most 2e-6 rad where the model still
 * rises), the right ray is taken to left-camera coordinates, and the point is
 * the midpoint of the two rays' common perpendicular, kept if the rays are
 * not parallel (|l x r|^2 > 1e-10 |l|^2 |r|^2), lie in front of both
 * centres and its left depth exceeds min_depth.
 *   depth [n] left-camera z of the point, else -1; may be NULL (no
 *         triangulation)
 *   xyz   [n][4] (x, y, z, 1) in left-camera coordinates, else zeros; may be
 *         NULL; 16-byte aligned */
typedef struct {
    int32_t *r_idx, *d1, *d2;
    float *depth, *xyz;
} ft_fisheye_out;

/* Search output for one camera:
 *   level  [M] predicted level, -1 if the point is not in view (or skipped)
 *   proj   [M][4] (u, v, u_right, viewing cosine), zeros when not in view
 *          (u_right is -1 for fisheye cameras); may be NULL
 *   mp_kp  [M] matched keypoint index after conflict resolution, else -1
 *   mp_d1, mp_d2 [M] best and second-best distance (-1 / 256 as above)
 *   kp_mp  [N] map point that owns keypoint k, else -1 */
typedef struct {
    int8_t *level;
    float *proj;
    int32_t *mp_kp, *mp_d1, *mp_d2, *kp_mp;
} ft_search_cam_out;

typedef struct {
    ft_search_cam_out left;
    ft_search_cam_out right;   /* fisheye frames only */
} ft_search_out;

/* Pose optimization output of one pinhole frame (next row f4):
 *   Rt        [12] refined pose: R (row-major, world -> camera) then t
 *   inlier    [M] 1 inlier, 0 outlier after the last round, -1 unmatched
 *             map point (M = the map's points)
 *   n_inliers [1] number of inliers
 * All three are device pointers. */
typedef struct {
    float *Rt;
    int8_t *inlier;
    int32_t *n_inliers;
} ft_pose_out;

/* A frame as seen by the search step.  Pinhole: left keypoints only, with
 * u_right from stereo matching (NULL: no stereo consistency check).
 * Fisheye: left and right keypoints, each camera with its own grid; O_right
 * is the right camera centre in world coordinates. */
typedef struct {
    int camera;                 /* ft_camera_model */
    ft_pinhole pinhole;
    ft_fisheye_rig fisheye;
    ft_keypoints left, right;
    const float *u_right;
    const uint8_t *taken_left;  /* keypoints already matched (may be NULL) */
    const uint8_t *taken_right;
    float O_right[3];
} ft_frame_view;

/* The last frame's points for the search of the last frame (next row f2;
 * the paper's initial pose estimation runs the same search by projection on
 * the previous frame's points, sections II-C and IV-E):
 *   pos  [n][4] world x, y, z and an unused float, 16-byte aligned
 *   desc [n][32], 16-byte aligned
 *   oct  [n] octave of the keypoint that observed the point in the last
 *        frame (points with an octave outside [0, nlevels) are not searched)
 *   skip [n] nonzero leaves a point out (may be NULL)
 *   pose the last frame's pose (world -> camera); with the current pose it
 *        gives the camera's motion along its viewing axis */
typedef struct {
    int n;
    const float *pos;
    const uint8_t *desc;
    const int8_t *oct;
    const uint8_t *skip;
    ft_pose pose;
} ft_last_frame_view;

/* One frame of a batch: stereo matching then search of local points (or,
 * with last non-NULL, of the last frame's points; map is then ignored). */
typedef struct {
    int camera;                 /* ft_camera_model */
    ft_pinhole pinhole;
    ft_fisheye_rig fisheye;
    ft_keypoints left, right;
    ft_pyramid pyr_left, pyr_right;     /* pinhole only */
    const uint8_t *taken_left, *taken_right;
    ft_pose pose;
    float O_right[3];                   /* fisheye only */
    ft_map_view map;
    ft_stereo_out stereo;               /* pinhole */
    ft_fisheye_out fisheye_out;         /* fisheye */
    ft_search_out search;
    const ft_last_frame_view *last;     /* HOST struct; NULL: search the local map */
    int build_pyramids;                 /* pinhole: nonzero = levels 1.. of pyr_left and pyr_right
                                           are built on the device from level 0 before the stereo
                                           step reads them (see ft_build_pyramid) */
    const ft_pose_out *pose_out;        /* HOST struct; pinhole frames: non-NULL = optimize the pose
                                           over the search's matches after the search (see
                                           ft_optimize_pose); NULL: no pose optimization */
} ft_frame_job;

/* A ragged batch.  frames points to HOST memory (n entries).  If
 * stage_in_bytes > 0 the library first copies stage_in_bytes from the
 * pinned host buffer stage_in_host to the device buffer stage_in_dev on the
 * stream (the frame pointers then refer into stage_in_dev); likewise it
 * copies stage_out_bytes from stage_out_dev to the pinned host buffer
 * stage_out_host after the work.  This is how a caller runs the whole path
 * from host memory through one call. */
typedef struct {
    int n;
    const ft_frame_job *frames;
    const void *stage_in_host;
    void *stage_in_dev;
    size_t stage_in_bytes;
    const void *stage_out_dev;
    void *stage_out_host;
    size_t stage_out_bytes;
} ft_batch;

typedef struct {
    int device;             /* CUDA device ordinal */
    size_t arena_bytes;     /* preallocated scratch (0: 64 MiB) */
    int max_frames;         /* largest batch (0: 256) */
    int use_graphs;         /* replay ft_track_batch through CUDA graphs */
} ft_ctx_desc;

typedef struct ft_ctx ft_ctx;

/* Launch shape of the fused kernel (chosen per batch-shape bucket by the
 * autotuner, or set by hand). */
typedef struct {
    int strip_rows;         /* image rows per pinhole stereo work item */
    int search_tile;        /* map points per search work item (multiple of 256) */
    int fisheye_tile;       /* left keypoints per fisheye work item (64, or 128 for any larger value) */
    int resolve_tile;       /* entries per conflict-resolution item */
    int ctas_per_sm;        /* persistent CTAs per SM (0: occupancy limit) */
    int search_stage;       /* search candidates: 0 = a camera's keypoint records and descriptors
                               staged in shared memory when they fit (up to 1536 keypoints), else
                               read from L2; 1 = always read from L2 */
    int split_search;       /* pinhole frames whose stereo runs in the same call: 1 = a search item
                               scans its candidates (every test but the stereo consistency) before
                               it waits for the stereo step and applies the consistency after it,
                               -1 = it waits for the stereo step first (less work: best for large
                               batches), 0 = automatic (1 for batches of at most 32 frames); results
                               are the same */
} ft_tuning;

/* Fill p with the default readings. */
void ft_params_default(ft_params *p);

/* Thread-local text of the last error of this thread ("" if none). */
const char *ft_last_error(void);

/* Create a context on desc->device: allocates the device arena once (the
 * paper preallocates all device memory at start-up, section IV-A), pinned
 * staging buffers and events.  Returns FT_ECUDA / FT_ENOMEM on failure. */
ft_status ft_create(ft_ctx **out, const ft_ctx_desc *desc);

/* Wait for the context's work, then free everything it owns. */
void ft_destroy(ft_ctx *ctx);

/* Synchronize the context's last stream, return the device status word
 * (0 or FT_ETIMEOUT) in *status and clear it. */
ft_status ft_sync_status(ft_ctx *ctx, int32_t *status);

/* Pinhole stereo matching of one frame (sections II-B, IV-C): row-band
 * Hamming search, SAD refinement over +-5 px at the keypoint's level,
 * parabola sub-pixel disparity, depth, median-based rejection.
 * params NULL = defaults.  Outputs: ft_stereo_out, each [left.n]. */
ft_status ft_stereo_match_pinhole(ft_ctx *ctx, void *stream, const ft_params *params,
                                  const ft_pinhole *cam, const ft_stereo_frame *frame,
                                  ft_stereo_out *out);

/* Fisheye stereo matching of one frame (sections II-B, IV-C): brute force
 * over the right keypoints inside [lap_r0, lap_r1] for every left keypoint
 * inside [lap_l0, lap_l1], best/second best and ratio test.  Outputs: each
 * [left->n]. */
ft_status ft_stereo_match_fisheye(ft_ctx *ctx, void *stream, const ft_params *params,
                                  const ft_fisheye_rig *rig, const ft_keypoints *left,
                                  const ft_keypoints *right, ft_fisheye_out *out);

/* Search of local map points by projection for one frame (sections II-D,
 * IV-E): frustum test, FP32 projection, predicted level, 64x48 grid-window
 * candidates, best/second-best Hamming with ratio test, and conflict
 * resolution (a keypoint keeps the smallest (distance, map index)). */
ft_status ft_search_local_points(ft_ctx *ctx, void *stream, const ft_params *params,
                                 const ft_frame_view *frame, const ft_pose *Tcw,
                                 const ft_map_view *map, ft_search_out *out);

/* Search of the last frame's points for one frame (next row f2): the
 * search by projection of the paper's initial pose estimation (sections
 * II-C, IV-E), adapted as the algorithm family does it (a reading): a point
 * is in view if it lies in front of the camera and projects inside the image
 * (no distance or viewing-angle test); its search radius is th_last *
 * scale[oct]; the candidate octaves are >= oct if the camera moved forward
 * by more than the stereo baseline along its viewing axis since the last
 * frame, <= oct if it moved backward, oct-1..oct+1 otherwise; the best
 * distance is accepted if <= th_search, without a ratio test; the grid
 * window, taken flags, stereo consistency (pinhole u_right) and conflict
 * resolution are those of the local-map search.  Outputs as
 * ft_search_local_points, with level = the point's octave and proj[3] = 0. */
ft_status ft_search_last_frame(ft_ctx *ctx, void *stream, const ft_params *params,
                               const ft_frame_view *frame, const ft_pose *Tcw,
                               const ft_last_frame_view *last, ft_search_out *out);

/* Pose optimization of one pinhole frame (next row f4): the refinement of
 * the camera pose with all the map points the search found in the frame
 * (section II-D; FastTrack switches it off, section IV-F).  The method is a
 * reading of the algorithm family's motion-only optimization:
 *   - observations: map point m with match k = mp_kp[m] (0 <= k < left.n) is
 *     observed at (left.x[k], left.y[k]) and, if frame->u_right is not NULL
 *     and u_right[k] >= 0, also at u_right[k] (a stereo observation, three
 *     residuals; else two).  Weight 1 / scale[left.oct[k]]^2.
 *   - po_rounds rounds, each run only while at least 3 observations are
 *     inliers (all are at the start): po_iters Gauss-Newton steps over the
 *     inliers in front of the camera with Huber weights (po_huber; delta^2 =
 *     po_chi2_mono or po_chi2_stereo), the update exp(d) multiplied on the
 *     left of the pose; then every observation is classified again: outlier
 *     if behind the camera or chi2 above its threshold.  A step whose normal
 *     matrix is not positive definite ends the optimization after that
 *     round's classification.
 * FP32 on the device, one work item per frame.  Inputs: frame->pinhole,
 * frame->left, frame->u_right (may be NULL), Tcw (the starting pose),
 * map->pos ([n][4], 16-byte aligned; the rest of the map is not read) and
 * mp_kp ([map->n] device int32, the search's matches).  Outputs: out. */
ft_status ft_optimize_pose(ft_ctx *ctx, void *stream, const ft_params *params,
                           const ft_frame_view *frame, const ft_pose *Tcw, const ft_map_view *map,
                           const int32_t *mp_kp, const ft_pose_out *out);

/* Keypoint extraction parameters (next row f3). */
typedef struct {
    int fast_th;                    /* FAST threshold t, in [1, 254] (20) */
    int edge;                       /* corners at least edge pixels from every border, >= 19 (19) */
    int max_kp[FT_MAX_LEVELS];      /* slots per level, each in [0, 4096] */
    const int8_t *pattern;          /* HOST [256][4] test pairs (x1, y1, x2, y2), every coordinate
                                       in [-13, 13]; copied by the call */
} ft_orb_params;

/* Keypoint extraction output of one image: n = sum of max_kp slots, level
 * l's keypoints in slots [sum of max_kp[< l], + max_kp[l]) in the order
 * (score descending, y, x), then padding.  DEVICE pointers:
 *   x, y     [n] level-0 coordinates (level pixel times scale[l], FP32);
 *            padding: -1e9 (no search or stereo step ever matches it)
 *   oct      [n] level (padding: 0)
 *   score    [n] FAST score (padding: -1)
 *   cs       [n][2] cosine and sine of the orientation (padding: 1, 0)
 *   desc     [n][32] descriptor, 16-byte aligned (padding: zeros)
 *   n_level  [nlevels + 1] keypoints found per level, then their total
 * x, y, oct and desc have the layout of ft_keypoints: the output feeds
 * stereo matching and the search directly, with n slots. */
typedef struct {
    float *x, *y;
    int8_t *oct;
    int32_t *score;
    float *cs;
    uint8_t *desc;
    int32_t *n_level;
} ft_orb_out;

/* Keypoint detection and description on the pyramid levels of n images
 * (next row f3): the paper's ORB extraction finds keypoints on every level,
 * describes each one and filters them (section II-A); FastTrack reuses an
 * existing GPU extractor and gives none of its steps (section IV-B).  The
 * reading follows the published methods (FAST, ORB):
 *   - FAST-9 on the level image: 9 contiguous pixels of the 16 on the
 *     radius-3 circle all brighter than I + t or all darker than I - t;
 *     only pixels at least edge pixels from every border;
 *   - score: the largest t at which the pixel is still a corner;
 *   - non-maximum suppression: a corner is dropped if a neighbour (8) is a
 *     corner with a higher score, or the same score and an earlier raster
 *     position;
 *   - filtering: per level the first max_kp[l] corners by (score
 *     descending, y, x);
 *   - orientation: m10 = sum u I, m01 = sum v I over u^2 + v^2 <= 225;
 *     |m| = sqrt(m10^2 + m01^2) in double rounded to float, cos = m10/|m|,
 *     sin = m01/|m| in FP32 ((1, 0) if both are 0);
 *   - descriptor: the level smoothed by the 5x5 binomial filter (1 4 6 4 1
 *     each way, /256 rounded half up, border replicated); test i rotates
 *     both pattern points by the orientation (u = round(c x - s y),
 *     v = round(s x + c y), FP32, each product rounded) and sets bit i % 8
 *     of byte i / 8 if S(p1) < S(p2).
 * pyr[i] are the images' pyramids (params->nlevels levels, each at most
 * 4096 x 4096; the pyramid's own sizes, device data); out[i] their outputs.
 * Uses scratch in the context's arena (about 2 bytes per level pixel).
 * Three kernel launches, asynchronous on the stream. */
ft_status ft_extract_orb(ft_ctx *ctx, void *stream, const ft_params *params, int n, const ft_pyramid *pyr,
                         const ft_orb_params *orb, const ft_orb_out *out);

/* Sizes of the pyramid levels of a width x height level 0 (next row f3, its
 * pyramid part): level l is round(width / scale[l]) x round(height /
 * scale[l]) with scale[l] the FP32 product of scale_factor (params NULL =
 * defaults).  Host function; w and h receive params->nlevels values. */
ft_status ft_pyramid_sizes(int width, int height, const ft_params *params, int *w, int *h);

/* Measure the current device's 32-bit popcount rate (popcounts per second):
 * a kernel of eight independent popcount chains per thread on every SM,
 * timed with events on the stream (best of three runs after one warm-up).
 * The denominator of the popcount roofline of the Hamming searches; not part
 * of the paper's method.  Allocates and frees 4 KB of device memory. */
ft_status ft_measure_popcount(void *stream, double *popc_per_s);

/* Memory diagnostic (not part of the paper's method): one 4-byte read every
 * stride_bytes (a multiple of 4, at least 256) over a 1 GiB buffer, plus a
 * second read second_bytes (a multiple of 4, 0: none, less than stride_bytes)
 * after each; one launch on the stream, waited for.  Read under a profiler's
 * DRAM counters it shows how many bytes an isolated read moves from DRAM:
 * the granularity that scattered reads, such as the refinement's patch rows,
 * pay.  *accesses receives the number of first reads.  Allocates and frees
 * 1 GiB of device memory. */
ft_status ft_scattered_reads(void *stream, int stride_bytes, int second_bytes, int *accesses);

/* Build levels 1..nlevels-1 of a pyramid from its level 0 on the device (the
 * paper runs ORB extraction, which produces the pyramid, on the GPU so that
 * the pyramid never crosses the bus; section IV-B).  Level l samples level 0
 * bilinearly at xs = (x + 0.5) * (W / w) - 0.5 (and ys likewise), clamped to
 * the image, in FP32 (this order: top = I00 (1-fx) + I01 fx, bottom likewise,
 * value = top (1-fy) + bottom fy), rounded half to even.  The caller owns
 * every level (sizes from ft_pyramid_sizes; 16-byte aligned, pitches
 * multiples of 16); levels 1.. are written, each row up to its width rounded
 * up to 4 (bytes past the width are zero).  Asynchronous on the stream. */
ft_status ft_build_pyramid(ft_ctx *ctx, void *stream, const ft_params *params, const ft_pyramid *pyr);

/* ft_build_pyramid for n images in one launch (at most 2 x max_frames
 * images); the images may differ in size.  Asynchronous on the stream. */
ft_status ft_build_pyramids(ft_ctx *ctx, void *stream, const ft_params *params, int n, const ft_pyramid *pyr);

/* Stereo matching followed by the search, for a ragged batch of frames, in
 * one persistent fused launch (CUDA-graph replayed per batch-shape bucket if
 * the context was created with use_graphs).  Each frame's results equal
 * those of the per-frame calls. */
ft_status ft_track_batch(ft_ctx *ctx, void *stream, const ft_params *params, const ft_batch *batch);

/* Time candidate launch shapes on this batch (iters runs each) and keep the
 * fastest for the batch's bucket; *best receives it (may be NULL).  The
 * candidates: strip rows 16/32/64, search tile 256/512/1024, fisheye tile
 * 64/128, every count of CTAs per SM up to the resident maximum, and both
 * search staging modes. */
ft_status ft_autotune(ft_ctx *ctx, void *stream, const ft_params *params, const ft_batch *batch,
                      int iters, ft_tuning *best);

/* Time candidate launch shapes for a stream of batches and keep the fastest
 * in every context for the batches' bucket.  A candidate runs as a sequence
 * of launches taken by the n contexts in turn, context i on streams[i] with
 * batches[i] (each context with its own arena and each batch with its own
 * buffers, so later launches start while earlier ones' last frames finish);
 * its score is the sequence's time divided by its launches (4 * iters * n of
 * them, then 16 * iters * n three times for the four best).  Shapes that
 * make a single launch short can lose here: longer work items waste less
 * when another launch fills the tail, and fewer CTAs per SM leave room for
 * the next launch.  2 <= n <= 16 distinct contexts on one device; every batch
 * must fall in the same bucket (FT_EINVAL otherwise); *best receives the
 * winner (may be NULL). */
ft_status ft_autotune_stream(ft_ctx *const *ctxs, void *const *streams, int n, const ft_params *params,
                             const ft_batch *const *batches, int iters, ft_tuning *best);

/* Set / get the launch shape used for a batch's bucket. */
ft_status ft_set_tuning(ft_ctx *ctx, const ft_batch *batch, const ft_tuning *t);
ft_status ft_get_tuning(ft_ctx *ctx, const ft_batch *batch, ft_tuning *t);

/* Persist / load the tuning table (text file, one bucket per line). */
ft_status ft_save_tuning(ft_ctx *ctx, const char *path);
ft_status ft_load_tuning(ft_ctx *ctx, const char *path);

/* Test hook for the bounded device waits: flags bit 0 makes the stereo step
 * withhold its "stereo done" signal, so the search step's wait runs out after
 * timeout_ns (0: the default of 2 s) and the call reports FT_ETIMEOUT through
 * ft_sync_status.  Use flags = 0 for normal operation. */
ft_status ft_set_debug(ft_ctx *ctx, unsigned flags, uint64_t timeout_ns);

/* Device-side trace of the fused kernel's work items (the tracing
 * subsystem): one record per item of the last call.  kind: 0 grid build,
 * 1 stereo, 2 search, 3 conflict resolution.  Times are the GPU global
 * timer in ns; wait_ns is the part of [t_start, t_end] spent in bounded
 * waits on other items. */
typedef struct {
    int32_t item, kind, frame, sm;
    uint64_t t_start, t_end, wait_ns;
    uint64_t mark[4];   /* phase ends inside the item (0: not reached); pinhole
                           stereo: staging done, Hamming phase done, SAD
                           rounds done, median done (last strip only) */
} ft_trace_record;

/* Enable tracing with room for `capacity` records per call (allocated once
 * here; 0 disables and frees it). */
ft_status ft_set_trace(ft_ctx *ctx, int capacity);

/* Synchronize, then copy up to max records of the last call to out;
 * *n receives the number of records the call produced (may exceed max). */
ft_status ft_read_trace(ft_ctx *ctx, ft_trace_record *out, int max, int *n);

/* ----------------------------------------------------------------------
 * Served request loop: continuous batching of tracking requests from many
 * independent camera streams on one GPU (an addition of this library; the
 * paper tracks one camera).
 *
 * Camera streams are admitted against an HBM budget: the server allocates a
 * device pool of hbm_budget bytes once and gives every admitted stream a
 * block for its resident state (both pyramids, the local map, the per-frame
 * keypoint block and the result block); a stream that does not fit is
 * refused with FT_EBUSY until others close.  Requests (one frame: keypoints,
 * descriptors, taken flags, pose and optionally the frame's level-0 images,
 * all in host memory) are copied into the stream's pinned staging at
 * submit.  A scheduler thread fills free
 * slots -- n_slots contexts, each with its own arena and CUDA stream -- with
 * batches of up to max_batch pending requests in arrival order, at most one
 * per stream and none of a stream whose previous request is still running;
 * one launch of ft_track_batch serves a batch.  Requests arriving while
 * batches run go to the next free slot, so work overlaps on the device.
 * Results are copied back to pinned host memory and returned by
 * ft_server_poll with submit / start / completion times (host clock, us).
 * With dry_run the server touches no GPU: batches "complete" after
 * dry_run_latency_us, for testing the scheduling and admission logic.
 * ---------------------------------------------------------------------- */
typedef struct ft_server ft_server;

typedef struct {
    int device;
    size_t hbm_budget;          /* device pool for resident stream state */
    int n_slots;                /* batches in flight at once (>= 1) */
    int max_batch;              /* frames per batch (>= 1) */
    size_t slot_arena_bytes;    /* scratch arena of each slot's context */
    int dry_run;                /* 1: no GPU, fake completions */
    double dry_run_latency_us;  /* fake batch duration */
    int queue_depth;            /* requests a stream may have waiting (staged at submit), 1-8
                                   (0: 2); one more is refused with FT_EBUSY */
} ft_server_desc;

/* A camera stream: its model, pyramid level sizes (pinhole; level pitch =
 * width) and capacities. */
typedef struct {
    int camera;
    ft_pinhole pinhole;
    ft_fisheye_rig fisheye;
    int nlevels;
    int level_width[FT_MAX_LEVELS], level_height[FT_MAX_LEVELS];
    int max_left, max_right, max_map;
} ft_stream_desc;

/* One frame of a stream (all pointers in host memory; taken may be NULL).
 * image_left / image_right (pinhole streams; both or neither): this frame's
 * level-0 images, level_width[0] x level_height[0] bytes with row pitch
 * image_pitch (>= the width).  They are copied at submit into the stream's
 * pinned staging; at launch they replace the stream's resident level 0 and
 * levels 1.. are rebuilt on the device from it in the same batch (as
 * ft_build_pyramid), so the stream's level sizes must be those of
 * ft_pyramid_sizes for level 0 under the server's parameters (FT_EINVAL
 * otherwise).  NULL: the frame uses the resident pyramids as they are (set
 * by ft_server_set_pyramids or by an earlier frame's images). */
typedef struct {
    int stream_id;
    uint64_t tag;
    ft_keypoints left, right;
    const uint8_t *taken_left, *taken_right;
    ft_pose pose;
    float O_right[3];
    const uint8_t *image_left, *image_right;
    int image_pitch;
} ft_request;

/* Host copies of one request's results (valid until the stream's second
 * next request completes). */
typedef struct {
    int n_left, n_right, n_map;
    ft_stereo_out stereo;       /* pinhole */
    ft_fisheye_out fisheye;     /* fisheye */
    ft_search_out search;
} ft_results;

typedef struct {
    uint64_t tag;
    int stream_id;
    int32_t status;
    double t_submit_us, t_start_us, t_done_us;
    ft_results results;
} ft_completion;

typedef struct {
    uint64_t submitted, completed, batches, frames_launched, streams_open, pending;
    size_t pool_used, pool_capacity;
    int32_t last_error;         /* status of the last failed launch (0: none) */
} ft_server_stats;

void ft_server_desc_default(ft_server_desc *d);
/* params NULL = defaults (the parameters every batch uses). */
ft_status ft_server_create(ft_server **out, const ft_server_desc *desc, const ft_params *params);
/* Stops the scheduler, waits for work in flight, frees everything. */
void ft_server_destroy(ft_server *s);
/* Admit a stream (FT_EBUSY: the HBM budget cannot hold it now). */
ft_status ft_server_open_stream(ft_server *s, const ft_stream_desc *d, int *stream_id);
/* Release a stream's block (FT_EBUSY while it has requests queued or running). */
ft_status ft_server_close_stream(ft_server *s, int stream_id);
/* Upload a stream's resident pyramids / local map from host memory (synchronous). */
ft_status ft_server_set_pyramids(ft_server *s, int stream_id, const ft_pyramid *left, const ft_pyramid *right);
ft_status ft_server_set_map(ft_server *s, int stream_id, const ft_map_view *map);
/* Queue one frame (FT_EBUSY: the stream already has two frames waiting). */
ft_status ft_server_submit(ft_server *s, const ft_request *req);
/* Move up to max completions to out, waiting up to timeout_us for the first;
 * returns how many. */
int ft_server_poll(ft_server *s, ft_completion *out, int max, int timeout_us);
ft_status ft_server_get_stats(ft_server *s, ft_server_stats *stats);

/* Pinhole stereo matching of one frame, like ft_stereo_match_pinhole, for
 * callers that must not allocate memory.  The paper has no counterpart: it is
 * an addition of this library.
 *
 * Who needs it: code that may not allocate device memory once it runs -- a
 * tracking loop with a hard per-frame deadline (cudaMalloc can block and
 * synchronize the device), a deployment that reserves all device memory at
 * start-up, or a host framework whose memory manager forbids allocations
 * behind its back.  Such callers cannot create an ft_ctx (ft_create
 * allocates its arena), so this call needs no context: its scratch (work
 * table, counters, row sort) lives in a fixed 2 MiB device array that is part
 * of the library, held on every device that loads the library until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The caller passes inputs and outputs as for
 * ft_stereo_match_pinhole, on the current device.
 *
 * Limits: at most 16384 left and 16384 right keypoints and 4096 image rows
 * per call; larger frames are rejected with FT_EINVAL and a message in
 * ft_last_error().  params are checked as by every other entry point
 * (FT_EINVAL before any device work).  The call copies its work table from
 * a buffer on the host stack, so a stream that is being captured is refused
 * with FT_EINVAL.
 *
 * The first call on a device looks up the array's device address and the
 * kernel's launch shape for that device (with the device current); make that
 * first call before starting any stream capture.  All calls share the one
 * array and each call overwrites what the previous one left there, so calls
 * whose GPU work overlaps (two streams at once) race and give wrong results:
 * keep them on one stream or order them.  If device_status is not NULL it
 * receives (on the stream) 0, or a nonzero value when a bounded device wait
 * ran out. */
ft_status ft_stereo_match_pinhole_noalloc(void *stream, const ft_params *params,
                                          const ft_pinhole *cam, const ft_stereo_frame *frame,
                                          ft_stereo_out *out, int32_t *device_status);

/* Kernel launches issued by this context so far (all entry points). */
uint64_t ft_launch_count(ft_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
