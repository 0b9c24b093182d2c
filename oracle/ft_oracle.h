/*
 * ft_oracle.h -- plain, slow, single-threaded CPU oracle for the FastTrack
 * tracking hot path (stereo matching and search of local map points).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or constant generator with the CUDA library; the library
 * never includes or links it.
 *
 * What it follows (paper: "FastTrack: GPU-Accelerated Tracking for Visual
 * SLAM"):
 *   - section II-B and IV-C: stereo matching.  Pinhole: per left keypoint, the
 *     best right keypoint in a band along the epipolar line (row), then a
 *     refinement that picks the best candidate among nearby pixels.  Fisheye:
 *     brute force over the right keypoints of the overlap region.
 *   - section II-D and IV-E: search of local map points by projection.  Each
 *     map point is projected into the frame independently and matched against
 *     the keypoints near its projection.
 * The paper prints no constants, windows or tie-breaks.  Every value below is
 * a documented reading of the algorithm family; each is a parameter.
 *
 * Floating point: FP32, each operation in the order written here, compiled
 * with -ffp-contract=off so no multiply-add is fused.  Division and sqrtf are
 * IEEE correctly rounded.  Integer work (Hamming, SAD) is exact.  The pose
 * optimization (next row f4) alone runs in double precision: the library
 * computes it in FP32 and is compared with a stated tolerance.
 */
#ifndef FT_ORACLE_H
#define FT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_DESC_BYTES 32   /* 256-bit ORB descriptor */
#define ORC_MAX_LEVELS 16
#define ORC_GRID_COLS 64
#define ORC_GRID_ROWS 48
#define ORC_NO_SHIFT (-128) /* sad_shift value when the SAD was not evaluated */

typedef struct {
    int   nlevels;          /* S, pyramid levels (8) */
    float scale_factor;     /* s, level scale (1.2) */
    /* stereo (pinhole) */
    int   th_stereo;        /* accept best Hamming distance d < th_stereo (75) */
    int   sad_w;            /* SAD half window, 5 -> 11x11 patch */
    int   sad_L;            /* SAD shift range, k in [-L, L] (5) */
    float median_factor;    /* reject SAD >= median_factor * median (1.5f*1.4f) */
    /* stereo (fisheye) */
    float fisheye_ratio;    /* accept d1 < ratio * d2 (0.7) */
    /* search of local points */
    int   th_search;        /* accept best distance d1 <= th_search (100) */
    float nn_ratio;         /* reject d1 > nn_ratio * d2 (0.8) ... */
    int   ratio_any_octave; /* ... always (1) or only when both share an octave (0) */
    float search_th;        /* search radius factor th (1.0) */
    float view_cos_min;     /* reject viewing cosine < 0.5 */
    float view_cos_narrow;  /* narrow radius when viewing cosine > 0.998 */
    float radius_narrow;    /* 2.5 px */
    float radius_wide;      /* 4.0 px */
    float dist_lo;          /* distance must be >= dist_lo * dmin (0.8) */
    float dist_hi;          /* distance must be <= dist_hi * dmax (1.2) */
    /* search of the last frame's points (next row f2) */
    float th_last;          /* radius = th_last * scale[last octave] (7) */
    /* fisheye triangulation (next row f1) */
    int   kb_iters;         /* Newton iterations of the Kannala-Brandt unprojection (10) */
    float min_depth;        /* keep a triangulated point only if its depth > min_depth (1e-4 m) */
    /* pose optimization (next row f4) */
    int   po_rounds;        /* classification rounds (4) */
    int   po_iters;         /* Gauss-Newton steps per round (10) */
    float po_chi2_mono;     /* outlier above this chi2, two residuals (5.991) */
    float po_chi2_stereo;   /* outlier above this chi2, three residuals (7.815) */
    int   po_huber;         /* Huber weights with delta^2 = the threshold (1) or none (0) */
} orc_params;

typedef struct {
    float fx, fy, cx, cy;
    float b;                /* baseline (m) */
    float bf;               /* baseline times fx */
    int   width, height;    /* level-0 image size */
    float min_x, max_x, min_y, max_y;   /* image bounds for frustum and grid */
} orc_pinhole;

typedef struct {
    float fx, fy, cx, cy;
    float k[4];             /* Kannala-Brandt k1..k4 */
    int   width, height;
    float min_x, max_x, min_y, max_y;
} orc_kb8;

typedef struct {
    float R[9];             /* row-major rotation world -> camera */
    float t[3];             /* translation world -> camera */
    float O[3];             /* camera centre in world coordinates */
} orc_pose;

/* One pyramid: level pointers and sizes (uint8, row pitch in bytes). */
typedef struct {
    int nlevels;
    const uint8_t *data[ORC_MAX_LEVELS];
    int width[ORC_MAX_LEVELS], height[ORC_MAX_LEVELS], pitch[ORC_MAX_LEVELS];
} orc_pyramid;

/* Keypoints: level-0 coordinates, octave, descriptor [n][32]. */
typedef struct {
    int n;
    const float *x, *y;
    const int8_t *oct;
    const uint8_t *desc;
} orc_keypoints;

/* ---- basic pieces ---------------------------------------------------- */
int  orc_hamming(const uint8_t *a, const uint8_t *b);
void orc_scale_table(int nlevels, float s, float *sc, float *isc);
float orc_atan2_pos(float y, float x);   /* atan2 for y >= 0, x >= 0 */

/* ---- stereo, pinhole (steps a1-a5) ----------------------------------- */
int orc_row_index(int nr, const float *yr, const int8_t *octr, const float *sc,
                  int H, int *row_ptr, int *row_idx, int cap);
void orc_stereo_best(const orc_params *p, const orc_pinhole *cam,
                     const orc_keypoints *L, const orc_keypoints *R,
                     const int *row_ptr, const int *row_idx,
                     int32_t *best_r, int32_t *dist);
int orc_sad_vector(const orc_params *p, const orc_pyramid *pl, const orc_pyramid *pr,
                   int level, int ul, int vl, int ur0, int32_t *sad);
int orc_subpixel(const int32_t *sad, int L, int kbest, int ur0, float scale, float xl,
                 float bf, float disp_hi, float *u_right, float *depth, float *delta);
void orc_median_reject(int n_kp, const int32_t *sad_best, float factor, float *u_right,
                       float *depth);
void orc_stereo_pinhole(const orc_params *p, const orc_pinhole *cam,
                        const orc_keypoints *L, const orc_keypoints *R,
                        const orc_pyramid *pl, const orc_pyramid *pr,
                        int32_t *best_r, int32_t *dist, int32_t *sad_shift,
                        int32_t *sad_best, float *u_right, float *depth);

/* ---- stereo, fisheye (step a6) ---------------------------------------- */
void orc_stereo_fisheye(const orc_params *p, const orc_keypoints *L, const orc_keypoints *R,
                        float lap_l0, float lap_l1, float lap_r0, float lap_r1,
                        int32_t *r_idx, int32_t *d1, int32_t *d2);

/* ---- fisheye triangulation (next row f1) ------------------------------ */
float orc_sin_series(float t);           /* sin t by its Taylor series to t^13, |t| <= 2 */
float orc_cos_series(float t);           /* cos t by its Taylor series to t^14, |t| <= 2 */
int orc_unproject_kb8(const orc_kb8 *cam, int iters, float u, float v, float *ray);
int orc_triangulate(const float *ray_l, const float *ray_r, const float *R_rl, const float *t_rl,
                    float min_depth, float *xyz);
void orc_fisheye_triangulate(const orc_params *p, const orc_kb8 *camL, const orc_kb8 *camR,
                             const float *R_rl, const float *t_rl, const orc_keypoints *L,
                             const orc_keypoints *R, const int32_t *r_idx, float *depth, float *xyz4);

/* ---- search of local points (steps a7-a10) --------------------------- */
int orc_grid_cell(float x, float y, float min_x, float max_x, float min_y, float max_y,
                  int *cx, int *cy);
int orc_project_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                        const float *Pw, const float *nrm, float dmin, float dmax,
                        float *out4, int *level);
int orc_project_kb8(const orc_params *p, const orc_kb8 *cam, const float *R, const float *t,
                    const float *O, const float *Pw, const float *nrm, float dmin, float dmax,
                    float *out4, int *level);
void orc_search_camera(const orc_params *p, float min_x, float max_x, float min_y, float max_y,
                       const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                       int M, const uint8_t *mp_desc, const int8_t *level, const float *proj,
                       int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp);
void orc_search_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                        const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                        int M, const float *pos, const float *nrm, const uint8_t *mp_desc,
                        const uint8_t *skip, int8_t *level, float *proj,
                        int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp);
void orc_search_fisheye(const orc_params *p, const orc_kb8 *camL, const orc_kb8 *camR,
                        const float *R_rl, const float *t_rl, const orc_pose *T,
                        const float *O_right,
                        const orc_keypoints *KL, const uint8_t *takenL,
                        const orc_keypoints *KR, const uint8_t *takenR,
                        int M, const float *pos, const float *nrm, const uint8_t *mp_desc,
                        const uint8_t *skip,
                        int8_t *level_l, float *proj_l, int32_t *mp_kp_l, int32_t *mp_d1_l,
                        int32_t *mp_d2_l, int32_t *kp_mp_l,
                        int8_t *level_r, float *proj_r, int32_t *mp_kp_r, int32_t *mp_d1_r,
                        int32_t *mp_d2_r, int32_t *kp_mp_r);

/* ---- image pyramid (next row f3, its pyramid part) ------------------- */
void orc_pyramid_sizes(int W, int H, int nlevels, float s, int *w, int *h);
void orc_resample_level(const uint8_t *src, int W, int H, int pitch, uint8_t *dst, int w, int h, int dpitch);

/* ---- search of the last frame's points (next row f2) ------------------ */
int orc_motion(const orc_pose *cur, const orc_pose *last, float b);
void orc_search_last_camera(const orc_params *p, float min_x, float max_x, float min_y, float max_y,
                            const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                            int M, const uint8_t *mp_desc, const int8_t *level, const float *proj,
                            int motion, int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2,
                            int32_t *kp_mp);
void orc_search_last_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                             const orc_pose *T_last, const orc_keypoints *K, const float *u_right,
                             const uint8_t *taken, int M, const float *pos, const uint8_t *mp_desc,
                             const int8_t *last_oct, const uint8_t *skip, int8_t *level, float *proj,
                             int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp);
void orc_search_last_fisheye(const orc_params *p, const orc_kb8 *camL, const orc_kb8 *camR,
                             const float *R_rl, const float *t_rl, float b, const orc_pose *T,
                             const orc_pose *T_last, const orc_keypoints *KL, const uint8_t *takenL,
                             const orc_keypoints *KR, const uint8_t *takenR, int M, const float *pos,
                             const uint8_t *mp_desc, const int8_t *last_oct, const uint8_t *skip,
                             int8_t *level_l, float *proj_l, int32_t *mp_kp_l, int32_t *mp_d1_l,
                             int32_t *mp_d2_l, int32_t *kp_mp_l,
                             int8_t *level_r, float *proj_r, int32_t *mp_kp_r, int32_t *mp_d1_r,
                             int32_t *mp_d2_r, int32_t *kp_mp_r);

/* ---- keypoint detection and description (next row f3) ----------------- */
typedef struct {
    int fast_th;                    /* FAST threshold t (20) */
    int edge;                       /* no corner closer than edge pixels to a border (19) */
    int max_kp[ORC_MAX_LEVELS];     /* keypoint slots per level */
    const int8_t *pattern;          /* [256][4] test pairs (x1, y1, x2, y2), |coordinates| <= 13 */
} orc_orb_params;

int orc_fast_score(const uint8_t *img, int pitch, int x, int y, int t);
void orc_smooth_level(const uint8_t *src, int w, int h, int pitch, uint8_t *dst);
void orc_orientation(const uint8_t *img, int pitch, int x, int y, float *cs2);
void orc_describe(const uint8_t *smooth, int pitch, int x, int y, const float *cs2, const int8_t *pattern,
                  uint8_t *desc32);
int orc_extract_orb(const orc_params *p, const orc_pyramid *pyr, const orc_orb_params *op,
                    float *x, float *y, int8_t *oct, int32_t *score, float *cs, uint8_t *desc,
                    int32_t *n_level);

/* ---- pose optimization (next row f4), double precision ---------------- */
void orc_se3_exp(const double *d6, double *R9, double *V9);
int orc_pose_residual(const orc_pinhole *cam, const double *R9, const double *t3, const float *Pw,
                      const double *obs3, int stereo, double *e3, double *J18);
int orc_optimize_pose_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T0,
                              const orc_keypoints *K, const float *u_right, int M, const float *pos,
                              const int32_t *mp_kp, double *Rt12, int8_t *inlier, double *chi2,
                              double *min_margin, int *rounds_run);

#ifdef __cplusplus
}
#endif
#endif
