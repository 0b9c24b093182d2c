/*
 * ft_oracle.c -- plain CPU oracle for the FastTrack tracking hot path.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Shares no code
 * with the CUDA library.  Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared.
 *
 * Steps, in the paper's order:
 *   stereo matching, pinhole (sections II-B, IV-C)
 *     a1  row-band index of right keypoints
 *     a2  best Hamming match per left keypoint inside its band
 *     a3  SAD refinement over +-L pixel shifts at the keypoint's level
 *     a4  parabola sub-pixel fit, disparity and depth
 *     a5  median-based outlier rejection over the frame's matches
 *   stereo matching, fisheye (sections II-B, IV-C)
 *     a6  brute force over the right overlap keypoints, best/second best + ratio
 *   search of local points by projection (sections II-D, IV-E)
 *     a7  64x48 keypoint grid
 *     a8  frustum test, FP32 projection, predicted scale level
 *     a9  cell-window gather, best/second-best Hamming, ratio test
 *     a10 a keypoint claimed by several map points keeps the smallest
 *         (distance, map point index); map points are searched independently
 *         as the paper states (section IV-E).
 *   and the next steps around them:
 *     f1  triangulation of the fisheye matches (section II-B)
 *     f2  search by projection of the last frame's points (sections II-C, IV-E)
 *     f3  the image pyramid built from level 0 (section IV-B)
 * The paper prints none of the constants; each is a parameter (orc_params).
 */
#include "ft_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Hamming distance: XOR byte by byte, count bits with a 256-entry table.   */
/* The table is built by counting the bits of each byte value one by one.   */
/* ------------------------------------------------------------------------ */
static int bit_count_table[256];
static int bit_count_ready = 0;

static void build_bit_count_table(void)
{
    for (int v = 0; v < 256; ++v) {
        int c = 0;
        for (int b = 0; b < 8; ++b) c += (v >> b) & 1;
        bit_count_table[v] = c;
    }
    bit_count_ready = 1;
}

int orc_hamming(const uint8_t *a, const uint8_t *b)
{
    if (!bit_count_ready) build_bit_count_table();
    int d = 0;
    for (int i = 0; i < ORC_DESC_BYTES; ++i) d += bit_count_table[a[i] ^ b[i]];
    return d;
}

/* Scale of level l: s^l accumulated in FP32, and its reciprocal. */
void orc_scale_table(int nlevels, float s, float *sc, float *isc)
{
    sc[0] = 1.0f;
    for (int l = 1; l < nlevels; ++l) sc[l] = sc[l - 1] * s;
    for (int l = 0; l < nlevels; ++l) isc[l] = 1.0f / sc[l];
}

/* ------------------------------------------------------------------------ */
/* atan2 on the first quadrant, written from the mathematics:               */
/*   atan2(y, x) = atan(y/x) if y <= x, else pi/2 - atan(x/y);             */
/*   for t in [0, 1]: atan(t) = pi/4 + atan((t-1)/(t+1)) if t > tan(pi/8); */
/*   for |a| <= tan(pi/8): the Taylor series sum_k (-1)^k a^(2k+1)/(2k+1), */
/*   truncated after k = 8 (remainder below 3e-9 for |a| <= 0.4143).       */
/* Coefficients are 1/(2k+1) divided out in FP32; Horner in a^2.           */
/* ------------------------------------------------------------------------ */
#define ORC_ATAN_TERMS 9

static float atan_small(float a)
{
    float c[ORC_ATAN_TERMS];
    for (int k = 0; k < ORC_ATAN_TERMS; ++k) {
        float inv = 1.0f / (float)(2 * k + 1);
        c[k] = (k & 1) ? -inv : inv;
    }
    float a2 = a * a;
    float p = c[ORC_ATAN_TERMS - 1];
    for (int k = ORC_ATAN_TERMS - 2; k >= 0; --k) p = c[k] + a2 * p;
    return a * p;
}

static float atan_unit(float t)   /* t in [0, 1] */
{
    const float tan_pi_8 = 0.41421356237309504880f;
    const float pi_4 = 0.78539816339744830962f;
    if (t > tan_pi_8) return pi_4 + atan_small((t - 1.0f) / (t + 1.0f));
    return atan_small(t);
}

float orc_atan2_pos(float y, float x)
{
    const float pi_2 = 1.57079632679489661923f;
    if (y == 0.0f) return 0.0f;                 /* includes y = x = 0 */
    if (y <= x) return atan_unit(y / x);
    return pi_2 - atan_unit(x / y);
}

/* ------------------------------------------------------------------------ */
/* a1: row-band index.  Right keypoint j covers image rows                  */
/* floor(y_j - r) .. ceil(y_j + r) with r = 2*scale[oct_j], clamped to the  */
/* image; each row lists its keypoints in ascending j (CSR).                */
/* Returns the number of entries, or -1 if it exceeds cap.                  */
/* ------------------------------------------------------------------------ */
static void band_rows(float y, float r, int H, int *lo, int *hi)
{
    int a = (int)floorf(y - r);
    int b = (int)ceilf(y + r);
    if (a < 0) a = 0;
    if (b > H - 1) b = H - 1;
    *lo = a;
    *hi = b;
}

int orc_row_index(int nr, const float *yr, const int8_t *octr, const float *sc,
                  int H, int *row_ptr, int *row_idx, int cap)
{
    int *count = (int *)calloc((size_t)H + 1, sizeof(int));
    for (int j = 0; j < nr; ++j) {
        int lo, hi;
        band_rows(yr[j], 2.0f * sc[octr[j]], H, &lo, &hi);
        for (int row = lo; row <= hi; ++row) count[row]++;
    }
    row_ptr[0] = 0;
    for (int row = 0; row < H; ++row) row_ptr[row + 1] = row_ptr[row] + count[row];
    int total = row_ptr[H];
    if (total > cap) {
        free(count);
        return -1;
    }
    for (int row = 0; row < H; ++row) count[row] = row_ptr[row];
    for (int j = 0; j < nr; ++j) {
        int lo, hi;
        band_rows(yr[j], 2.0f * sc[octr[j]], H, &lo, &hi);
        for (int row = lo; row <= hi; ++row) row_idx[count[row]++] = j;
    }
    free(count);
    return total;
}

/* ------------------------------------------------------------------------ */
/* a2: for left keypoint i, scan the row list of row (int)y_i.  A right     */
/* keypoint j is a candidate if its octave is within one of i's and its x   */
/* lies in [x_i - disp_hi, x_i - disp_lo], with disp_lo = 0 and disp_hi = bf / b (the   */
/* nearest depth is one baseline).  Best = smallest (d, j).  dist[i] is     */
/* that smallest d (-1 without candidates); best_r[i] = j if d < th_stereo. */
/* ------------------------------------------------------------------------ */
void orc_stereo_best(const orc_params *p, const orc_pinhole *cam,
                     const orc_keypoints *L, const orc_keypoints *R,
                     const int *row_ptr, const int *row_idx,
                     int32_t *best_r, int32_t *dist)
{
    const float z_near = cam->b;
    const float disp_lo = 0.0f;
    const float disp_hi = cam->bf / z_near;
    for (int i = 0; i < L->n; ++i) {
        best_r[i] = -1;
        dist[i] = -1;
        if (L->y[i] < 0.0f) continue;
        int row = (int)L->y[i];
        if (row >= cam->height) continue;
        if (row_ptr[row + 1] == row_ptr[row]) continue;
        const float u_lo = L->x[i] - disp_hi;
        const float u_hi = L->x[i] - disp_lo;
        if (u_hi < 0.0f) continue;
        const int oct_l = L->oct[i];
        int bestd = 1 << 30, bestj = -1;
        for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
            int j = row_idx[e];
            if (R->oct[j] < oct_l - 1 || R->oct[j] > oct_l + 1) continue;
            if (R->x[j] < u_lo || R->x[j] > u_hi) continue;
            int d = orc_hamming(L->desc + (size_t)i * ORC_DESC_BYTES,
                                R->desc + (size_t)j * ORC_DESC_BYTES);
            if (d < bestd || (d == bestd && j < bestj)) {
                bestd = d;
                bestj = j;
            }
        }
        if (bestj < 0) continue;
        dist[i] = bestd;
        if (bestd < p->th_stereo) best_r[i] = bestj;
    }
}

/* ------------------------------------------------------------------------ */
/* a3: SAD of the (2w+1)x(2w+1) left patch centred on (ul, vl) against the  */
/* right patches centred on (ur0 + k, vl), k = -L..L, at pyramid level      */
/* `level`.  Every patch first has its own centre pixel subtracted.         */
/* Returns 0 (sad untouched) unless the left window and all right windows   */
/* lie inside the level images.                                             */
/* ------------------------------------------------------------------------ */
int orc_sad_vector(const orc_params *p, const orc_pyramid *pl, const orc_pyramid *pr,
                   int level, int ul, int vl, int ur0, int32_t *sad)
{
    const int w = p->sad_w, L = p->sad_L;
    const int wl = pl->width[level], hl = pl->height[level];
    const int wr = pr->width[level], hr = pr->height[level];
    if (vl - w < 0 || vl + w > hl - 1 || vl + w > hr - 1) return 0;
    if (ul - w < 0 || ul + w > wl - 1) return 0;
    if (ur0 - L - w < 0 || ur0 + L + w > wr - 1) return 0;

    const uint8_t *IL = pl->data[level];
    const uint8_t *IR = pr->data[level];
    const int sl = pl->pitch[level], sr = pr->pitch[level];
    const int cL = IL[(size_t)vl * sl + ul];
    for (int k = -L; k <= L; ++k) {
        const int cR = IR[(size_t)vl * sr + (ur0 + k)];
        int s = 0;
        for (int dy = -w; dy <= w; ++dy) {
            for (int dx = -w; dx <= w; ++dx) {
                int a = IL[(size_t)(vl + dy) * sl + (ul + dx)] - cL;
                int b = IR[(size_t)(vl + dy) * sr + (ur0 + k + dx)] - cR;
                s += abs(a - b);
            }
        }
        sad[k + L] = s;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* a4: parabola through (k*-1, k*, k*+1) of the SAD curve, vertex offset    */
/* delta = (S- - S+) / (2 (S- + S+ - 2 S0)); right coordinate              */
/* uR = scale * (ur0 + k* + delta); disparity = xl - uR must lie in        */
/* [0, disp_hi); a disparity of exactly 0 is replaced by 0.01 px; depth =     */
/* bf / disparity.  Returns 1 if accepted.                                  */
/* ------------------------------------------------------------------------ */
int orc_subpixel(const int32_t *sad, int L, int kbest, int ur0, float scale, float xl,
                 float bf, float disp_hi, float *u_right, float *depth, float *delta)
{
    const float disp_lo = 0.0f;
    const float sad_m1 = (float)sad[kbest + L - 1];
    const float sad_0 = (float)sad[kbest + L];
    const float sad_p1 = (float)sad[kbest + L + 1];
    const float dk = (sad_m1 - sad_p1) / (2.0f * (sad_m1 + sad_p1 - 2.0f * sad_0));
    *delta = dk;
    if (dk < -1.0f || dk > 1.0f) return 0;   /* unreachable: |dk| <= 0.5 */
    float ur_sub = scale * ((float)ur0 + (float)kbest + dk);
    float disparity = xl - ur_sub;
    if (!(disparity >= disp_lo && disparity < disp_hi)) return 0;
    if (disparity <= 0.0f) {
        disparity = 0.01f;
        ur_sub = xl - 0.01f;
    }
    *depth = bf / disparity;
    *u_right = ur_sub;
    return 1;
}

/* ascending integer sort (insertion sort; n is a few thousand at most) */
static void sort_ints(int *v, int n)
{
    for (int i = 1; i < n; ++i) {
        int x = v[i], j = i - 1;
        while (j >= 0 && v[j] > x) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = x;
    }
}

/* ------------------------------------------------------------------------ */
/* a5: over the accepted matches (sad_best >= 0), median = element n/2 of   */
/* the ascending sort; every match with SAD >= factor * median loses its    */
/* u_right and depth (set to -1).  Nothing happens when n = 0.             */
/* ------------------------------------------------------------------------ */
void orc_median_reject(int n_kp, const int32_t *sad_best, float factor, float *u_right,
                       float *depth)
{
    int n = 0;
    for (int i = 0; i < n_kp; ++i)
        if (sad_best[i] >= 0) ++n;
    if (n == 0) return;
    int *v = (int *)malloc(sizeof(int) * (size_t)n);
    int m = 0;
    for (int i = 0; i < n_kp; ++i)
        if (sad_best[i] >= 0) v[m++] = sad_best[i];
    sort_ints(v, n);
    const int median = v[n / 2];
    const float sad_cut = factor * (float)median;
    for (int i = 0; i < n_kp; ++i) {
        if (sad_best[i] >= 0 && (float)sad_best[i] >= sad_cut) {
            u_right[i] = -1.0f;
            depth[i] = -1.0f;
        }
    }
    free(v);
}

void orc_stereo_pinhole(const orc_params *p, const orc_pinhole *cam,
                        const orc_keypoints *L, const orc_keypoints *R,
                        const orc_pyramid *pl, const orc_pyramid *pr,
                        int32_t *best_r, int32_t *dist, int32_t *sad_shift,
                        int32_t *sad_best, float *u_right, float *depth)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);

    /* a1 */
    const int H = cam->height;
    int *row_ptr = (int *)malloc(sizeof(int) * ((size_t)H + 1));
    int cap = 0;
    for (int j = 0; j < R->n; ++j) {
        int lo, hi;
        band_rows(R->y[j], 2.0f * sc[R->oct[j]], H, &lo, &hi);
        if (hi >= lo) cap += hi - lo + 1;
    }
    int *row_idx = (int *)malloc(sizeof(int) * ((size_t)cap + 1));
    orc_row_index(R->n, R->y, R->oct, sc, H, row_ptr, row_idx, cap);

    /* a2 */
    orc_stereo_best(p, cam, L, R, row_ptr, row_idx, best_r, dist);

    const float disp_hi = cam->bf / cam->b;
    const int Ls = p->sad_L;
    int32_t sad[2 * 64 + 1];

    for (int i = 0; i < L->n; ++i) {
        sad_shift[i] = ORC_NO_SHIFT;
        sad_best[i] = -1;
        u_right[i] = -1.0f;
        depth[i] = -1.0f;
        const int j = best_r[i];
        if (j < 0) continue;

        /* a3: level coordinates, SAD vector, first strict minimum */
        const int l = L->oct[i];
        const int ul = (int)roundf(L->x[i] * isc[l]);
        const int vl = (int)roundf(L->y[i] * isc[l]);
        const int ur0 = (int)roundf(R->x[j] * isc[l]);
        if (!orc_sad_vector(p, pl, pr, l, ul, vl, ur0, sad)) continue;
        int kbest = -Ls;
        for (int k = -Ls + 1; k <= Ls; ++k)
            if (sad[k + Ls] < sad[kbest + Ls]) kbest = k;
        sad_shift[i] = kbest;
        if (kbest == -Ls || kbest == Ls) continue;

        /* a4 */
        float delta;
        if (orc_subpixel(sad, Ls, kbest, ur0, sc[l], L->x[i], cam->bf, disp_hi, &u_right[i],
                         &depth[i], &delta))
            sad_best[i] = sad[kbest + Ls];
    }

    /* a5 */
    orc_median_reject(L->n, sad_best, p->median_factor, u_right, depth);
    free(row_ptr);
    free(row_idx);
}

/* ------------------------------------------------------------------------ */
/* a6: fisheye.  Left keypoints with x in [lap_l0, lap_l1] are matched by   */
/* brute force against right keypoints with x in [lap_r0, lap_r1].  d1, d2  */
/* are the two smallest (d, j); d2 = 256 if only one right keypoint exists. */
/* Accept j1 if (float)d1 < ratio * (float)d2.  Left keypoints outside the  */
/* overlap (or without candidates) get r_idx = d1 = d2 = -1.                */
/* ------------------------------------------------------------------------ */
void orc_stereo_fisheye(const orc_params *p, const orc_keypoints *L, const orc_keypoints *R,
                        float lap_l0, float lap_l1, float lap_r0, float lap_r1,
                        int32_t *r_idx, int32_t *d1, int32_t *d2)
{
    for (int i = 0; i < L->n; ++i) {
        r_idx[i] = -1;
        d1[i] = -1;
        d2[i] = -1;
        if (!(L->x[i] >= lap_l0 && L->x[i] <= lap_l1)) continue;
        int bd = 0, bj = -1, sd = 0, sj = -1;
        for (int j = 0; j < R->n; ++j) {
            if (!(R->x[j] >= lap_r0 && R->x[j] <= lap_r1)) continue;
            int d = orc_hamming(L->desc + (size_t)i * ORC_DESC_BYTES,
                                R->desc + (size_t)j * ORC_DESC_BYTES);
            /* keep the two smallest (d, j) pairs */
            if (bj < 0 || d < bd || (d == bd && j < bj)) {
                sd = bd;
                sj = bj;
                bd = d;
                bj = j;
            } else if (sj < 0 || d < sd || (d == sd && j < sj)) {
                sd = d;
                sj = j;
            }
        }
        if (bj < 0) continue;
        d1[i] = bd;
        d2[i] = (sj >= 0) ? sd : 256;
        if ((float)d1[i] < p->fisheye_ratio * (float)d2[i]) r_idx[i] = bj;
    }
}

/* ------------------------------------------------------------------------ */
/* a7: grid cell of a keypoint: round((x - min_x) * 64 / (max_x - min_x)),  */
/* same in y with 48 rows.  Returns 0 if the cell lies outside the grid.    */
/* ------------------------------------------------------------------------ */
int orc_grid_cell(float x, float y, float min_x, float max_x, float min_y, float max_y,
                  int *cx, int *cy)
{
    const float iw = (float)ORC_GRID_COLS / (max_x - min_x);
    const float ih = (float)ORC_GRID_ROWS / (max_y - min_y);
    *cx = (int)roundf((x - min_x) * iw);
    *cy = (int)roundf((y - min_y) * ih);
    if (*cx < 0 || *cx >= ORC_GRID_COLS || *cy < 0 || *cy >= ORC_GRID_ROWS) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* a8: frustum test and projection.  A point needs camera z > 0 (a point on */
/* the camera plane has no pinhole projection).  Shared part (after the     */
/* image test):                                                             */
/* distance to the camera centre within [dist_lo*dmin, dist_hi*dmax],      */
/* viewing cosine with the mean normal >= view_cos_min, predicted level =   */
/* smallest l with scale[l] >= dmax / dist (else S-1).                     */
/* out4 = (u, v, u_right, viewing cosine).  Returns 1 if in view.          */
/* ------------------------------------------------------------------------ */
static void transform(const float *R, const float *t, const float *P, float *Pc)
{
    Pc[0] = R[0] * P[0] + R[1] * P[1] + R[2] * P[2] + t[0];
    Pc[1] = R[3] * P[0] + R[4] * P[1] + R[5] * P[2] + t[1];
    Pc[2] = R[6] * P[0] + R[7] * P[1] + R[8] * P[2] + t[2];
}

static int distance_and_scale(const orc_params *p, const float *O, const float *Pw,
                              const float *nrm, float dmin, float dmax,
                              float *view_cos, int *level)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);
    const float PO[3] = {Pw[0] - O[0], Pw[1] - O[1], Pw[2] - O[2]};
    const float dist = sqrtf(PO[0] * PO[0] + PO[1] * PO[1] + PO[2] * PO[2]);
    const float d_far = p->dist_hi * dmax;
    const float d_near = p->dist_lo * dmin;
    if (dist < d_near || dist > d_far) return 0;
    const float vc = (PO[0] * nrm[0] + PO[1] * nrm[1] + PO[2] * nrm[2]) / dist;
    if (vc < p->view_cos_min) return 0;
    const float ratio = dmax / dist;
    int lv = p->nlevels - 1;
    for (int l = 0; l < p->nlevels; ++l) {
        if (sc[l] >= ratio) {
            lv = l;
            break;
        }
    }
    *view_cos = vc;
    *level = lv;
    return 1;
}

int orc_project_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                        const float *Pw, const float *nrm, float dmin, float dmax,
                        float *out4, int *level)
{
    float Pc[3];
    transform(T->R, T->t, Pw, Pc);
    if (!(Pc[2] > 0.0f)) return 0;   /* behind, on the camera plane, or NaN */
    const float invz = 1.0f / Pc[2];
    const float u = cam->fx * Pc[0] * invz + cam->cx;
    const float v = cam->fy * Pc[1] * invz + cam->cy;
    if (u < cam->min_x || u > cam->max_x) return 0;
    if (v < cam->min_y || v > cam->max_y) return 0;
    const float ur = u - cam->bf * invz;
    float vc;
    if (!distance_and_scale(p, T->O, Pw, nrm, dmin, dmax, &vc, level)) return 0;
    out4[0] = u;
    out4[1] = v;
    out4[2] = ur;
    out4[3] = vc;
    return 1;
}

/* Kannala-Brandt (equidistant, 4 coefficients):                           */
/*   rho = |(x, y)|, theta = atan2(rho, z),                                */
/*   theta_d = theta * (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8) */
/*   (Horner in theta^2), u = fx * theta_d * x / rho + cx (rho = 0: u = cx). */
static void kb8_project(const orc_kb8 *cam, const float *Pc, float *u, float *v)
{
    const float rho = sqrtf(Pc[0] * Pc[0] + Pc[1] * Pc[1]);
    if (rho == 0.0f) {
        *u = cam->cx;
        *v = cam->cy;
        return;
    }
    const float theta = orc_atan2_pos(rho, Pc[2]);
    const float t2 = theta * theta;
    float poly = cam->k[3];
    poly = cam->k[2] + t2 * poly;
    poly = cam->k[1] + t2 * poly;
    poly = cam->k[0] + t2 * poly;
    poly = 1.0f + t2 * poly;
    const float thetad = theta * poly;
    *u = cam->fx * thetad * Pc[0] / rho + cam->cx;
    *v = cam->fy * thetad * Pc[1] / rho + cam->cy;
}

int orc_project_kb8(const orc_params *p, const orc_kb8 *cam, const float *R, const float *t,
                    const float *O, const float *Pw, const float *nrm, float dmin, float dmax,
                    float *out4, int *level)
{
    float Pc[3];
    transform(R, t, Pw, Pc);
    if (!(Pc[2] > 0.0f)) return 0;   /* behind, on the camera plane, or NaN */
    float u, v;
    kb8_project(cam, Pc, &u, &v);
    if (u < cam->min_x || u > cam->max_x) return 0;
    if (v < cam->min_y || v > cam->max_y) return 0;
    float vc;
    if (!distance_and_scale(p, O, Pw, nrm, dmin, dmax, &vc, level)) return 0;
    out4[0] = u;
    out4[1] = v;
    out4[2] = -1.0f;
    out4[3] = vc;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* f1: fisheye triangulation.  The paper says only that stereo matches      */
/* serve to compute depth (section II-B); the reading here:                 */
/*  - unprojection of a Kannala-Brandt pixel: m = ((u-cx)/fx, (v-cy)/fy),    */
/*    theta_d = |m|; theta solves theta*(1+k1 t+k2 t^2+k3 t^3+k4 t^4) =      */
/*    theta_d (t = theta^2) by kb_iters Newton steps from theta = theta_d,   */
/*    kept if the residual is at most 2e-6 rad where the model still rises   */
/*    (a pixel past the lens model's maximum has no ray);                     */
/*    the ray is (m * sin(theta)/theta_d, cos(theta)) ((0, 0, 1) at the       */
/*    principal point);                                                       */
/*  - the two rays, in left-camera coordinates (right centre C = -R^T t,     */
/*    right ray R^T r), are joined by their common perpendicular; the point  */
/*    is its midpoint, kept when the rays are not parallel                   */
/*    (|l x r|^2 > 1e-10 |l|^2 |r|^2), both ray parameters are positive and  */
/*    its depth (left z) exceeds min_depth.                                  */
/* sin and cos are their Taylor series (written out below, |t| <= 2 keeps   */
/* the remainder under 2e-8), so both implementations share one definition.*/
/* ------------------------------------------------------------------------ */
float orc_sin_series(float t)
{
    /* t * (1 - t^2/3! + t^4/5! - ... + t^12/13!), Horner in t^2 */
    const float t2 = t * t;
    float s = 1.60590444e-10f;               /*  1/13! */
    s = -2.50521079e-08f + t2 * s;           /* -1/11! */
    s = 2.75573188e-06f + t2 * s;            /*  1/9!  */
    s = -1.98412701e-04f + t2 * s;           /* -1/7!  */
    s = 8.33333377e-03f + t2 * s;            /*  1/5!  */
    s = -1.66666672e-01f + t2 * s;           /* -1/3!  */
    s = 1.0f + t2 * s;
    return t * s;
}

float orc_cos_series(float t)
{
    /* 1 - t^2/2! + t^4/4! - ... - t^14/14!, Horner in t^2 */
    const float t2 = t * t;
    float c = -1.14707454e-11f;              /* -1/14! */
    c = 2.08767559e-09f + t2 * c;            /*  1/12! */
    c = -2.75573200e-07f + t2 * c;           /* -1/10! */
    c = 2.48015876e-05f + t2 * c;            /*  1/8!  */
    c = -1.38888892e-03f + t2 * c;           /* -1/6!  */
    c = 4.16666679e-02f + t2 * c;            /*  1/4!  */
    c = -0.5f + t2 * c;                      /* -1/2!  */
    return 1.0f + t2 * c;
}

int orc_unproject_kb8(const orc_kb8 *cam, int iters, float u, float v, float *ray)
{
    const float mx = (u - cam->cx) / cam->fx;
    const float my = (v - cam->cy) / cam->fy;
    const float thd = sqrtf(mx * mx + my * my);
    if (thd == 0.0f) {
        ray[0] = 0.0f;
        ray[1] = 0.0f;
        ray[2] = 1.0f;
        return 1;
    }
    float th = thd, f = 0.0f, dp = 1.0f;
    for (int it = 0; it <= iters; ++it) {
        const float t2 = th * th;
        float poly = cam->k[3];
        poly = cam->k[2] + t2 * poly;
        poly = cam->k[1] + t2 * poly;
        poly = cam->k[0] + t2 * poly;
        poly = 1.0f + t2 * poly;
        f = th * poly - thd;
        dp = 9.0f * cam->k[3];
        dp = 7.0f * cam->k[2] + t2 * dp;
        dp = 5.0f * cam->k[1] + t2 * dp;
        dp = 3.0f * cam->k[0] + t2 * dp;
        dp = 1.0f + t2 * dp;
        if (it == iters) break;                  /* the last pass only measures the residual */
        th = th - f / dp;
    }
    /* no solution (a pixel beyond the lens model's monotonic range), not
     * converged, or outside the series' range */
    if (!(fabsf(f) <= 2e-6f && dp > 0.0f && th >= 0.0f && th <= 2.0f)) return 0;
    const float s = orc_sin_series(th) / thd;
    ray[0] = mx * s;
    ray[1] = my * s;
    ray[2] = orc_cos_series(th);
    return 1;
}

static float dot3(const float *a, const float *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const float *a, const float *b, float *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Lines s*l (left centre at the origin) and C + t*r: with n = l x r the
 * closest points have s = ((C x r).n)/(n.n) and t = ((C x l).n)/(n.n); the
 * cross products keep FP32 accurate for rays a few milliradians apart. */
int orc_triangulate(const float *ray_l, const float *ray_r, const float *R_rl, const float *t_rl,
                    float min_depth, float *xyz)
{
    float C[3], dr[3], n[3], cr[3], cl[3];
    for (int i = 0; i < 3; ++i) {
        C[i] = -(R_rl[i] * t_rl[0] + R_rl[3 + i] * t_rl[1] + R_rl[6 + i] * t_rl[2]);
        dr[i] = R_rl[i] * ray_r[0] + R_rl[3 + i] * ray_r[1] + R_rl[6 + i] * ray_r[2];
    }
    cross3(ray_l, dr, n);
    const float nn = dot3(n, n);
    if (!(nn > 1e-10f * (dot3(ray_l, ray_l) * dot3(dr, dr)))) return 0;
    cross3(C, dr, cr);
    cross3(C, ray_l, cl);
    const float s = dot3(cr, n) / nn;
    const float t = dot3(cl, n) / nn;
    if (!(s > 0.0f && t > 0.0f)) return 0;
    for (int i = 0; i < 3; ++i) xyz[i] = 0.5f * (s * ray_l[i] + (C[i] + t * dr[i]));
    return xyz[2] > min_depth;
}

void orc_fisheye_triangulate(const orc_params *p, const orc_kb8 *camL, const orc_kb8 *camR,
                             const float *R_rl, const float *t_rl, const orc_keypoints *L,
                             const orc_keypoints *R, const int32_t *r_idx, float *depth, float *xyz4)
{
    for (int i = 0; i < L->n; ++i) {
        float P[3] = {0.0f, 0.0f, 0.0f}, rl[3], rr[3];
        int ok = 0;
        const int j = r_idx[i];
        if (j >= 0 && orc_unproject_kb8(camL, p->kb_iters, L->x[i], L->y[i], rl) &&
            orc_unproject_kb8(camR, p->kb_iters, R->x[j], R->y[j], rr))
            ok = orc_triangulate(rl, rr, R_rl, t_rl, p->min_depth, P);
        depth[i] = ok ? P[2] : -1.0f;
        if (xyz4) {
            for (int c = 0; c < 3; ++c) xyz4[4 * i + c] = ok ? P[c] : 0.0f;
            xyz4[4 * i + 3] = ok ? 1.0f : 0.0f;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a9 + a10 for one camera.  For each map point in view (level >= 0):      */
/*   radius = (narrow if cos > view_cos_narrow else wide) * th * scale[lv];  */
/*   cells [floor((u-min_x-r)*iw), ceil((u-min_x+r)*iw)] clamped to the     */
/*   grid (same in y); keep keypoints of those cells with octave in         */
/*   [lv-1, lv], |x-u| < r, |y-v| < r, not taken, and (if u_right is given) */
/*   u_right <= 0 or |ur - u_right| <= r.  d1/d2 = two smallest (d, k);     */
/*   accept k1 if d1 <= th_search and not (ratio applies and                */
/*   d1 > nn_ratio * d2), where the ratio applies when both share an octave */
/*   (or always with ratio_any_octave).                                     */
/*   a10: each keypoint keeps the smallest (d1, m) among the map points     */
/*   that accepted it; the others get mp_kp = -1.                           */
/* ------------------------------------------------------------------------ */
void orc_search_camera(const orc_params *p, float min_x, float max_x, float min_y, float max_y,
                       const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                       int M, const uint8_t *mp_desc, const int8_t *level, const float *proj,
                       int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);
    const float iw = (float)ORC_GRID_COLS / (max_x - min_x);
    const float ih = (float)ORC_GRID_ROWS / (max_y - min_y);

    /* a7: cell lists, cells in column-major order (ix, then iy), keypoints in
     * ascending index inside a cell */
    const int ncell = ORC_GRID_COLS * ORC_GRID_ROWS;
    int *cell_ptr = (int *)calloc((size_t)ncell + 1, sizeof(int));
    int *cell_idx = (int *)malloc(sizeof(int) * ((size_t)K->n + 1));
    int *kcell = (int *)malloc(sizeof(int) * ((size_t)K->n + 1));
    for (int k = 0; k < K->n; ++k) {
        int cx, cy;
        kcell[k] = -1;
        if (orc_grid_cell(K->x[k], K->y[k], min_x, max_x, min_y, max_y, &cx, &cy)) {
            kcell[k] = cx * ORC_GRID_ROWS + cy;
            cell_ptr[kcell[k] + 1]++;
        }
    }
    for (int c = 0; c < ncell; ++c) cell_ptr[c + 1] += cell_ptr[c];
    int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
    for (int c = 0; c < ncell; ++c) fill[c] = cell_ptr[c];
    for (int k = 0; k < K->n; ++k)
        if (kcell[k] >= 0) cell_idx[fill[kcell[k]]++] = k;

    int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * ((size_t)K->n + 1));
    for (int k = 0; k < K->n; ++k) owner[k] = -1;

    for (int m = 0; m < M; ++m) {
        mp_kp[m] = -1;
        mp_d1[m] = -1;
        mp_d2[m] = -1;
        const int lv = level[m];
        if (lv < 0) continue;
        const float u = proj[4 * m + 0], v = proj[4 * m + 1];
        const float ur = proj[4 * m + 2], vc = proj[4 * m + 3];
        float r = (vc > p->view_cos_narrow) ? p->radius_narrow : p->radius_wide;
        r = r * p->search_th;
        r = r * sc[lv];
        const int minLevel = lv - 1, maxLevel = lv;

        int x0 = (int)floorf((u - min_x - r) * iw);
        if (x0 < 0) x0 = 0;
        int x1 = (int)ceilf((u - min_x + r) * iw);
        if (x1 > ORC_GRID_COLS - 1) x1 = ORC_GRID_COLS - 1;
        int y0 = (int)floorf((v - min_y - r) * ih);
        if (y0 < 0) y0 = 0;
        int y1 = (int)ceilf((v - min_y + r) * ih);
        if (y1 > ORC_GRID_ROWS - 1) y1 = ORC_GRID_ROWS - 1;
        if (x0 >= ORC_GRID_COLS || x1 < 0 || y0 >= ORC_GRID_ROWS || y1 < 0) continue;

        int bd = 0, bk = -1, sd = 0, sk = -1;
        for (int ix = x0; ix <= x1; ++ix) {
            for (int iy = y0; iy <= y1; ++iy) {
                const int c = ix * ORC_GRID_ROWS + iy;
                for (int e = cell_ptr[c]; e < cell_ptr[c + 1]; ++e) {
                    const int k = cell_idx[e];
                    if (K->oct[k] < minLevel || K->oct[k] > maxLevel) continue;
                    const float distx = K->x[k] - u;
                    const float disty = K->y[k] - v;
                    if (!(fabsf(distx) < r && fabsf(disty) < r)) continue;
                    if (taken && taken[k]) continue;
                    if (u_right && u_right[k] > 0.0f) {
                        const float er = fabsf(ur - u_right[k]);
                        if (er > r) continue;
                    }
                    const int d = orc_hamming(mp_desc + (size_t)m * ORC_DESC_BYTES,
                                              K->desc + (size_t)k * ORC_DESC_BYTES);
                    if (bk < 0 || d < bd || (d == bd && k < bk)) {
                        sd = bd;
                        sk = bk;
                        bd = d;
                        bk = k;
                    } else if (sk < 0 || d < sd || (d == sd && k < sk)) {
                        sd = d;
                        sk = k;
                    }
                }
            }
        }
        if (bk < 0) continue;
        mp_d1[m] = bd;
        mp_d2[m] = (sk >= 0) ? sd : 256;
        if (bd > p->th_search) continue;
        const int oct1 = K->oct[bk];
        const int oct2 = (sk >= 0) ? K->oct[sk] : -1;
        if ((p->ratio_any_octave || oct1 == oct2) &&
            (float)bd > p->nn_ratio * (float)mp_d2[m])
            continue;
        /* a10: claim keypoint bk with key (d1, m); the smaller key wins */
        const int64_t key = ((int64_t)bd << 32) | (int64_t)m;
        if (owner[bk] < 0 || key < owner[bk]) owner[bk] = key;
        mp_kp[m] = bk;
    }
    for (int k = 0; k < K->n; ++k) kp_mp[k] = (owner[k] < 0) ? -1 : (int32_t)(owner[k] & 0xffffffff);
    for (int m = 0; m < M; ++m)
        if (mp_kp[m] >= 0 && kp_mp[mp_kp[m]] != m) mp_kp[m] = -1;
    free(owner);
    free(fill);
    free(kcell);
    free(cell_idx);
    free(cell_ptr);
}

void orc_search_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                        const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                        int M, const float *pos, const float *nrm, const uint8_t *mp_desc,
                        const uint8_t *skip, int8_t *level, float *proj,
                        int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp)
{
    for (int m = 0; m < M; ++m) {
        level[m] = -1;
        proj[4 * m + 0] = proj[4 * m + 1] = proj[4 * m + 2] = proj[4 * m + 3] = 0.0f;
        if (skip && skip[m]) continue;
        int lv;
        if (orc_project_pinhole(p, cam, T, pos + 4 * m, nrm + 4 * m, pos[4 * m + 3],
                                nrm[4 * m + 3], proj + 4 * m, &lv))
            level[m] = (int8_t)lv;
        else
            proj[4 * m + 0] = proj[4 * m + 1] = proj[4 * m + 2] = proj[4 * m + 3] = 0.0f;
    }
    orc_search_camera(p, cam->min_x, cam->max_x, cam->min_y, cam->max_y, K, u_right, taken,
                      M, mp_desc, level, proj, mp_kp, mp_d1, mp_d2, kp_mp);
}

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
                        int32_t *mp_d2_r, int32_t *kp_mp_r)
{
    /* right camera: T_rw = T_rl * T_lw, composed in FP32 in this order */
    float Rr[9], tr[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Rr[3 * i + j] = R_rl[3 * i + 0] * T->R[0 + j] + R_rl[3 * i + 1] * T->R[3 + j] +
                            R_rl[3 * i + 2] * T->R[6 + j];
        tr[i] = R_rl[3 * i + 0] * T->t[0] + R_rl[3 * i + 1] * T->t[1] +
                R_rl[3 * i + 2] * T->t[2] + t_rl[i];
    }
    for (int m = 0; m < M; ++m) {
        int lv;
        level_l[m] = level_r[m] = -1;
        for (int c = 0; c < 4; ++c) proj_l[4 * m + c] = proj_r[4 * m + c] = 0.0f;
        if (skip && skip[m]) continue;
        const float *Pw = pos + 4 * m, *n = nrm + 4 * m;
        if (orc_project_kb8(p, camL, T->R, T->t, T->O, Pw, n, Pw[3], n[3], proj_l + 4 * m, &lv))
            level_l[m] = (int8_t)lv;
        else
            for (int c = 0; c < 4; ++c) proj_l[4 * m + c] = 0.0f;
        if (orc_project_kb8(p, camR, Rr, tr, O_right, Pw, n, Pw[3], n[3], proj_r + 4 * m, &lv))
            level_r[m] = (int8_t)lv;
        else
            for (int c = 0; c < 4; ++c) proj_r[4 * m + c] = 0.0f;
    }
    orc_search_camera(p, camL->min_x, camL->max_x, camL->min_y, camL->max_y, KL, NULL, takenL,
                      M, mp_desc, level_l, proj_l, mp_kp_l, mp_d1_l, mp_d2_l, kp_mp_l);
    orc_search_camera(p, camR->min_x, camR->max_x, camR->min_y, camR->max_y, KR, NULL, takenR,
                      M, mp_desc, level_r, proj_r, mp_kp_r, mp_d1_r, mp_d2_r, kp_mp_r);
}

/* ------------------------------------------------------------------------ */
/* f2: search by projection of the last frame's points.  The paper runs    */
/* the same search by projection in the initial pose estimation, adapted,  */
/* with the previous frame's points as input (sections II-C, IV-E).  The    */
/* adaptation is a reading of the algorithm family's last-frame search:     */
/*  - a point is in view if its camera z > 0 and its projection lies in the */
/*    image bounds (no distance or viewing-angle test); its octave is the   */
/*    octave of the keypoint that observed it in the last frame; points     */
/*    with an octave outside [0, S-1] are not searched;                     */
/*  - radius = th_last * scale[octave];                                     */
/*  - octave window by the camera motion: with c = R_last O_cur + t_last    */
/*    (the current centre in last-camera coordinates), forward (c.z > b)    */
/*    keeps octaves >= the point's, backward (-c.z > b) octaves <= it,      */
/*    otherwise octave-1 .. octave+1;                                       */
/*  - accept the best distance d1 <= th_search, without a ratio test;       */
/*  - the cell window, taken flags, stereo consistency and the conflict     */
/*    rule are those of a9 and a10.                                         */
/* ------------------------------------------------------------------------ */
int orc_motion(const orc_pose *cur, const orc_pose *last, float b)
{
    float c[3];
    transform(last->R, last->t, cur->O, c);
    if (c[2] > b) return 1;
    if (-c[2] > b) return -1;
    return 0;
}

void orc_search_last_camera(const orc_params *p, float min_x, float max_x, float min_y, float max_y,
                            const orc_keypoints *K, const float *u_right, const uint8_t *taken,
                            int M, const uint8_t *mp_desc, const int8_t *level, const float *proj,
                            int motion, int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2,
                            int32_t *kp_mp)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);
    const float iw = (float)ORC_GRID_COLS / (max_x - min_x);
    const float ih = (float)ORC_GRID_ROWS / (max_y - min_y);
    int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * ((size_t)K->n + 1));
    for (int k = 0; k < K->n; ++k) owner[k] = -1;
    /* every keypoint's grid cell (a7) */
    int *kx = (int *)malloc(sizeof(int) * ((size_t)K->n + 1));
    int *ky = (int *)malloc(sizeof(int) * ((size_t)K->n + 1));
    for (int k = 0; k < K->n; ++k)
        if (!orc_grid_cell(K->x[k], K->y[k], min_x, max_x, min_y, max_y, &kx[k], &ky[k])) kx[k] = -1;

    for (int m = 0; m < M; ++m) {
        mp_kp[m] = -1;
        mp_d1[m] = -1;
        mp_d2[m] = -1;
        const int lv = level[m];
        if (lv < 0) continue;
        const float u = proj[4 * m + 0], v = proj[4 * m + 1], ur = proj[4 * m + 2];
        const float r = p->th_last * sc[lv];
        const int minLevel = motion > 0 ? lv : (motion < 0 ? 0 : lv - 1);
        const int maxLevel = motion > 0 ? p->nlevels - 1 : (motion < 0 ? lv : lv + 1);
        int x0 = (int)floorf((u - min_x - r) * iw);
        if (x0 < 0) x0 = 0;
        int x1 = (int)ceilf((u - min_x + r) * iw);
        if (x1 > ORC_GRID_COLS - 1) x1 = ORC_GRID_COLS - 1;
        int y0 = (int)floorf((v - min_y - r) * ih);
        if (y0 < 0) y0 = 0;
        int y1 = (int)ceilf((v - min_y + r) * ih);
        if (y1 > ORC_GRID_ROWS - 1) y1 = ORC_GRID_ROWS - 1;
        if (x0 >= ORC_GRID_COLS || x1 < 0 || y0 >= ORC_GRID_ROWS || y1 < 0) continue;
        /* the keypoints of the window's cells, in ascending index */
        int bd = 0, bk = -1, sd = 0, sk = -1;
        for (int k = 0; k < K->n; ++k) {
            if (kx[k] < x0 || kx[k] > x1 || ky[k] < y0 || ky[k] > y1) continue;
            if (K->oct[k] < minLevel || K->oct[k] > maxLevel) continue;
            if (!(fabsf(K->x[k] - u) < r && fabsf(K->y[k] - v) < r)) continue;
            if (taken && taken[k]) continue;
            if (u_right && u_right[k] > 0.0f && fabsf(ur - u_right[k]) > r) continue;
            const int d = orc_hamming(mp_desc + (size_t)m * ORC_DESC_BYTES, K->desc + (size_t)k * ORC_DESC_BYTES);
            if (bk < 0 || d < bd) {
                sd = bd;
                sk = bk;
                bd = d;
                bk = k;
            } else if (sk < 0 || d < sd) {
                sd = d;
                sk = k;
            }
        }
        if (bk < 0) continue;
        mp_d1[m] = bd;
        mp_d2[m] = (sk >= 0) ? sd : 256;
        if (bd > p->th_search) continue;
        const int64_t key = ((int64_t)bd << 32) | (int64_t)m;
        if (owner[bk] < 0 || key < owner[bk]) owner[bk] = key;
        mp_kp[m] = bk;
    }
    for (int k = 0; k < K->n; ++k) kp_mp[k] = (owner[k] < 0) ? -1 : (int32_t)(owner[k] & 0xffffffff);
    for (int m = 0; m < M; ++m)
        if (mp_kp[m] >= 0 && kp_mp[mp_kp[m]] != m) mp_kp[m] = -1;
    free(ky);
    free(kx);
    free(owner);
}

/* in-view test and projection of a last-frame point (f2) */
static int last_level(const orc_params *p, const int8_t *last_oct, int m)
{
    const int lv = last_oct[m];
    return (lv >= 0 && lv < p->nlevels) ? lv : -1;
}

void orc_search_last_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T,
                             const orc_pose *T_last, const orc_keypoints *K, const float *u_right,
                             const uint8_t *taken, int M, const float *pos, const uint8_t *mp_desc,
                             const int8_t *last_oct, const uint8_t *skip, int8_t *level, float *proj,
                             int32_t *mp_kp, int32_t *mp_d1, int32_t *mp_d2, int32_t *kp_mp)
{
    for (int m = 0; m < M; ++m) {
        level[m] = -1;
        for (int c = 0; c < 4; ++c) proj[4 * m + c] = 0.0f;
        if ((skip && skip[m]) || last_level(p, last_oct, m) < 0) continue;
        float Pc[3];
        transform(T->R, T->t, pos + 4 * m, Pc);
        if (!(Pc[2] > 0.0f)) continue;
        const float invz = 1.0f / Pc[2];
        const float u = cam->fx * Pc[0] * invz + cam->cx;
        const float v = cam->fy * Pc[1] * invz + cam->cy;
        if (u < cam->min_x || u > cam->max_x || v < cam->min_y || v > cam->max_y) continue;
        level[m] = (int8_t)last_level(p, last_oct, m);
        proj[4 * m + 0] = u;
        proj[4 * m + 1] = v;
        proj[4 * m + 2] = u - cam->bf * invz;
    }
    orc_search_last_camera(p, cam->min_x, cam->max_x, cam->min_y, cam->max_y, K, u_right, taken, M,
                           mp_desc, level, proj, orc_motion(T, T_last, cam->b), mp_kp, mp_d1, mp_d2,
                           kp_mp);
}

void orc_search_last_fisheye(const orc_params *p, const orc_kb8 *camL, const orc_kb8 *camR,
                             const float *R_rl, const float *t_rl, float b, const orc_pose *T,
                             const orc_pose *T_last, const orc_keypoints *KL, const uint8_t *takenL,
                             const orc_keypoints *KR, const uint8_t *takenR, int M, const float *pos,
                             const uint8_t *mp_desc, const int8_t *last_oct, const uint8_t *skip,
                             int8_t *level_l, float *proj_l, int32_t *mp_kp_l, int32_t *mp_d1_l,
                             int32_t *mp_d2_l, int32_t *kp_mp_l,
                             int8_t *level_r, float *proj_r, int32_t *mp_kp_r, int32_t *mp_d1_r,
                             int32_t *mp_d2_r, int32_t *kp_mp_r)
{
    /* right camera pose R_rw = R_rl R_lw, t_rw = R_rl t_lw + t_rl (as in a8) */
    float Rr[9], tr[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Rr[3 * i + j] = R_rl[3 * i] * T->R[j] + R_rl[3 * i + 1] * T->R[3 + j] + R_rl[3 * i + 2] * T->R[6 + j];
        tr[i] = R_rl[3 * i] * T->t[0] + R_rl[3 * i + 1] * T->t[1] + R_rl[3 * i + 2] * T->t[2] + t_rl[i];
    }
    for (int m = 0; m < M; ++m) {
        level_l[m] = level_r[m] = -1;
        for (int c = 0; c < 4; ++c) proj_l[4 * m + c] = proj_r[4 * m + c] = 0.0f;
        if ((skip && skip[m]) || last_level(p, last_oct, m) < 0) continue;
        for (int side = 0; side < 2; ++side) {
            const orc_kb8 *cam = side ? camR : camL;
            float Pc[3], u, v;
            transform(side ? Rr : T->R, side ? tr : T->t, pos + 4 * m, Pc);
            if (!(Pc[2] > 0.0f)) continue;
            kb8_project(cam, Pc, &u, &v);
            if (u < cam->min_x || u > cam->max_x || v < cam->min_y || v > cam->max_y) continue;
            int8_t *lv = side ? level_r : level_l;
            float *pr = side ? proj_r : proj_l;
            lv[m] = (int8_t)last_level(p, last_oct, m);
            pr[4 * m + 0] = u;
            pr[4 * m + 1] = v;
            pr[4 * m + 2] = -1.0f;
        }
    }
    const int motion = orc_motion(T, T_last, b);
    orc_search_last_camera(p, camL->min_x, camL->max_x, camL->min_y, camL->max_y, KL, NULL, takenL, M,
                           mp_desc, level_l, proj_l, motion, mp_kp_l, mp_d1_l, mp_d2_l, kp_mp_l);
    orc_search_last_camera(p, camR->min_x, camR->max_x, camR->min_y, camR->max_y, KR, NULL, takenR, M,
                           mp_desc, level_r, proj_r, motion, mp_kp_r, mp_d1_r, mp_d2_r, kp_mp_r);
}

/* ------------------------------------------------------------------------ */
/* f3 (pyramid part): the image pyramid built from level 0.  The paper runs */
/* ORB extraction on the GPU so that the pyramid, most of stereo matching's */
/* input, never crosses the bus (section IV-B); it prints no resampling.     */
/* Reading (each level straight from level 0, as the family resizes):      */
/*  - level l is round(W / scale[l]) x round(H / scale[l]) (FP32 division);  */
/*  - output pixel (x, y) samples level 0 at xs = (x + 0.5) * (W / w) - 0.5, */
/*    ys likewise, each clamped to [0, W-1] / [0, H-1], bilinearly:         */
/*    with x0 = floor(xs), x1 = min(x0 + 1, W - 1), fx = xs - x0 (same in y),*/
/*    top = I(x0,y0)(1-fx) + I(x1,y0) fx, bottom likewise on y1,            */
/*    value = top (1-fy) + bottom fy, rounded half to even and clamped to   */
/*    [0, 255]; FP32, in this order.                                         */
/* ------------------------------------------------------------------------ */
void orc_pyramid_sizes(int W, int H, int nlevels, float s, int *w, int *h)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(nlevels, s, sc, isc);
    for (int l = 0; l < nlevels; ++l) {
        w[l] = (int)roundf((float)W / sc[l]);
        h[l] = (int)roundf((float)H / sc[l]);
    }
}

void orc_resample_level(const uint8_t *src, int W, int H, int pitch, uint8_t *dst, int w, int h, int dpitch)
{
    const float sx = (float)W / (float)w, sy = (float)H / (float)h;
    for (int y = 0; y < h; ++y) {
        float ys = ((float)y + 0.5f) * sy - 0.5f;
        if (ys < 0.0f) ys = 0.0f;
        if (ys > (float)(H - 1)) ys = (float)(H - 1);
        const int y0 = (int)floorf(ys);
        const int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
        const float fy = ys - (float)y0;
        for (int x = 0; x < w; ++x) {
            float xs = ((float)x + 0.5f) * sx - 0.5f;
            if (xs < 0.0f) xs = 0.0f;
            if (xs > (float)(W - 1)) xs = (float)(W - 1);
            const int x0 = (int)floorf(xs);
            const int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
            const float fx = xs - (float)x0;
            const float p00 = src[(size_t)y0 * pitch + x0], p01 = src[(size_t)y0 * pitch + x1];
            const float p10 = src[(size_t)y1 * pitch + x0], p11 = src[(size_t)y1 * pitch + x1];
            const float top = p00 * (1.0f - fx) + p01 * fx;
            const float bot = p10 * (1.0f - fx) + p11 * fx;
            float v = rintf(top * (1.0f - fy) + bot * fy);
            if (v < 0.0f) v = 0.0f;
            if (v > 255.0f) v = 255.0f;
            dst[(size_t)y * dpitch + x] = (uint8_t)v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* f4: pose optimization.  The paper's tracking refines the camera pose     */
/* with all the map points its search found in the frame (section II-D);    */
/* FastTrack switches the step off (section IV-F).  The reading, the        */
/* algorithm family's motion-only optimization, in double precision:       */
/*  - observations: a map point m matched to keypoint k = mp_kp[m] >= 0     */
/*    is observed at (x_k, y_k) and, when u_right[k] >= 0, also at the      */
/*    right coordinate u_right[k] (three residuals; else two).  Its weight  */
/*    is w = 1 / scale[oct_k]^2 (scale from the FP32 table).                */
/*  - the pose starts at the search's pose; every observation starts as an  */
/*    inlier.                                                               */
/*  - po_rounds rounds; a round runs only while at least 3 observations are */
/*    inliers.  It takes po_iters Gauss-Newton steps over the inliers that  */
/*    lie in front of the camera (z > 0): residual e = observation -        */
/*    projection, chi2 = w |e|^2, Huber factor h = 1 if chi2 <= th else     */
/*    sqrt(th / chi2) (th the threshold of the observation's kind; h = 1    */
/*    without Huber); H += h w J^T J, g += h w J^T e, J the derivative of   */
/*    the projection for a perturbation exp(d) multiplied on the left of    */
/*    the pose; d solves H d = g (Cholesky; if H is not positive definite   */
/*    the optimization stops with the current pose); the pose becomes       */
/*    exp(d) (R, t).                                                        */
/*  - after each round every observation is classified again at the new     */
/*    pose: an outlier if z <= 0 or chi2 > th, else an inlier.              */
/*  - exp(d), d = (w, v): theta = |w|, R_d = I + a [w]x + b [w]x^2,          */
/*    V = I + b [w]x + c [w]x^2, a = sin(theta)/theta,                       */
/*    b = (1 - cos(theta))/theta^2, c = (theta - sin(theta))/theta^3, and   */
/*    below theta = 0.01 their series 1 - theta^2/6, 1/2 - theta^2/24,      */
/*    1/6 - theta^2/120; then R <- R_d R, t <- R_d t + V v.                 */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

void orc_se3_exp(const double *d6, double *R9, double *V9)
{
    const double *w = d6;
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b, c;
    if (th < 0.01) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
        c = (th - sin(th)) / (th2 * th);
    }
    const double W[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    double W2[9];
    mat3_mul(W, W, W2);
    for (int i = 0; i < 9; ++i) {
        const double id = (i % 4 == 0) ? 1.0 : 0.0;
        R9[i] = id + a * W[i] + b * W2[i];
        V9[i] = id + b * W[i] + c * W2[i];
    }
}

/* Residual e = obs - projection of world point Pw at pose (R, t) and its
 * Jacobian J (rows u, v[, u_right], 6 columns: rotation then translation of
 * the left perturbation).  Returns 0 if the point is not in front (z <= 0). */
int orc_pose_residual(const orc_pinhole *cam, const double *R9, const double *t3, const float *Pw,
                      const double *obs3, int stereo, double *e3, double *J18)
{
    const double P[3] = {Pw[0], Pw[1], Pw[2]};
    double Pc[3];
    for (int i = 0; i < 3; ++i) Pc[i] = R9[3 * i] * P[0] + R9[3 * i + 1] * P[1] + R9[3 * i + 2] * P[2] + t3[i];
    const double x = Pc[0], y = Pc[1], z = Pc[2];
    if (!(z > 0.0)) return 0;
    const double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy, bf = cam->bf;
    const double iz = 1.0 / z, iz2 = iz * iz;
    const double u = fx * x * iz + cx, v = fy * y * iz + cy;
    e3[0] = obs3[0] - u;
    e3[1] = obs3[1] - v;
    e3[2] = stereo ? obs3[2] - (u - bf * iz) : 0.0;
    /* d projection / d Pc */
    const double D[9] = {fx * iz, 0.0, -fx * x * iz2,
                         0.0, fy * iz, -fy * y * iz2,
                         fx * iz, 0.0, -fx * x * iz2 + bf * iz2};
    /* d Pc / d (w, v) = [ -[Pc]x | I ] */
    const double S[18] = {0.0, z, -y, 1.0, 0.0, 0.0,
                          -z, 0.0, x, 0.0, 1.0, 0.0,
                          y, -x, 0.0, 0.0, 0.0, 1.0};
    const int rows = stereo ? 3 : 2;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c)
            J18[6 * r + c] = r < rows ? D[3 * r] * S[c] + D[3 * r + 1] * S[6 + c] + D[3 * r + 2] * S[12 + c] : 0.0;
    return 1;
}

/* Solve H d = g for symmetric positive definite H (6x6) by Cholesky. */
static int solve6(const double *H, const double *g, double *d)
{
    double Lm[36] = {0};
    for (int j = 0; j < 6; ++j) {
        double s = H[6 * j + j];
        for (int k = 0; k < j; ++k) s -= Lm[6 * j + k] * Lm[6 * j + k];
        if (!(s > 0.0)) return 0;
        Lm[6 * j + j] = sqrt(s);
        for (int i = j + 1; i < 6; ++i) {
            double q = H[6 * i + j];
            for (int k = 0; k < j; ++k) q -= Lm[6 * i + k] * Lm[6 * j + k];
            Lm[6 * i + j] = q / Lm[6 * j + j];
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= Lm[6 * i + k] * y[k];
        y[i] = s / Lm[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= Lm[6 * k + i] * d[k];
        d[i] = s / Lm[6 * i + i];
    }
    return 1;
}

int orc_optimize_pose_pinhole(const orc_params *p, const orc_pinhole *cam, const orc_pose *T0,
                              const orc_keypoints *K, const float *u_right, int M, const float *pos,
                              const int32_t *mp_kp, double *Rt12, int8_t *inlier, double *chi2,
                              double *min_margin, int *rounds_run)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);
    double R[9], t[3];
    for (int i = 0; i < 9; ++i) R[i] = T0->R[i];
    for (int i = 0; i < 3; ++i) t[i] = T0->t[i];
    double margin = INFINITY;
    int rounds = 0;
    for (int m = 0; m < M; ++m) {
        inlier[m] = (mp_kp[m] >= 0 && mp_kp[m] < K->n) ? 1 : -1;
        chi2[m] = -1.0;
    }
    for (int round = 0; round < p->po_rounds; ++round) {
        int n_in = 0;
        for (int m = 0; m < M; ++m) n_in += inlier[m] == 1;
        if (n_in < 3) break;
        int ok = 1;
        for (int it = 0; it < p->po_iters && ok; ++it) {
            double H[36] = {0}, g[6] = {0};
            for (int m = 0; m < M; ++m) {
                if (inlier[m] != 1) continue;
                const int k = mp_kp[m];
                const int oct = K->oct[k];
                const double s = (oct >= 0 && oct < p->nlevels) ? (double)sc[oct] : 1.0;
                const double w = 1.0 / (s * s);
                const int stereo = u_right != NULL && u_right[k] >= 0.0f;
                const double obs[3] = {K->x[k], K->y[k], stereo ? (double)u_right[k] : 0.0};
                double e[3], J[18];
                if (!orc_pose_residual(cam, R, t, pos + 4 * m, obs, stereo, e, J)) continue;
                const double c2 = w * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                const double th = stereo ? p->po_chi2_stereo : p->po_chi2_mono;
                const double h = (!p->po_huber || c2 <= th) ? 1.0 : sqrt(th / c2);
                const int rows = stereo ? 3 : 2;
                for (int a = 0; a < 6; ++a) {
                    for (int r = 0; r < rows; ++r) g[a] += h * w * J[6 * r + a] * e[r];
                    for (int b2 = 0; b2 < 6; ++b2)
                        for (int r = 0; r < rows; ++r) H[6 * a + b2] += h * w * J[6 * r + a] * J[6 * r + b2];
                }
            }
            double d[6], Rd[9], V[9];
            if (!solve6(H, g, d)) {
                ok = 0;
                break;
            }
            orc_se3_exp(d, Rd, V);
            double Rn[9], tn[3];
            mat3_mul(Rd, R, Rn);
            for (int i = 0; i < 3; ++i)
                tn[i] = Rd[3 * i] * t[0] + Rd[3 * i + 1] * t[1] + Rd[3 * i + 2] * t[2] +
                        V[3 * i] * d[3] + V[3 * i + 1] * d[4] + V[3 * i + 2] * d[5];
            memcpy(R, Rn, sizeof(R));
            memcpy(t, tn, sizeof(t));
        }
        ++rounds;
        /* classify every observation at the new pose */
        for (int m = 0; m < M; ++m) {
            if (inlier[m] < 0) continue;
            const int k = mp_kp[m];
            const int oct = K->oct[k];
            const double s = (oct >= 0 && oct < p->nlevels) ? (double)sc[oct] : 1.0;
            const int stereo = u_right != NULL && u_right[k] >= 0.0f;
            const double obs[3] = {K->x[k], K->y[k], stereo ? (double)u_right[k] : 0.0};
            const double th = stereo ? p->po_chi2_stereo : p->po_chi2_mono;
            double e[3], J[18];
            if (!orc_pose_residual(cam, R, t, pos + 4 * m, obs, stereo, e, J)) {
                inlier[m] = 0;
                chi2[m] = INFINITY;
                continue;
            }
            const double c2 = (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) / (s * s);
            chi2[m] = c2;
            inlier[m] = c2 > th ? 0 : 1;
            const double mg = fabs(c2 - th) / th;
            if (mg < margin) margin = mg;
        }
        if (!ok) break;
    }
    for (int i = 0; i < 9; ++i) Rt12[i] = R[i];
    for (int i = 0; i < 3; ++i) Rt12[9 + i] = t[i];
    int n_in = 0;
    for (int m = 0; m < M; ++m) n_in += inlier[m] == 1;
    if (min_margin) *min_margin = margin;
    if (rounds_run) *rounds_run = rounds;
    return n_in;
}

/* ------------------------------------------------------------------------ */
/* f3: keypoints and descriptors on the pyramid levels.  The paper's ORB     */
/* extraction builds the pyramid, finds keypoints on every level, describes */
/* each one and filters them (section II-A), reusing an existing GPU        */
/* extractor (section IV-B) whose steps it does not give.  The reading      */
/* follows the published methods the name refers to -- the FAST segment     */
/* test (Rosten and Drummond), the intensity-centroid orientation and the   */
/* steered binary tests of ORB (Rublee et al.) -- with these choices:       */
/*  - FAST-9 on the level image: pixel p with intensity I is a corner if 9  */
/*    contiguous pixels of the 16 on the radius-3 Bresenham circle are all  */
/*    brighter than I + t or all darker than I - t; only pixels at least    */
/*    `edge` pixels from every border are tested;                           */
/*  - score: the largest threshold at which p is still a corner, i.e. the   */
/*    best arc's smallest intensity difference minus one;                   */
/*  - non-maximum suppression: a corner is kept unless one of its 8         */
/*    neighbours is a corner with a higher score, or an equal score and an  */
/*    earlier raster position;                                              */
/*  - filtering: per level the first max_kp[l] kept corners in the order    */
/*    (score descending, y, x); the level's slots after them are padding    */
/*    (x = y = -1e9, octave 0, score -1, orientation (1, 0), zero           */
/*    descriptor);                                                          */
/*  - orientation: moments m10 = sum u I, m01 = sum v I over the disk       */
/*    u^2 + v^2 <= 15^2 of the level image; |m| = sqrt(m10^2 + m01^2) in    */
/*    double, rounded to float; cos = m10/|m|, sin = m01/|m| in FP32 ((1,0)  */
/*    when both moments are 0);                                             */
/*  - descriptor: the level smoothed by the 5x5 binomial filter (weights    */
/*    1 4 6 4 1 in each direction, sum 256, rounded half up, borders        */
/*    replicated); test i takes the pattern pair (x1, y1, x2, y2), rotates   */
/*    each point by the orientation in FP32 (u = round(c x - s y),          */
/*    v = round(s x + c y), products and difference rounded separately) and */
/*    sets bit i (bit i % 8 of byte i / 8) if S(p1) < S(p2);                */
/*  - keypoint coordinates in level-0 pixels: x0 = x_l * scale[l] (FP32).    */
/* ------------------------------------------------------------------------ */
static const int fast_circle[16][2] = {
    {0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0}, {3, 1}, {2, 2}, {1, 3},
    {0, 3}, {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

/* score of pixel (x, y) if it passes the segment test at threshold t, else -1 */
int orc_fast_score(const uint8_t *img, int pitch, int x, int y, int t)
{
    const int c = img[(size_t)y * pitch + x];
    int d[16];
    for (int i = 0; i < 16; ++i)
        d[i] = img[(size_t)(y + fast_circle[i][1]) * pitch + (x + fast_circle[i][0])] - c;
    int best = -1000;
    for (int start = 0; start < 16; ++start) {
        int lo_b = 1000, lo_d = 1000;       /* smallest brighter / darker difference over the arc */
        for (int k = 0; k < 9; ++k) {
            const int v = d[(start + k) % 16];
            if (v < lo_b) lo_b = v;
            if (-v < lo_d) lo_d = -v;
        }
        if (lo_b > best) best = lo_b;
        if (lo_d > best) best = lo_d;
    }
    /* a corner at t iff the best arc's smallest difference exceeds t */
    return best > t ? best - 1 : -1;
}

void orc_smooth_level(const uint8_t *src, int w, int h, int pitch, uint8_t *dst)
{
    static const int wt[5] = {1, 4, 6, 4, 1};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int acc = 0;
            for (int j = -2; j <= 2; ++j) {
                int yy = y + j;
                yy = yy < 0 ? 0 : (yy > h - 1 ? h - 1 : yy);
                for (int i = -2; i <= 2; ++i) {
                    int xx = x + i;
                    xx = xx < 0 ? 0 : (xx > w - 1 ? w - 1 : xx);
                    acc += wt[j + 2] * wt[i + 2] * src[(size_t)yy * pitch + xx];
                }
            }
            dst[(size_t)y * w + x] = (uint8_t)((acc + 128) >> 8);
        }
}

void orc_orientation(const uint8_t *img, int pitch, int x, int y, float *cs2)
{
    long long m10 = 0, m01 = 0;
    for (int v = -15; v <= 15; ++v)
        for (int u = -15; u <= 15; ++u) {
            if (u * u + v * v > 15 * 15) continue;
            const int I = img[(size_t)(y + v) * pitch + (x + u)];
            m10 += (long long)u * I;
            m01 += (long long)v * I;
        }
    if (m10 == 0 && m01 == 0) {
        cs2[0] = 1.0f;
        cs2[1] = 0.0f;
        return;
    }
    const double n2 = (double)m10 * (double)m10 + (double)m01 * (double)m01;
    const float nm = (float)sqrt(n2);
    cs2[0] = (float)m10 / nm;
    cs2[1] = (float)m01 / nm;
}

void orc_describe(const uint8_t *smooth, int pitch, int x, int y, const float *cs2, const int8_t *pattern,
                  uint8_t *desc32)
{
    const float c = cs2[0], s = cs2[1];
    memset(desc32, 0, 32);
    for (int i = 0; i < 256; ++i) {
        int val[2];
        for (int q = 0; q < 2; ++q) {
            const float px = (float)pattern[4 * i + 2 * q], py = (float)pattern[4 * i + 2 * q + 1];
            const float a = c * px, b = s * py, e = s * px, f = c * py;
            const int u = (int)roundf(a - b);
            const int v = (int)roundf(e + f);
            val[q] = smooth[(size_t)(y + v) * pitch + (x + u)];
        }
        if (val[0] < val[1]) desc32[i >> 3] |= (uint8_t)(1u << (i & 7));
    }
}

typedef struct {
    int score, x, y;
} orc_corner;

/* (score descending, y, x) */
static int corner_before(const orc_corner *a, const orc_corner *b)
{
    if (a->score != b->score) return a->score > b->score;
    if (a->y != b->y) return a->y < b->y;
    return a->x < b->x;
}

int orc_extract_orb(const orc_params *p, const orc_pyramid *pyr, const orc_orb_params *op,
                    float *x, float *y, int8_t *oct, int32_t *score, float *cs, uint8_t *desc,
                    int32_t *n_level)
{
    float sc[ORC_MAX_LEVELS], isc[ORC_MAX_LEVELS];
    orc_scale_table(p->nlevels, p->scale_factor, sc, isc);
    int slot = 0, total = 0;
    for (int l = 0; l < p->nlevels; ++l) {
        const uint8_t *img = pyr->data[l];
        const int w = pyr->width[l], h = pyr->height[l], pitch = pyr->pitch[l];
        const int e = op->edge;
        /* scores of every tested pixel (-1: not a corner or not tested) */
        int *sco = (int *)malloc(sizeof(int) * (size_t)w * (size_t)h);
        for (int i = 0; i < w * h; ++i) sco[i] = -1;
        for (int yy = e; yy < h - e; ++yy)
            for (int xx = e; xx < w - e; ++xx) sco[yy * w + xx] = orc_fast_score(img, pitch, xx, yy, op->fast_th);
        /* non-maximum suppression, then the kept corners in the filtering order */
        orc_corner *kept = (orc_corner *)malloc(sizeof(orc_corner) * ((size_t)w * h + 1));
        int nk = 0;
        for (int yy = e; yy < h - e; ++yy)
            for (int xx = e; xx < w - e; ++xx) {
                const int sp = sco[yy * w + xx];
                if (sp < 0) continue;
                int keep = 1;
                for (int dy = -1; dy <= 1 && keep; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy) continue;
                        const int qx = xx + dx, qy = yy + dy;
                        if (qx < 0 || qy < 0 || qx >= w || qy >= h) continue;
                        const int sq = sco[qy * w + qx];
                        if (sq < 0) continue;
                        const int earlier = qy < yy || (qy == yy && qx < xx);
                        if (sq > sp || (sq == sp && earlier)) {
                            keep = 0;
                            break;
                        }
                    }
                if (keep) kept[nk++] = (orc_corner){sp, xx, yy};
            }
        /* insertion sort by (score desc, y, x); levels hold a few thousand */
        for (int i = 1; i < nk; ++i) {
            orc_corner v = kept[i];
            int j = i - 1;
            while (j >= 0 && corner_before(&v, &kept[j])) {
                kept[j + 1] = kept[j];
                --j;
            }
            kept[j + 1] = v;
        }
        const int cap = op->max_kp[l];
        const int n = nk < cap ? nk : cap;
        uint8_t *sm = (uint8_t *)malloc((size_t)w * h);
        orc_smooth_level(img, w, h, pitch, sm);
        for (int i = 0; i < cap; ++i) {
            const int k = slot + i;
            if (i < n) {
                const orc_corner *c = &kept[i];
                x[k] = (float)c->x * sc[l];
                y[k] = (float)c->y * sc[l];
                oct[k] = (int8_t)l;
                score[k] = c->score;
                orc_orientation(img, pitch, c->x, c->y, cs + 2 * k);
                orc_describe(sm, w, c->x, c->y, cs + 2 * k, op->pattern, desc + 32 * k);
            } else {
                x[k] = y[k] = -1.0e9f;
                oct[k] = 0;
                score[k] = -1;
                cs[2 * k] = 1.0f;
                cs[2 * k + 1] = 0.0f;
                memset(desc + 32 * k, 0, 32);
            }
        }
        n_level[l] = n;
        total += n;
        slot += cap;
        free(sm);
        free(kept);
        free(sco);
    }
    n_level[p->nlevels] = total;
    return slot;
}
