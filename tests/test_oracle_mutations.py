"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle source (on the CPU), builds it, and runs the
oracle pin suite against that copy: the suite has to fail."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ft_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("hamming_short", "i < ORC_DESC_BYTES; ++i) d +=", "i < ORC_DESC_BYTES - 1; ++i) d +="),
    ("band_ceil", "int b = (int)ceilf(y + r);", "int b = (int)floorf(y + r);"),
    ("tie_last_j", "if (d < bestd || (d == bestd && j < bestj)) {", "if (d <= bestd) {"),
    ("octave_window", "R->oct[j] > oct_l + 1", "R->oct[j] > oct_l"),
    ("disparity_sign", "const float u_lo = L->x[i] - disp_hi;", "const float u_lo = L->x[i] + disp_hi;"),
    ("threshold_le", "if (bestd < p->th_stereo)", "if (bestd <= p->th_stereo + 10)"),
    ("centre_right", "int b = IR[(size_t)(vl + dy) * sr + (ur0 + k + dx)] - cR;",
     "int b = IR[(size_t)(vl + dy) * sr + (ur0 + k + dx)] - cL;"),
    ("shift_sign", "(ur0 + k + dx)] - cR;", "(ur0 - k + dx)] - cR;"),
    ("sad_bounds", "ur0 + L + w > wr - 1", "ur0 + w > wr - 1"),
    ("parabola_sign", "(sad_m1 - sad_p1) / (2.0f", "(sad_p1 - sad_m1) / (2.0f"),
    ("parabola_factor", "/ (2.0f * (sad_m1 + sad_p1 - 2.0f * sad_0))", "/ ((sad_m1 + sad_p1 - 2.0f * sad_0))"),
    ("median_index", "const int median = v[n / 2];", "const int median = v[(n - 1) / 2];"),
    ("median_strict", "(float)sad_best[i] >= sad_cut", "(float)sad_best[i] > sad_cut"),
    ("fisheye_overlap", "if (!(R->x[j] >= lap_r0 && R->x[j] <= lap_r1)) continue;", ""),
    ("fisheye_second", "d2[i] = (sj >= 0) ? sd : 256;", "d2[i] = (sj >= 0) ? sd : 255;"),
    ("transpose_R", "Pc[0] = R[0] * P[0] + R[1] * P[1] + R[2] * P[2] + t[0];",
     "Pc[0] = R[0] * P[0] + R[3] * P[1] + R[6] * P[2] + t[0];"),
    ("ur_sign", "const float ur = u - cam->bf * invz;", "const float ur = u + cam->bf * invz;"),
    ("level_table", "if (sc[l] >= ratio) {", "if (sc[l] > ratio * 1.1f) {"),
    ("viewcos_strict", "if (vc < p->view_cos_min) return 0;", "if (vc <= p->view_cos_min) return 0;"),
    ("window_no_radius", "int x0 = (int)floorf((u - min_x - r) * iw);", "int x0 = (int)floorf((u - min_x) * iw);"),
    ("cell_index", "const int c = ix * ORC_GRID_ROWS + iy;", "const int c = iy * ORC_GRID_ROWS + ix;"),
    ("y_test_uses_x", "fabsf(distx) < r && fabsf(disty) < r", "fabsf(distx) < r && fabsf(distx) < r"),
    ("ratio_octave", "(p->ratio_any_octave || oct1 == oct2)", "(p->ratio_any_octave || oct1 != oct2)"),
    ("conflict_max", "if (owner[bk] < 0 || key < owner[bk]) owner[bk] = key;",
     "if (owner[bk] < 0 || key > owner[bk]) owner[bk] = key;"),
    ("stereo_check", "if (er > r) continue;", "if (er > 2.0f * r) continue;"),
    ("kb8_horner", "float poly = cam->k[3];", "float poly = cam->k[0];"),
    ("atan_reduction", "return pi_4 + atan_small", "return pi_4 - atan_small"),
    ("taken_ignored", "if (taken && taken[k]) continue;", ""),
    # fisheye triangulation (next row f1)
    ("tri_centre_sign", "C[i] = -(R_rl[i] * t_rl[0] + R_rl[3 + i] * t_rl[1] + R_rl[6 + i] * t_rl[2]);",
     "C[i] = (R_rl[i] * t_rl[0] + R_rl[3 + i] * t_rl[1] + R_rl[6 + i] * t_rl[2]);"),
    ("tri_rotation_transpose", "dr[i] = R_rl[i] * ray_r[0] + R_rl[3 + i] * ray_r[1] + R_rl[6 + i] * ray_r[2];",
     "dr[i] = R_rl[3 * i] * ray_r[0] + R_rl[3 * i + 1] * ray_r[1] + R_rl[3 * i + 2] * ray_r[2];"),
    ("tri_param_swap", "const float s = dot3(cr, n) / nn;", "const float s = dot3(cl, n) / nn;"),
    ("tri_parallel_guard", "if (!(nn > 1e-10f * (dot3(ray_l, ray_l) * dot3(dr, dr)))) return 0;", ""),
    ("tri_depth_threshold", "return xyz[2] > min_depth;", "return xyz[2] > 0.0f;"),
    ("unproject_fy", "const float my = (v - cam->cy) / cam->fy;", "const float my = (v - cam->cy) / cam->fx;"),
    ("newton_residual_sign", "f = th * poly - thd;", "f = th * poly + thd;"),
    ("newton_no_check", "if (!(fabsf(f) <= 2e-6f && dp > 0.0f", "if (!(fabsf(f) <= 2e10f && dp > -1e30f"),
    ("sine_coefficient", "s = -1.66666672e-01f + t2 * s;", "s = -1.66666672e-02f + t2 * s;"),
    ("cosine_coefficient", "c = -0.5f + t2 * c;", "c = -0.25f + t2 * c;"),
    # search of the last frame's points (next row f2)
    ("last_forward_window", "const int minLevel = motion > 0 ? lv : (motion < 0 ? 0 : lv - 1);",
     "const int minLevel = motion > 0 ? lv - 1 : (motion < 0 ? 0 : lv - 1);"),
    ("last_backward_window", "const int maxLevel = motion > 0 ? p->nlevels - 1 : (motion < 0 ? lv : lv + 1);",
     "const int maxLevel = motion > 0 ? p->nlevels - 1 : (motion < 0 ? lv + 1 : lv + 1);"),
    ("last_radius_octave", "const float r = p->th_last * sc[lv];", "const float r = p->th_last * sc[0];"),
    ("last_motion_sign", "if (-c[2] > b) return -1;", "if (c[2] < b) return -1;"),
    ("last_ratio_added", "if (bd > p->th_search) continue;\n        const int64_t key = ((int64_t)bd << 32) | (int64_t)m;\n        if (owner[bk] < 0 || key < owner[bk]) owner[bk] = key;\n        mp_kp[m] = bk;\n    }\n    for (int k = 0; k < K->n; ++k) kp_mp[k] = (owner[k] < 0) ? -1 : (int32_t)(owner[k] & 0xffffffff);\n    for (int m = 0; m < M; ++m)\n        if (mp_kp[m] >= 0 && kp_mp[mp_kp[m]] != m) mp_kp[m] = -1;\n    free(ky);",
     "if (bd > p->th_search || (float)bd > 0.8f * (float)mp_d2[m]) continue;\n        const int64_t key = ((int64_t)bd << 32) | (int64_t)m;\n        if (owner[bk] < 0 || key < owner[bk]) owner[bk] = key;\n        mp_kp[m] = bk;\n    }\n    for (int k = 0; k < K->n; ++k) kp_mp[k] = (owner[k] < 0) ? -1 : (int32_t)(owner[k] & 0xffffffff);\n    for (int m = 0; m < M; ++m)\n        if (mp_kp[m] >= 0 && kp_mp[mp_kp[m]] != m) mp_kp[m] = -1;\n    free(ky);"),
    ("last_octave_range", "return (lv >= 0 && lv < p->nlevels) ? lv : -1;", "return (lv >= -1 && lv < p->nlevels) ? (lv < 0 ? 0 : lv) : -1;"),
    # image pyramid (next row f3)
    ("pyr_half_pixel", "float xs = ((float)x + 0.5f) * sx - 0.5f;", "float xs = (float)x * sx;"),
    ("pyr_weights_swapped", "const float top = p00 * (1.0f - fx) + p01 * fx;",
     "const float top = p00 * fx + p01 * (1.0f - fx);"),
    ("pyr_no_y_weight", "const float fy = ys - (float)y0;", "const float fy = 0.0f;"),
    ("pyr_size_floor", "w[l] = (int)roundf((float)W / sc[l]);", "w[l] = (int)((float)W / sc[l]);"),
    ("pyr_round_floor", "float v = rintf(top * (1.0f - fy) + bot * fy);", "float v = floorf(top * (1.0f - fy) + bot * fy);"),
    ("pyr_fused_vertical", "float v = rintf(top * (1.0f - fy) + bot * fy);", "float v = rintf(fmaf(top, 1.0f - fy, bot * fy));"),
    # right fisheye camera of the search (T_rw = T_rl T_lw, centre O_right)
    ("right_R_transposed", "Rr[3 * i + j] = R_rl[3 * i + 0] * T->R[0 + j] + R_rl[3 * i + 1] * T->R[3 + j] +\n                            R_rl[3 * i + 2] * T->R[6 + j];",
     "Rr[3 * i + j] = R_rl[0 + i] * T->R[0 + j] + R_rl[3 + i] * T->R[3 + j] +\n                            R_rl[6 + i] * T->R[6 + j];"),
    ("right_t_dropped", "R_rl[3 * i + 2] * T->t[2] + t_rl[i];\n    }\n    for (int m = 0; m < M; ++m) {\n        int lv;",
     "R_rl[3 * i + 2] * T->t[2];\n    }\n    for (int m = 0; m < M; ++m) {\n        int lv;"),
    ("right_centre_is_left", "orc_project_kb8(p, camR, Rr, tr, O_right,", "orc_project_kb8(p, camR, Rr, tr, T->O,"),
    ("last_right_R_transposed",
     "Rr[3 * i + j] = R_rl[3 * i] * T->R[j] + R_rl[3 * i + 1] * T->R[3 + j] + R_rl[3 * i + 2] * T->R[6 + j];",
     "Rr[3 * i + j] = R_rl[i] * T->R[j] + R_rl[3 + i] * T->R[3 + j] + R_rl[6 + i] * T->R[6 + j];"),
    ("last_right_t_dropped",
     "tr[i] = R_rl[3 * i] * T->t[0] + R_rl[3 * i + 1] * T->t[1] + R_rl[3 * i + 2] * T->t[2] + t_rl[i];",
     "tr[i] = R_rl[3 * i] * T->t[0] + R_rl[3 * i + 1] * T->t[1] + R_rl[3 * i + 2] * T->t[2];"),
    # keypoint detection and description (next row f3)
    ("fast_circle_offset", "{0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0},", "{0, -3}, {1, -3}, {2, -2}, {3, -2}, {3, 0},"),
    ("fast_arc_eight", "for (int k = 0; k < 9; ++k) {", "for (int k = 0; k < 8; ++k) {"),
    ("fast_score_offset", "return best > t ? best - 1 : -1;", "return best > t ? best : -1;"),
    ("fast_not_strict", "return best > t ? best - 1 : -1;", "return best >= t ? best - 1 : -1;"),
    ("nms_tie_later", "if (sq > sp || (sq == sp && earlier)) {", "if (sq > sp || (sq == sp && !earlier)) {"),
    ("filter_order_x_first", "if (a->y != b->y) return a->y < b->y;\n    return a->x < b->x;",
     "if (a->x != b->x) return a->x < b->x;\n    return a->y < b->y;"),
    ("smooth_no_rounding", "dst[(size_t)y * w + x] = (uint8_t)((acc + 128) >> 8);", "dst[(size_t)y * w + x] = (uint8_t)(acc >> 8);"),
    ("orientation_radius", "if (u * u + v * v > 15 * 15) continue;", "if (u * u + v * v > 14 * 14) continue;"),
    ("orientation_sign", "cs2[1] = (float)m01 / nm;", "cs2[1] = -(float)m01 / nm;"),
    ("describe_rotation_sign", "const int u = (int)roundf(a - b);", "const int u = (int)roundf(a + b);"),
    ("describe_compare", "if (val[0] < val[1]) desc32", "if (val[0] <= val[1]) desc32"),
    ("keypoint_level_scale", "x[k] = (float)c->x * sc[l];", "x[k] = (float)c->x;"),
    # pose optimization (next row f4)
    ("pose_jacobian_sign", "const double S[18] = {0.0, z, -y, 1.0, 0.0, 0.0,", "const double S[18] = {0.0, -z, y, 1.0, 0.0, 0.0,"),
    ("pose_stereo_bf_sign", "-fx * x * iz2 + bf * iz2};", "-fx * x * iz2 - bf * iz2};"),
    ("pose_weight_not_squared", "const double w = 1.0 / (s * s);", "const double w = 1.0 / s;"),
    ("pose_huber_no_sqrt", "c2 <= th) ? 1.0 : sqrt(th / c2);", "c2 <= th) ? 1.0 : th / c2;"),
    ("pose_right_multiplied", "mat3_mul(Rd, R, Rn);", "mat3_mul(R, Rd, Rn);"),
    ("pose_exp_series_sign", "a = 1.0 - th2 / 6.0;", "a = 1.0 + th2 / 6.0;"),
    ("pose_exp_v_coefficient", "V9[i] = id + b * W[i] + c * W2[i];", "V9[i] = id + a * W[i] + c * W2[i];"),
    ("pose_stereo_threshold", "const double th = stereo ? p->po_chi2_stereo : p->po_chi2_mono;\n            double e[3], J[18];",
     "const double th = p->po_chi2_mono;\n            double e[3], J[18];"),
    ("pose_min_three", "if (n_in < 3) break;", "if (n_in < 2) break;"),
    ("last_view_distance", "        level[m] = (int8_t)last_level(p, last_oct, m);\n        proj[4 * m + 0] = u;",
     "        if (Pc[2] > 8.0f) continue;\n        level[m] = (int8_t)last_level(p, last_oct, m);\n        proj[4 * m + 0] = u;"),
]


def _run_mutant(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name}: text not found"
    mut = src.replace(old, new, 1)
    cdir = os.path.join(tmp, name)
    os.makedirs(cdir)
    cpath = os.path.join(cdir, "ft_oracle.c")
    open(cpath, "w").write(mut)
    hsrc = os.path.join(ROOT, "oracle", "ft_oracle.h")
    open(os.path.join(cdir, "ft_oracle.h"), "w").write(open(hsrc).read())
    so = os.path.join(cdir, "libmut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", so,
                    cpath, "-lm"], check=True)
    env = dict(os.environ, FT_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_stereo.py"),
                        os.path.join(ROOT, "tests", "test_oracle_search.py"),
                        os.path.join(ROOT, "tests", "test_oracle_triangulation.py"),
                        os.path.join(ROOT, "tests", "test_oracle_lastframe.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pyramid.py"),
                        os.path.join(ROOT, "tests", "test_oracle_fisheye_rig.py"),
                        os.path.join(ROOT, "tests", "test_oracle_mirror.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pose.py"),
                        os.path.join(ROOT, "tests", "test_oracle_orb.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            results = list(ex.map(lambda m: _run_mutant(tmp, *m), MUTANTS))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins missed planted mistakes: {survivors}"
