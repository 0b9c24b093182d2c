"""Shared helpers of the GPU tests: comparisons of library outputs with the
CPU oracle, element by element, with the tolerances stated here.

Tolerances: indices, Hamming distances, SAD shifts and SAD values must be
bit-exact; levels and the projection (u, v, u_right, viewing cosine) are
FP32 in the same operation order on both sides, so they must be bit-exact
too; u_right of stereo within 1e-4 px and depth within 1e-5 relative (the
stated parity bound; both are in fact expected bit-exact).
"""
import numpy as np

TOL_PX = 1e-4
TOL_REL = 1e-5

STEREO_INT = ("best_r", "dist", "sad_shift", "sad_best")
FISHEYE_INT = ("r_idx", "d1", "d2")
SEARCH_INT = ("mp_kp", "mp_d1", "mp_d2", "kp_mp")


def _diff(name, a, b):
    bad = np.nonzero(a != b)[0] if a.ndim == 1 else np.nonzero(np.any(a != b, axis=-1))[0]
    i = bad[:5]
    return f"{name}: {len(bad)} of {len(a)} differ, first at {i.tolist()}: gpu {a[i].tolist()} oracle {b[i].tolist()}"


def assert_stereo_equal(gpu: dict, ref: dict, where: str = ""):
    for k in STEREO_INT:
        assert np.array_equal(gpu[k], ref[k]), where + _diff(k, gpu[k], ref[k])
    for k in ("u_right", "depth"):
        assert np.array_equal(gpu[k] < 0, ref[k] < 0), where + _diff(k + " (<0)", gpu[k] < 0, ref[k] < 0)
    m = ref["u_right"] >= 0
    if m.any():
        assert np.max(np.abs(gpu["u_right"][m] - ref["u_right"][m])) <= TOL_PX, where + "u_right"
        rel = np.abs(gpu["depth"][m] - ref["depth"][m]) / np.abs(ref["depth"][m])
        assert np.max(rel) <= TOL_REL, where + "depth"


def assert_fisheye_equal(gpu: dict, ref: dict, where: str = ""):
    for k in FISHEYE_INT:
        assert np.array_equal(gpu[k], ref[k]), where + _diff(k, gpu[k], ref[k])
    # triangulation: the same FP32 operations in the same order on both sides
    for k in ("fdepth", "xyz"):
        assert np.array_equal(gpu[k].view(np.uint32), ref[k].view(np.uint32)), where + _diff(k, gpu[k], ref[k])


def assert_search_equal(gpu: dict, ref: dict, side: str, ref_side: str | None = None, where: str = ""):
    """gpu keys are suffixed _l/_r; ref keys per oracle function (suffix or none)."""
    sfx = "" if ref_side is None else "_" + ref_side
    lv_g, lv_r = gpu["level_" + side], ref["level" + sfx]
    assert np.array_equal(lv_g, lv_r), where + _diff("level", lv_g, lv_r)
    pg, pr = gpu["proj_" + side], ref["proj" + sfx]
    assert np.array_equal(pg.view(np.uint32), pr.view(np.uint32)), where + _diff("proj", pg, pr)
    for k in SEARCH_INT:
        a, b = gpu[f"{k}_{side}"], ref[k + sfx]
        assert np.array_equal(a, b), where + _diff(k, a, b)


def stereo_view(out: dict) -> dict:
    return {k: out[k] for k in STEREO_INT + ("u_right", "depth")}
