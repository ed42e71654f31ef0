"""Comparison of CUDA-path results with the FP64 oracle (test helper).

Tolerances (FP32 storage): integers and flags bit-exact; maps
|gpu - ref| <= 1e-5 |ref| + 1e-10; projected coordinates within
1e-3 px * (1 + r^2), r = distance of the point from the principal point in
focal lengths -- Eq. 6 divides by d_z, so FP64 rounding of the pose inputs
is amplified by (1 + r^2) for directions far from the optical axis (1e-3 px
flat for directions near the axis).  16-bit storage adds the format's
rounding: 2^-8 (bf16) / 2^-11 (fp16) relative, plus fp16's subnormal step.
"""
import numpy as np

import oracle as O

MAP_RTOL, MAP_ATOL = 1e-5, 1e-10
STORAGE_RTOL = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
STORAGE_ATOL = {"f32": 0.0, "bf16": 0.0, "f16": 2.0 ** -25}
INT_FIELDS = ("frame_index", "status", "n_valid", "valid_mask", "focus_valid",
              "focus_px_x", "focus_px_y")


def coord_tol(u, v, intr):
    fx, fy, cx, cy = intr
    r2 = ((np.asarray(u) - cx) / fx) ** 2 + ((np.asarray(v) - cy) / fy) ** 2
    return 1e-3 * (1.0 + r2)


def map_tol(ref, storage="f32", divisor=None):
    """Per-pixel bound.  ``divisor`` (the FP64 map maximum) marks a map divided
    by its own maximum: the quotient carries the bound of the numerator and of
    the divisor, one FP32 division rounding, and for 16-bit storage a second
    rounding; absolute terms scale by 1 / divisor."""
    if divisor is None:
        return (MAP_RTOL + STORAGE_RTOL[storage]) * np.abs(ref) + MAP_ATOL + STORAGE_ATOL[storage]
    rtol = 2 * MAP_RTOL + 2.0 ** -24 + 2 * STORAGE_RTOL[storage]
    atol = (MAP_ATOL + STORAGE_ATOL[storage]) / divisor + STORAGE_ATOL[storage]
    return rtol * np.abs(ref) + atol


def check_frame(info, pts, ref_info, ref_pts, intr, where=""):
    """Bit-exact integers, coordinates within coord_tol, spreads within 1e-9."""
    for k in INT_FIELDS:
        assert int(info[k]) == int(ref_info[k]), f"{where} {k}: {info[k]} != {ref_info[k]}"
    if ref_info["focus_valid"]:
        t = coord_tol(ref_info["focus_u"], ref_info["focus_v"], intr)
        assert abs(info["focus_u"] - ref_info["focus_u"]) <= t, where
        assert abs(info["focus_v"] - ref_info["focus_v"]) <= t, where
    if pts is not None:
        valid = ref_pts.valid
        assert np.array_equal(pts["valid"].astype(bool), valid), where
        t = coord_tol(ref_pts.u[valid], ref_pts.v[valid], intr)
        assert np.all(np.abs(pts["u"][valid] - ref_pts.u[valid]) <= t), where
        assert np.all(np.abs(pts["v"][valid] - ref_pts.v[valid]) <= t), where
        np.testing.assert_allclose(pts["sigma"][valid], ref_pts.sigma[valid], rtol=1e-9, err_msg=where)
        np.testing.assert_allclose(pts["s"][valid], ref_pts.s[valid], rtol=1e-9, err_msg=where)


def check_argmax(info, M_ref, n_valid, storage="f32", where=""):
    """The GPU argmax is a maximiser of the FP64 map up to the map tolerance."""
    if n_valid == 0:
        assert info["argmax_x"] == -1 and info["argmax_y"] == -1 and info["map_max"] == 0.0, where
        return
    x, y = int(info["argmax_x"]), int(info["argmax_y"])
    mx = M_ref.max()
    assert 0 <= x < M_ref.shape[1] and 0 <= y < M_ref.shape[0], where
    assert M_ref[y, x] >= mx - (2 * MAP_RTOL * mx + MAP_ATOL), where
    assert abs(float(info["map_max"]) - mx) <= MAP_RTOL * mx + MAP_ATOL, where


def check_map(got, ref, storage="f32", where="", divisor=None):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    tol = map_tol(ref, storage, divisor)
    bad = err > tol
    if bad.any():
        i = np.unravel_index(np.argmax(err - tol), err.shape)
        raise AssertionError(f"{where}: {int(bad.sum())} pixels out of tolerance; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r}")
    return float(err.max()), float((err / np.maximum(np.abs(ref), 1e-30))[ref > 1e-6].max(initial=0))
