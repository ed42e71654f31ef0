"""Comparison of CUDA-path results with the FP64 oracle (test helper).

Tolerances (FP32 storage): integers and flags bit-exact; maps
|gpu - ref| <= 1e-5 |ref| + 1e-10; projected coordinates of points that
land inside the image within a flat 1e-3 px; coordinates of points outside
it within 1e-3 px * (1 + r^2), r = distance of the point from the principal
point in focal lengths -- Eq. 6 divides by d_z, so FP64 rounding of the pose
inputs is amplified by (1 + r^2) for directions far from the optical axis,
and no FP64 pipeline holds a flat 1e-3 px at a thousand focal lengths.
16-bit storage adds the format's rounding: 2^-8 (bf16) / 2^-11 (fp16)
relative, plus fp16's subnormal step.

Every coordinate comparison is recorded in ``COORD_ERR`` (largest |du|,
|dv| inside and outside the image, and how many points), every map
comparison in ``MAP_ERR`` (largest relative error where the reference
exceeds 1e-6, largest absolute error, pixels compared, per storage); the
test session prints both records at its end.
"""
import numpy as np

import oracle as O

MAP_RTOL, MAP_ATOL = 1e-5, 1e-10
COORD_TOL_PX = 1e-3
STORAGE_RTOL = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
STORAGE_ATOL = {"f32": 0.0, "bf16": 0.0, "f16": 2.0 ** -25}
INT_FIELDS = ("frame_index", "status", "n_valid", "valid_mask", "focus_valid",
              "focus_px_x", "focus_px_y")

# largest coordinate errors seen by this process: {"in_image"|"off_image": [du, dv, count]}
COORD_ERR = {"in_image": [0.0, 0.0, 0], "off_image": [0.0, 0.0, 0]}
# largest map errors seen by this process: {storage[+"/max"]: [rel, abs, pixels]}
MAP_ERR = {}


def in_image(u, v, size):
    """Points whose projection lies on the pixel grid (centres 0..W-1, 0..H-1,
    half a pixel of margin)."""
    width, height = size
    u, v = np.asarray(u), np.asarray(v)
    return (u >= -0.5) & (u <= width - 0.5) & (v >= -0.5) & (v <= height - 0.5)


def coord_tol(u, v, intr, size=None):
    """Flat 1e-3 px inside the image (when its size is given), else
    1e-3 px * (1 + r^2)."""
    fx, fy, cx, cy = intr
    u, v = np.asarray(u, dtype=np.float64), np.asarray(v, dtype=np.float64)
    r2 = ((u - cx) / fx) ** 2 + ((v - cy) / fy) ** 2
    tol = COORD_TOL_PX * (1.0 + r2)
    if size is not None:
        tol = np.where(in_image(u, v, size), COORD_TOL_PX, tol)
    return tol


def _record(du, dv, inside):
    du, dv, inside = np.atleast_1d(du), np.atleast_1d(dv), np.atleast_1d(inside)
    for key, sel in (("in_image", inside), ("off_image", ~inside)):
        if sel.any():
            rec = COORD_ERR[key]
            rec[0] = max(rec[0], float(du[sel].max()))
            rec[1] = max(rec[1], float(dv[sel].max()))
            rec[2] += int(sel.sum())


def check_coords(u, v, ref_u, ref_v, intr, size, where=""):
    """GPU coordinates against the oracle's, recorded in COORD_ERR."""
    ref_u, ref_v = np.asarray(ref_u, dtype=np.float64), np.asarray(ref_v, dtype=np.float64)
    du = np.abs(np.asarray(u, dtype=np.float64) - ref_u)
    dv = np.abs(np.asarray(v, dtype=np.float64) - ref_v)
    inside = in_image(ref_u, ref_v, size) if size is not None else np.zeros(ref_u.shape, bool)
    _record(du, dv, inside)
    t = coord_tol(ref_u, ref_v, intr, size)
    assert np.all(du <= t) and np.all(dv <= t), (
        f"{where}: coordinates off by up to ({du.max():.3g}, {dv.max():.3g}) px")


def check_frame(info, pts, ref_info, ref_pts, intr, where="", size=None):
    """Bit-exact integers, coordinates within coord_tol, spreads within 1e-9.
    ``size`` = (width, height) of the map holds in-image points to the flat
    1e-3 px."""
    for k in INT_FIELDS:
        assert int(info[k]) == int(ref_info[k]), f"{where} {k}: {info[k]} != {ref_info[k]}"
    if ref_info["focus_valid"]:
        check_coords(info["focus_u"], info["focus_v"], ref_info["focus_u"], ref_info["focus_v"],
                     intr, size, where=f"{where} focus")
    if pts is not None:
        valid = ref_pts.valid
        assert np.array_equal(pts["valid"].astype(bool), valid), where
        if valid.any():
            check_coords(pts["u"][valid], pts["v"][valid], ref_pts.u[valid], ref_pts.v[valid],
                         intr, size, where=f"{where} points")
        np.testing.assert_allclose(pts["sigma"][valid], ref_pts.sigma[valid], rtol=1e-9, err_msg=where)
        np.testing.assert_allclose(pts["s"][valid], ref_pts.s[valid], rtol=1e-9, err_msg=where)


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
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(got - ref)
    big = ref > 1e-6
    rec = MAP_ERR.setdefault(storage + ("/max" if divisor is not None else ""), [0.0, 0.0, 0])
    if err.size:
        rec[0] = max(rec[0], float((err[big] / ref[big]).max(initial=0.0)))
        rec[1] = max(rec[1], float(err.max()))
        rec[2] += int(err.size)
    tol = map_tol(ref, storage, divisor)
    bad = err > tol
    if bad.any():
        i = np.unravel_index(np.argmax(err - tol), err.shape)
        raise AssertionError(f"{where}: {int(bad.sum())} pixels out of tolerance; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r}")
    return float(err.max()), float((err / np.maximum(np.abs(ref), 1e-30))[ref > 1e-6].max(initial=0))


def assert_not_vacuous(ref_values, frac, where=""):
    """A sampled comparison means something only where the reference map is
    not (nearly) zero: at least ``frac`` of the sampled reference values must
    exceed 1e-3."""
    ref_values = np.asarray(ref_values)
    got = float((ref_values > 1e-3).mean()) if ref_values.size else 0.0
    assert got >= frac, f"{where}: only {got:.3f} of sampled reference values exceed 1e-3 (need {frac})"
    return got
