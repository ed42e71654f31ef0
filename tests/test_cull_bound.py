"""The bound behind the map kernels' point culling (Eq. 7).

The kernels drop a point from a rectangle of pixels (a unit, or one warp's
strip of it) when the product of its largest column factor and its largest
row factor over the rectangle, times 1/Z, is below 2^-40; those factors are
taken at the rectangle's pixel nearest to the point, coordinate by
coordinate.  This file checks, by brute force in FP64, that this product is
the point's largest contribution to any pixel of the rectangle, and that the
at most 32 points dropped from a pixel stay inside the absolute map
tolerance.
"""
import numpy as np
import pytest

from tests import parity

CULL = 2.0 ** -40


def nearest_peak(u, v, sigma, inv_n, x0, x1, y0, y1):
    xn = min(max(np.rint(u), x0), x1)
    yn = min(max(np.rint(v), y0), y1)
    c = 1.0 / (2.0 * sigma * sigma)
    return np.exp(-(xn - u) ** 2 * c) * np.exp(-(yn - v) ** 2 * c) * inv_n


def brute_peak(u, v, sigma, inv_n, x0, x1, y0, y1):
    X = np.arange(x0, x1 + 1, dtype=np.float64)[None, :]
    Y = np.arange(y0, y1 + 1, dtype=np.float64)[:, None]
    return (np.exp(-((X - u) ** 2 + (Y - v) ** 2) / (2.0 * sigma * sigma)) * inv_n).max()


@pytest.mark.parametrize("seed", range(4))
def test_nearest_pixel_factors_bound_every_pixel(seed):
    rng = np.random.default_rng(seed)
    for _ in range(300):
        x0, y0 = (int(t) for t in rng.integers(0, 2000, 2))
        x1, y1 = x0 + int(rng.integers(0, 130)), y0 + int(rng.integers(0, 130))
        # points inside, beside and far from the rectangle, half-integer ties included
        u = x0 + rng.uniform(-400, (x1 - x0) + 400)
        v = y0 + rng.uniform(-400, (y1 - y0) + 400)
        if rng.random() < 0.2:
            u = np.floor(u) + 0.5
        sigma = rng.uniform(2.0, 200.0)
        inv_n = 1.0 / int(rng.integers(1, 33))
        near = nearest_peak(u, v, sigma, inv_n, x0, x1, y0, y1)
        brute = brute_peak(u, v, sigma, inv_n, x0, x1, y0, y1)
        assert brute <= near * (1 + 1e-12) and near <= brute * (1 + 1e-12)


def test_dropped_points_stay_inside_the_absolute_tolerance():
    # at most 32 points per window, each contributing below 2^-40 at any pixel
    assert 32 * CULL < parity.MAP_ATOL
    assert 32 * CULL == 2.0 ** -35
