"""Synthetic scene (ground plane + axis-aligned boxes) and its ray-cast z-depth.

Stands in for the per-frame depth maps that the paper takes from its
depth/pose foundation model (Section 2.2): a ground plane 1.6 m below the
starting eye height and seeded boxes standing on it along the walker's path.
Depth is the z-depth (camera-frame z) of the first surface hit along the ray
through each pixel centre; rays that hit nothing within 200 m get 0, the
"invalid depth" value.
"""
import math
from dataclasses import dataclass

import numpy as np

from .rng import Xoshiro256ss

GROUND_Y = 1.6
MAX_RANGE = 200.0


@dataclass
class Box:
    lo: np.ndarray  # (3,) min corner
    hi: np.ndarray  # (3,) max corner


def make_scene(traj, n_boxes=20, seed=1):
    """Boxes at arc length U[3, L+10] m along the body path, lateral U[-3, 3] m."""
    rng = Xoshiro256ss(seed * 2 + 1)
    length = traj.spec.speed * traj.spec.n_frames / traj.spec.fps
    boxes = []
    for _ in range(n_boxes):
        s = rng.uniform(3.0, length + 10.0)
        off = rng.uniform(-3.0, 3.0)
        w = rng.uniform(0.3, 1.2)
        d = rng.uniform(0.3, 1.2)
        h = rng.uniform(0.5, 2.5)
        pos, psi = traj.path_at_arc(s)
        right = np.array([math.cos(psi), 0.0, -math.sin(psi)])
        cx, _, cz = pos + off * right
        boxes.append(Box(np.array([cx - w / 2, GROUND_Y - h, cz - d / 2]),
                         np.array([cx + w / 2, GROUND_Y, cz + d / 2])))
    return boxes


def _pixel_rays(width, height, fx, fy, cx, cy, r_c2w, x0, x1, y0, y1):
    xs = (np.arange(x0, x1, dtype=np.float64) - cx) / fx
    ys = (np.arange(y0, y1, dtype=np.float64) - cy) / fy
    dc = np.empty((y1 - y0, x1 - x0, 3))
    dc[..., 0] = xs[None, :]
    dc[..., 1] = ys[:, None]
    dc[..., 2] = 1.0
    return dc @ r_c2w.T  # world directions; camera z component is 1


def _box_rect(box, r_c2w, centre, fx, fy, cx, cy, width, height):
    """Pixel rectangle covering the box, or None when it is behind the camera."""
    corners = np.array([[box.lo[0] if i & 1 == 0 else box.hi[0],
                         box.lo[1] if i & 2 == 0 else box.hi[1],
                         box.lo[2] if i & 4 == 0 else box.hi[2]] for i in range(8)])
    pc = (corners - centre) @ r_c2w  # camera coordinates
    z = pc[:, 2]
    if np.all(z <= 0.0):
        return None
    if np.any(z <= 1e-3):
        return (0, width, 0, height)
    u = cx + fx * pc[:, 0] / z
    v = cy + fy * pc[:, 1] / z
    x0 = max(0, int(math.floor(u.min())) - 1)
    x1 = min(width, int(math.ceil(u.max())) + 2)
    y0 = max(0, int(math.floor(v.min())) - 1)
    y1 = min(height, int(math.ceil(v.max())) + 2)
    if x0 >= x1 or y0 >= y1:
        return None
    return (x0, x1, y0, y1)


def render_depth(boxes, r_c2w, centre, intr, width, height, dtype=np.float32):
    """Ray-cast z-depth image (height x width) for one camera."""
    fx, fy, cx, cy = intr
    depth = np.full((height, width), np.inf)
    dw = _pixel_rays(width, height, fx, fy, cx, cy, r_c2w, 0, width, 0, height)
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = (GROUND_Y - centre[1]) / dw[..., 1]
        depth = np.where((dw[..., 1] > 0) & (tg > 0), tg, np.inf)
        for box in boxes:
            rect = _box_rect(box, r_c2w, centre, fx, fy, cx, cy, width, height)
            if rect is None:
                continue
            x0, x1, y0, y1 = rect
            d = dw[y0:y1, x0:x1]
            t1 = (box.lo - centre) / d
            t2 = (box.hi - centre) / d
            tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
            hit = (tmin <= tmax) & (tmax > 0)
            t = np.where(tmin > 0, tmin, tmax)
            sub = depth[y0:y1, x0:x1]
            depth[y0:y1, x0:x1] = np.where(hit & (t < sub), t, sub)
    depth = np.where(depth <= MAX_RANGE, depth, 0.0)
    return depth.astype(dtype)
