"""Hand-built camera trajectories for closed-form tests (input construction only)."""
import math

import numpy as np


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def w2c(r_c2w, centre):
    """World-to-camera 3x4 pose of a camera with rotation r_c2w at centre."""
    r = np.asarray(r_c2w, dtype=np.float64).T
    out = np.zeros((3, 4))
    out[:, :3] = r
    out[:, 3] = -(r @ np.asarray(centre, dtype=np.float64))
    return out


def trajectory(centres, rots=None):
    n = len(centres)
    if rots is None:
        rots = [np.eye(3)] * n
    return np.stack([w2c(rots[k], centres[k]) for k in range(n)])
