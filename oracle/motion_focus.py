"""FP64 CPU oracle of the motion-focus path -- TEST INFRASTRUCTURE ONLY.

This module is the slow, plain reference against which the CUDA path is
checked.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm may import it; the product library never calls it,
and it shares no code with the CUDA path (it imports numpy and the standard
library only).

It follows "Motion Focus Recognition in Fast-Moving Egocentric Video"
(arXiv 2601.07154) step by step, in the paper's order:

* Section 2.2  sliding-batch ingestion with incremental, gravity-locked
               anchoring (yaw + translation only) and emission of the
               non-overlapping frames                       -> ``OracleStream``
* Eq. 1        camera centres from the inverted world-to-camera pose
                                                            -> ``camera_centre``
* Eqs. 2-3     velocity / acceleration by differencing, generalised to a
               K-sample causal least-squares quadratic fit (K=3 is exactly
               p_t - 2 p_{t-1} + p_{t-2})                   -> ``ls_weights``
* Eq. 4        rotation of the motion vector into the current camera n
* Eqs. 5-6     pinhole projection with the real intrinsics, rescaled to the
               map resolution                               -> ``frame_points``
* Eq. 7        N magnitude-scaled Gaussians, normalised    -> ``focus_map``
* Fig. 1/5     motion-guided depth                          -> ``guided_depth``

Readings of points the paper leaves open (all fixed identically in the CUDA
path's specification):

* which N points: the motion vectors of the last W frames i = n-W+1..n, all
  projected into the current frame n (Fig. 4 caption: "to the n-th frame");
* smoothing: a causal least-squares polynomial fit (degree 2, or degree 1 for
  the 2-sample heading case) over the K newest poses ending at i; ACCEL takes
  twice the quadratic coefficient (the acceleration), HEADING the linear
  coefficient (the velocity at the newest sample, the contrast case the
  paper mentions after Eq. 6);
* validity: rho = max_j |p_j - p_n| over the window's good poses; a point is
  valid iff rho > 1e-12 * max_j |p_j|, |d_i| > 1e-9 rho and |d_iz| > 1e-3 |d_i|;
  Eq. 6 is applied literally (the sign of d_z is not used);
* s_i = clamp(|d_i| / mean_valid |d|, s_lo, s_hi), spread sigma_i =
  sigma_rel * fx' * s_i, Z = number of valid points (or, optionally, the map's
  largest value when that is at least 2^-20, so that the map peaks at 1);
* intrinsics compensation (Section 1, "real camera intrinsics as physical
  constraints"): K given at a calibration resolution is rescaled to the map
  resolution with pixel centres at integer coordinates;
* motion-guided depth G = M * min(1, d0 / D) for finite D > 0, else 0;
* poses whose rotation is not orthonormal to 1e-6 (or that are not finite)
  are "bad": a frame with a bad pose is empty, and a point whose K-sample fit
  touches a bad pose is invalid;
* depth alignment across batches (Section 2.2, Fig. 3 caption; optional):
  every batch-local batch after the first gets one scale s_b = s_{b-1} * m,
  m = the lower median of the single-precision ratios D_prev / D_cur over the
  overlap frames' pixels where both depths are finite and > 0 (s_0 = 1; no
  such pixel: m = 1).  The batch's translations are multiplied by s_b before
  anchoring and its depth by s_b in the guided depth, so that batches a
  monocular model returns at different scales share the first batch's.
"""
import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

MODE_ACCEL = 0
MODE_HEADING = 1
POSES_WORLD = 0
POSES_BATCH_LOCAL = 1

FRAME_OK = 0
FRAME_EMPTY = 1
FRAME_BAD_POSE = 2

RIGID_TOL = 1e-6        # max |R R^T - I| for a pose to count as rigid
STATIC_REL = 1e-12      # rho <= STATIC_REL * max|p_j|: the camera did not move
VALID_REL_NORM = 1e-9   # |d_i| must exceed this fraction of rho
VALID_REL_Z = 1e-3      # |d_iz| must exceed this fraction of |d_i|


@dataclass
class Params:
    width: int
    height: int
    window: int = 8             # W = N motion points (1..32)
    smooth_len: int = 15        # K samples of the least-squares fit
    mode: int = MODE_ACCEL
    pose_frame: int = POSES_WORLD
    overlap: int = 0            # O shared frames between batches (batch-local)
    calib_width: int = 0        # resolution the intrinsics refer to (0: same)
    calib_height: int = 0
    sigma_rel: float = 0.1
    s_lo: float = 0.25
    s_hi: float = 4.0
    depth_ref_m: float = 1.0
    normalize: str = "count"    # Z of Eq. 7: "count" (valid points) or "max" (map maximum)
    depth_align: bool = False   # batch-local only: one depth scale per batch (Section 2.2)


# Z = map maximum applies to maps whose count-normalised maximum is at least
# this; a lower maximum means every point lies many sigma outside the image,
# and such a map is left count-normalised.
NORM_FLOOR = 2.0 ** -20


# ---------------------------------------------------------------- Eqs. 2-3 --
def _exact_inverse(mat):
    """Gauss-Jordan inverse of a small matrix of Fractions (exact)."""
    n = len(mat)
    a = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(mat)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        p = a[col][col]
        a[col] = [x / p for x in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [row[n:] for row in a]


def ls_weights_exact(K, mode):
    """Causal least-squares derivative weights as exact rationals.

    The K newest positions of a point's trajectory sit at tau_k = -k
    (k = 0 is the newest).  Fitting p(tau) = c0 + c1 tau + c2 tau^2 by least
    squares gives c = (A^T A)^{-1} A^T q, linear in the samples, so the
    motion vector is d = sum_k w_k q_{i-k} with
        ACCEL:   d = 2 c2 (second derivative), needs K >= 3;
        HEADING: d = c1   (first derivative at the newest sample); with K = 2
                 the fit is a line, c1 = q_i - q_{i-1} (Eq. 2).
    For K = 3 ACCEL this is exactly (1, -2, 1) (Eq. 3).
    """
    if mode == MODE_ACCEL and K < 3:
        raise ValueError("ACCEL needs K >= 3")
    if mode == MODE_HEADING and K < 2:
        raise ValueError("HEADING needs K >= 2")
    deg = 2 if K >= 3 else 1
    taus = [Fraction(-k) for k in range(K)]
    rows = [[t ** e for e in range(deg + 1)] for t in taus]
    normal = [[sum(r[a] * r[b] for r in rows) for b in range(deg + 1)] for a in range(deg + 1)]
    inv = _exact_inverse(normal)
    coeff, factor = (2, 2) if mode == MODE_ACCEL else (1, 1)
    return [factor * sum(inv[coeff][b] * rows[k][b] for b in range(deg + 1)) for k in range(K)]


def ls_weights(K, mode):
    """The exact weights rounded once to FP64 (index k weights q_{i-k})."""
    return np.array([float(w) for w in ls_weights_exact(K, mode)], dtype=np.float64)


# ------------------------------------------------------------------ Eq. 1 --
def to4x4(T34):
    T = np.eye(4)
    T[:3, :4] = T34
    return T


def camera_centre(T34):
    """Eq. 1: p_t = (T^{w->c})^{-1}[0:3, 3], by a general 4x4 inverse."""
    return np.linalg.inv(to4x4(T34))[:3, 3]


def is_rigid(T34):
    T34 = np.asarray(T34, dtype=np.float64)
    if not np.all(np.isfinite(T34)):
        return False
    R = T34[:, :3]
    err = np.max(np.abs(R @ R.T - np.eye(3)))
    return bool(err <= RIGID_TOL)


# ------------------------------------------------------------ Section 2.2 --
def rot_y(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def anchor_transform(T_anchor_world, L_anchor_local):
    """Gravity-locked local-to-world transform H from the shared anchor frame.

    Full rigid alignment: H_full = (T_a)^{-1} L_a maps local coordinates to
    world coordinates (both poses are world-to-camera of the same camera).
    Gravity lock: only the yaw about the world y axis (gravity) is kept --
    R_y(psi) with psi = atan2(R02 - R20, R00 + R22), the rotation about y
    closest to R_H -- and the translation is chosen so that the anchor's
    camera centre lands on its world position.
    """
    Ta = to4x4(T_anchor_world)
    La = to4x4(L_anchor_local)
    Hf = np.linalg.inv(Ta) @ La
    R = Hf[:3, :3]
    psi = math.atan2(R[0, 2] - R[2, 0], R[0, 0] + R[2, 2])
    Ry = rot_y(psi)
    c_world = camera_centre(T_anchor_world)
    c_local = camera_centre(L_anchor_local)
    H = np.eye(4)
    H[:3, :3] = Ry
    H[:3, 3] = c_world - Ry @ c_local
    return H


def depth_scale_ratio(prev, cur):
    """Depth alignment of two batches over their shared frames (Section 2.2,
    Fig. 3): the lower median (sorted[(n-1)//2]) of the ratios prev / cur,
    each an IEEE single-precision quotient, over the pixels where both depths
    are finite and > 0; None when no pixel qualifies."""
    a = np.asarray(prev, dtype=np.float32).ravel()
    b = np.asarray(cur, dtype=np.float32).ravel()
    ok = np.isfinite(a) & np.isfinite(b) & (a > 0) & (b > 0)
    if not ok.any():
        return None
    r = np.sort(np.divide(a[ok], b[ok], dtype=np.float32))
    return float(r[(r.size - 1) // 2])


# -------------------------------------------------------------- Eqs. 5-6 --
def compensated_intrinsics(K, p: Params):
    """Rescale (fx, fy, cx, cy) from the calibration to the map resolution."""
    fx, fy, cx, cy = (float(v) for v in K)
    wc = p.calib_width or p.width
    hc = p.calib_height or p.height
    if wc != p.width:
        sx = p.width / wc
        fx, cx = fx * sx, (cx + 0.5) * sx - 0.5
    if hc != p.height:
        sy = p.height / hc
        fy, cy = fy * sy, (cy + 0.5) * sy - 0.5
    return fx, fy, cx, cy


@dataclass
class FramePoints:
    index: int
    status: int
    u: np.ndarray        # (W,) slot s <-> frame i = n - W + 1 + s
    v: np.ndarray
    sigma: np.ndarray
    s: np.ndarray
    valid: np.ndarray    # (W,) bool
    d_cam: np.ndarray    # (W, 3) motion vectors in camera n

    @property
    def n_valid(self):
        return int(self.valid.sum())

    @property
    def valid_mask(self):
        return int(sum(1 << k for k, ok in enumerate(self.valid) if ok))


def frame_points(world, bad, n, K, p: Params):
    """Motion points of frame n (Eqs. 1-6) from the world poses of frames 0..n.

    ``world[j]`` is the 3x4 world-to-camera pose of emitted frame j and
    ``bad[j]`` flags a pose that failed the rigidity check.
    """
    W, Ks = p.window, p.smooth_len
    w = ls_weights(Ks, p.mode)
    u = np.zeros(W)
    v = np.zeros(W)
    sig = np.zeros(W)
    mag = np.zeros(W)
    valid = np.zeros(W, dtype=bool)
    dcam = np.zeros((W, 3))
    if bad[n]:
        return FramePoints(n, FRAME_BAD_POSE, u, v, sig, mag, valid, dcam)

    fx, fy, cx, cy = compensated_intrinsics(K, p)
    first = max(0, n - W - Ks + 2)
    good = [j for j in range(first, n + 1) if not bad[j]]
    centres = {j: camera_centre(world[j]) for j in good}          # Eq. 1
    pn = centres[n]
    rho = max(float(np.linalg.norm(centres[j] - pn)) for j in good)
    pmax = max(float(np.linalg.norm(centres[j])) for j in good)
    Rn = np.asarray(world[n], dtype=np.float64)[:, :3]             # R_n^{w->c}
    moving = rho > 0.0 and rho > STATIC_REL * pmax

    norms = np.zeros(W)
    for s in range(W):
        i = n - W + 1 + s
        lo = i - Ks + 1
        if not moving or lo < 0 or any(bad[j] for j in range(lo, i + 1)):
            continue
        a_w = np.zeros(3)
        for k in range(Ks):                                         # Eqs. 2-3
            a_w = a_w + w[k] * centres[i - k]
        a_c = Rn @ a_w                                              # Eq. 4
        nd = float(np.linalg.norm(a_c))
        if not (nd > VALID_REL_NORM * rho and abs(a_c[2]) > VALID_REL_Z * nd):
            continue
        valid[s] = True
        dcam[s] = a_c
        norms[s] = nd
        u[s] = cx + fx * a_c[0] / a_c[2]                            # Eq. 6
        v[s] = cy + fy * a_c[1] / a_c[2]
    nv = int(valid.sum())
    if nv:
        mean = float(norms[valid].sum()) / nv
        for s in range(W):
            if valid[s]:
                mag[s] = min(max(norms[s] / mean, p.s_lo), p.s_hi)
                sig[s] = p.sigma_rel * fx * mag[s]
    status = FRAME_OK if nv else FRAME_EMPTY
    return FramePoints(n, status, u, v, sig, mag, valid, dcam)


# ------------------------------------------------------------------ Eq. 7 --
def focus_map(pts: FramePoints, width, height, xs=None, ys=None):
    """Eq. 7 with Z = number of valid points; pixel (x, y) sits at (x, y).

    With ``xs``/``ys`` (1-D arrays of equal length) only those pixels are
    evaluated; otherwise the full height x width map is returned.
    """
    if xs is None:
        X = np.arange(width, dtype=np.float64)[None, :]
        Y = np.arange(height, dtype=np.float64)[:, None]
        out = np.zeros((height, width))
    else:
        X = np.asarray(xs, dtype=np.float64)
        Y = np.asarray(ys, dtype=np.float64)
        out = np.zeros(X.shape)
    nv = pts.n_valid
    if nv == 0:
        return out
    for s in np.nonzero(pts.valid)[0]:
        r2 = (X - pts.u[s]) ** 2 + (Y - pts.v[s]) ** 2
        out = out + np.exp(-r2 / (2.0 * pts.sigma[s] ** 2))
    return out / nv


def guided_depth(M, D, d0):
    """Motion-guided depth: G = M * min(1, d0 / D) for finite D > 0, else 0."""
    D = np.asarray(D, dtype=np.float64)
    ok = np.isfinite(D) & (D > 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        wgt = np.where(ok, np.minimum(1.0, d0 / np.where(ok, D, 1.0)), 0.0)
    return M * wgt


def map_argmax(M, n_valid):
    """(x, y, max) of the map, ties to the lowest linear index; (-1,-1,0) if empty."""
    if n_valid == 0:
        return -1, -1, 0.0
    k = int(np.argmax(M))
    h, w = M.shape
    return k % w, k // w, float(M.flat[k])


def focus_pixel(pts: FramePoints, width, height):
    """Focus = the newest motion point (slot W-1), rounded half-to-even."""
    s = len(pts.valid) - 1
    if not pts.valid[s]:
        return 0, 0.0, 0.0, -1, -1
    u, v = float(pts.u[s]), float(pts.v[s])
    x, y = int(np.rint(u)), int(np.rint(v))
    if not (0 <= x < width and 0 <= y < height):
        x, y = -1, -1
    return 1, u, v, x, y


# ------------------------------------------------------------ Section 2.2 --
class OracleStream:
    """Sliding-batch ingestion (Section 2.2) feeding the per-frame oracle."""

    def __init__(self, p: Params):
        self.p = p
        self.world = []     # world-to-camera 3x4 poses of emitted frames
        self.bad = []
        self.K = []         # intrinsics in force for each emitted frame
        self.depth = []     # depth image of each emitted frame (or None)
        self.scale = []     # depth alignment scale of each emitted frame
        self.pushes = 0
        self.batch_scale = 1.0      # s of the last batch
        self.overlap_depth = None   # that batch's last `overlap` depth planes

    def push(self, poses, depth, K):
        """Ingest one batch of n poses (n,3,4) and depth (n,H,W); returns #emitted."""
        p = self.p
        poses = np.asarray(poses, dtype=np.float64).reshape(-1, 3, 4)
        n = poses.shape[0]
        local = p.pose_frame == POSES_BATCH_LOCAL
        O = p.overlap if (local and self.pushes > 0) else 0
        if n <= O:
            raise ValueError("a batch must hold more frames than the overlap")
        s_b = 1.0
        if local and p.depth_align:
            if self.pushes > 0:
                m = None
                if depth is not None and self.overlap_depth is not None and O > 0:
                    m = depth_scale_ratio(self.overlap_depth, np.asarray(depth)[:O])
                s_b = self.batch_scale * (m if m is not None else 1.0)
            poses = poses.copy()
            poses[:, :, 3] *= s_b       # the batch's translations in the first batch's scale
            self.batch_scale = s_b
            self.overlap_depth = (None if depth is None or p.overlap == 0
                                  else np.asarray(depth)[n - p.overlap:].copy())
        rigid = [is_rigid(T) for T in poses]
        if local and self.pushes > 0:
            a = O - 1
            anchor_bad = self.bad[-1] or not rigid[a]
            H = None if anchor_bad else anchor_transform(self.world[-1], poses[a])
        for k in range(O, n):
            if local and self.pushes > 0:
                if H is None:
                    Tw = poses[k].copy()
                    b = True
                else:
                    Tw = (to4x4(poses[k]) @ np.linalg.inv(H))[:3, :4]
                    b = not rigid[k]
            else:
                Tw = poses[k].copy()
                b = not rigid[k]
            self.world.append(Tw)
            self.bad.append(b)
            self.K.append(np.asarray(K, dtype=np.float64).copy())
            self.depth.append(None if depth is None else depth[k])
            self.scale.append(s_b)
        self.pushes += 1
        return n - O

    @property
    def n_emitted(self):
        return len(self.world)

    def points(self, n):
        return frame_points(self.world, self.bad, n, self.K[n], self.p)

    def frame(self, n, full_maps=True):
        """All outputs of emitted frame n: info dict, points, and maps (FP64)."""
        p = self.p
        pts = self.points(n)
        info = {"frame_index": n, "status": pts.status, "n_valid": pts.n_valid,
                "valid_mask": pts.valid_mask}
        fv, fu, fvv, px, py = focus_pixel(pts, p.width, p.height)
        info.update(focus_valid=fv, focus_u=fu, focus_v=fvv, focus_px_x=px, focus_px_y=py)
        M = G = None
        if full_maps:
            M = focus_map(pts, p.width, p.height)
            if p.normalize == "max" and M.max() >= NORM_FLOOR:
                # Z = the map's largest point sum: the map peaks at exactly 1
                M = M / M.max()
            if self.depth[n] is not None:
                D = self.depth[n] if self.scale[n] == 1.0 else self.scale[n] * np.asarray(
                    self.depth[n], dtype=np.float64)
                G = guided_depth(M, D, p.depth_ref_m)
            ax, ay, mx = map_argmax(M, pts.n_valid)
            info.update(argmax_x=ax, argmax_y=ay, map_max=mx)
        return info, pts, M, G
