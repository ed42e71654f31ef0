"""Synthetic walking-subject camera trajectories.

World frame: x right, y down (gravity), z forward; the camera starts at the
origin looking along +z.  The body moves at constant speed along its heading
psi_body (rotation about the world y axis).  The head adds a yaw sway and a
pitch bob on top of the body heading, and the "measured" pose gets iid
position noise and a small random rotation, as a pose estimator would report
it (Section 2.2 takes poses from a foundation model; Section 2.1 describes
handheld walking, scooter and biking capture at 30/60 fps).

Poses are returned as world-to-camera 3x4 matrices [R | t] (row-major, FP64),
the form in which the method consumes them (Section 2.3).
"""
import math
from dataclasses import dataclass

import numpy as np

from .rng import Xoshiro256ss


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rot_axis_angle(w):
    """Rotation matrix of the axis-angle vector w (Rodrigues)."""
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.eye(3)
    k = np.asarray(w, dtype=np.float64) / th
    kx = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(th) * kx + (1.0 - math.cos(th)) * (kx @ kx)


@dataclass
class WalkerSpec:
    n_frames: int
    fps: float = 30.0
    speed: float = 1.4            # m/s along the body heading
    sway_deg: float = 10.0        # head yaw sway amplitude
    sway_hz: float = 0.5
    bob_deg: float = 3.0          # pitch bob amplitude
    bob_hz: float = 2.0
    sigma_t: float = 0.01         # position noise per axis, metres
    sigma_r_deg: float = 0.5      # rotation noise per axis (axis-angle), degrees
    turns: bool = False           # piecewise-constant body yaw rate
    turn_rate_deg: float = 45.0   # |yaw rate| bound for turns
    turn_seg_s: tuple = (1.0, 3.0)
    climb: float = 0.0            # vertical speed in m/s (negative y is up)
    accel: float = 0.0            # forward acceleration magnitude, m/s^2 (0: constant speed)
    accel_seg_s: tuple = (1.0, 2.5)
    speed_range: tuple = (0.5, 3.0)
    seed: int = 1


@dataclass
class Trajectory:
    poses_w2c: np.ndarray   # (n, 3, 4) world-to-camera, FP64
    rot_c2w: np.ndarray     # (n, 3, 3) camera-to-world rotation (noisy)
    centres: np.ndarray     # (n, 3) camera centres in world (noisy)
    body_pos: np.ndarray    # (n, 3) noise-free body path
    body_yaw: np.ndarray    # (n,) body heading
    times: np.ndarray       # (n,) seconds
    spec: WalkerSpec

    def path_at_arc(self, s):
        """Noise-free body position and heading at arc length s (extrapolated)."""
        t = s / self.spec.speed
        dt = 1.0 / self.spec.fps
        k = int(t / dt)
        if k >= len(self.times) - 1:
            k = len(self.times) - 1
            psi = self.body_yaw[k]
            base = self.body_pos[k]
            rem = (t - self.times[k]) * self.spec.speed
            return base + rem * np.array([math.sin(psi), 0.0, math.cos(psi)]), psi
        return self.body_pos[k], self.body_yaw[k]


def walk(spec: WalkerSpec) -> Trajectory:
    """Generate a seeded walker trajectory; all draws come from one xoshiro stream."""
    rng = Xoshiro256ss(spec.seed * 2 + 0)
    n = spec.n_frames
    dt = 1.0 / spec.fps
    times = np.arange(n, dtype=np.float64) * dt

    # body yaw rate schedule
    rates = np.zeros(n)
    if spec.turns:
        t0 = 0.0
        total = n * dt
        while t0 < total:
            dur = rng.uniform(*spec.turn_seg_s)
            rate = math.radians(rng.uniform(-spec.turn_rate_deg, spec.turn_rate_deg))
            lo = int(math.ceil(t0 / dt))
            hi = min(n, int(math.ceil((t0 + dur) / dt)))
            rates[lo:hi] = rate
            t0 += dur

    # forward speed: constant, or (accel > 0) speeding up and slowing down in
    # turn, in segments of seeded length and rate (a scooter or a runner
    # changing pace), kept within speed_range.  Its draws come from a stream
    # of their own, so constant-speed walkers are unchanged.
    speeds = np.full(n, spec.speed)
    if spec.accel > 0.0:
        arng = Xoshiro256ss(spec.seed * 2 + (1 << 40))
        acc = np.zeros(n)
        t0, sign = 0.0, 1.0
        while t0 < n * dt:
            dur = arng.uniform(*spec.accel_seg_s)
            a = sign * spec.accel * arng.uniform(0.6, 1.0)
            lo = int(math.ceil(t0 / dt))
            hi = min(n, int(math.ceil((t0 + dur) / dt)))
            acc[lo:hi] = a
            t0 += dur
            sign = -sign
        lo_v, hi_v = spec.speed_range
        for k in range(1, n):
            speeds[k] = min(hi_v, max(lo_v, speeds[k - 1] + acc[k - 1] * dt))

    body_yaw = np.zeros(n)
    body_pos = np.zeros((n, 3))
    for k in range(1, n):
        body_yaw[k] = body_yaw[k - 1] + rates[k - 1] * dt
        psi = body_yaw[k - 1]
        step = speeds[k - 1] * dt
        body_pos[k] = body_pos[k - 1] + np.array(
            [step * math.sin(psi), -spec.climb * dt, step * math.cos(psi)])

    poses = np.zeros((n, 3, 4))
    rc2w = np.zeros((n, 3, 3))
    centres = np.zeros((n, 3))
    sway = math.radians(spec.sway_deg)
    bob = math.radians(spec.bob_deg)
    sr = math.radians(spec.sigma_r_deg)
    for k in range(n):
        t = times[k]
        yaw = body_yaw[k] + sway * math.sin(2.0 * math.pi * spec.sway_hz * t)
        pitch = bob * math.sin(2.0 * math.pi * spec.bob_hz * t)
        noise_p = np.array([rng.normal(0.0, spec.sigma_t) for _ in range(3)])
        noise_w = np.array([rng.normal(0.0, sr) for _ in range(3)])
        r = rot_axis_angle(noise_w) @ rot_y(yaw) @ rot_x(pitch)
        c = body_pos[k] + noise_p
        rc2w[k] = r
        centres[k] = c
        # world-to-camera: rotation R^T, translation -R^T c
        rw = r.T.copy()
        poses[k, :, :3] = rw
        poses[k, :, 3] = -(rw @ c)
    return Trajectory(poses, rc2w, centres, body_pos, body_yaw, times, spec)
