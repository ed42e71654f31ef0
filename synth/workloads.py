"""Named synthetic workloads (sizes, intrinsics, windows, seeds).

* ``small_stream``: one stream, 64 frames of 320x240 at 30 fps, fx=fy=260,
  principal point (160, 120), window 8; FP32 depth.
* ``hd_stream``: one stream, 900 frames of 1920x1080, fx=fy=1500, principal
  point (960, 540), window 16, running turns up to 45 deg/s.
* ``mixed_streams``: many streams with resolutions drawn from 640x480,
  1280x720, 1920x1080 and 3840x2160, lengths 120..1800 frames, windows 8..32
  and fx=fy in [0.7, 1.2] x width (the resolution mix of the paper's dataset,
  Table 1, widened to the sizes phone cameras record).

Large workloads cannot hold one distinct ray-cast depth image per frame in a
reasonable generation time, so each stream renders a ring of depth images at
evenly spaced trajectory times and frame k uses ring entry k mod R.  Depth
content has no effect on the cost of the path.
"""
from dataclasses import dataclass, field

import numpy as np

from .rng import Xoshiro256ss
from .scene import make_scene, render_depth
from .walker import WalkerSpec, walk

RESOLUTIONS = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))


@dataclass
class StreamWorkload:
    name: str
    width: int
    height: int
    n_frames: int
    window: int
    smooth_len: int
    intr: tuple          # (fx, fy, cx, cy)
    spec: WalkerSpec
    n_boxes: int = 20
    ring: int = 0        # 0: one depth image per frame; R > 0: ring of R images
    _traj: object = field(default=None, repr=False)
    _boxes: object = field(default=None, repr=False)
    _ring_cache: dict = field(default_factory=dict, repr=False)

    @property
    def traj(self):
        if self._traj is None:
            self._traj = walk(self.spec)
        return self._traj

    @property
    def boxes(self):
        if self._boxes is None:
            self._boxes = make_scene(self.traj, self.n_boxes, seed=self.spec.seed)
        return self._boxes

    @property
    def poses(self):
        """(n, 3, 4) FP64 world-to-camera poses."""
        return self.traj.poses_w2c

    def K(self):
        return np.array(self.intr, dtype=np.float64)

    def render(self, k, dtype=np.float32):
        """Ray-cast depth of frame k (ignores the ring)."""
        tr = self.traj
        return render_depth(self.boxes, tr.rot_c2w[k], tr.centres[k], self.intr,
                            self.width, self.height, dtype)

    def ring_frame_index(self, k):
        if self.ring <= 0:
            return k
        slot = k % self.ring
        return (slot * self.n_frames) // self.ring

    def depth(self, k, dtype=np.float32):
        """Depth image used for frame k (ring entry when ``ring`` > 0)."""
        src = self.ring_frame_index(k)
        if src not in self._ring_cache:
            self._ring_cache[src] = self.render(src, np.float32)
        return self._ring_cache[src].astype(dtype)

    def depth_stack(self, lo, hi, dtype=np.float32):
        return np.stack([self.depth(k, dtype) for k in range(lo, hi)])


def small_stream(seed=1, n_frames=64, window=8, smooth_len=15):
    spec = WalkerSpec(n_frames=n_frames, seed=seed)
    return StreamWorkload("320x240x64", 320, 240, n_frames, window, smooth_len,
                          (260.0, 260.0, 160.0, 120.0), spec)


def hd_stream(seed=2, n_frames=900, window=16, smooth_len=15, ring=8, accel=0.0):
    """``accel`` > 0 adds forward speed changes of up to that many m/s^2, so
    that ACCEL-mode motion points land in view."""
    spec = WalkerSpec(n_frames=n_frames, seed=seed, turns=True, accel=accel)
    name = f"1920x1080x{n_frames}" + (f"_accel{accel:g}" if accel else "")
    return StreamWorkload(name, 1920, 1080, n_frames, window, smooth_len,
                          (1500.0, 1500.0, 960.0, 540.0), spec, ring=ring)


def mixed_streams(n_streams=64, cfg=4, ring=8, smooth_len=15, max_frames=None, accel=0.0):
    """Seeded mixed-resolution streams; stream s uses seed 1000*cfg + s.
    ``accel`` > 0 gives every walker forward speed changes (see hd_stream)."""
    out = []
    for s in range(n_streams):
        seed = 1000 * cfg + s
        rng = Xoshiro256ss(seed * 2 + 2)
        w, h = rng.choice(RESOLUTIONS)
        n = int(rng.uniform(120, 1801))
        if max_frames is not None:
            n = min(n, max_frames)
        win = int(rng.uniform(8, 33))
        f = rng.uniform(0.7, 1.2) * w
        spec = WalkerSpec(n_frames=n, seed=seed, turns=True, accel=accel)
        out.append(StreamWorkload(f"{w}x{h}x{n}", w, h, n, win, smooth_len,
                                  (f, f, w / 2.0, h / 2.0), spec, ring=ring))
    return out
