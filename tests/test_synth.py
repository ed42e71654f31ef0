"""The seeded input generators: reproducible, and shaped as the workloads state."""
import numpy as np

from synth import Xoshiro256ss, hd_stream, mixed_streams, small_stream, splitmix64


def test_splitmix64_first_output():
    # published first output of splitmix64 seeded with 0
    assert splitmix64(0)[1] == 0xE220A8397B1DCDAF


def test_xoshiro_deterministic_and_uniform():
    a, b = Xoshiro256ss(42), Xoshiro256ss(42)
    xs = [a.uniform() for _ in range(20000)]
    assert xs[:50] == [b.uniform() for _ in range(50)]
    assert abs(np.mean(xs) - 0.5) < 0.01 and 0.0 <= min(xs) and max(xs) < 1.0
    g = Xoshiro256ss(7)
    zs = np.array([g.normal() for _ in range(20000)])
    assert abs(zs.mean()) < 0.03 and abs(zs.std() - 1.0) < 0.03


def test_workload_shapes():
    w = small_stream()
    assert w.poses.shape == (64, 3, 4)
    d = w.depth(5)
    assert d.shape == (240, 320) and d.dtype == np.float32
    assert np.all(np.isfinite(d)) and d.min() >= 0.0 and 0 < d.max() <= 200.0
    # rigid poses
    R = w.poses[:, :, :3]
    assert np.max(np.abs(R @ np.swapaxes(R, 1, 2) - np.eye(3))) < 1e-12
    h = hd_stream()
    assert h.poses.shape == (900, 3, 4) and (h.width, h.height) == (1920, 1080)
    assert h.ring_frame_index(9) == h.ring_frame_index(1)
    ms = mixed_streams(8)
    assert all((m.width, m.height) in ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))
               for m in ms)
    assert all(120 <= m.n_frames <= 1800 and 8 <= m.window <= 32 for m in ms)
