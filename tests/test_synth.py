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
    assert all(0.7 * m.width <= m.intr[0] == m.intr[1] <= 1.2 * m.width for m in ms)
    assert all(m.intr[2:] == (m.width / 2.0, m.height / 2.0) for m in ms)
    big = mixed_streams(64)
    assert {(m.width, m.height) for m in big} == {(640, 480), (1280, 720), (1920, 1080), (3840, 2160)}
    assert min(m.window for m in big) <= 10 and max(m.window for m in big) >= 30


def test_walker_follows_its_recipe():
    """30 fps walker at 1.4 m/s, 10 deg / 0.5 Hz yaw sway, 3 deg / 2 Hz pitch
    bob, 1 cm and 0.5 deg pose noise, turns bounded by 45 deg/s."""
    from synth import WalkerSpec, walk
    tr = walk(WalkerSpec(n_frames=600, seed=3, turns=True))
    step = np.linalg.norm(np.diff(tr.body_pos, axis=0), axis=1)
    assert np.allclose(step, 1.4 / 30.0, rtol=1e-12)
    rate = np.abs(np.diff(tr.body_yaw)) * 30.0
    assert rate.max() <= np.radians(45.0) + 1e-12 and rate.max() > np.radians(5.0)
    noise = tr.centres - tr.body_pos
    assert abs(noise.std() - 0.01) < 0.002 and abs(noise.mean()) < 0.002
    # camera yaw about the body heading: sway of 10 deg (+ 0.5 deg noise)
    fwd = tr.rot_c2w[:, :, 2]
    yaw = np.arctan2(fwd[:, 0], fwd[:, 2])
    rel = np.degrees(np.angle(np.exp(1j * (yaw - tr.body_yaw))))
    assert 9.0 < np.abs(rel).max() < 12.5
    # world-to-camera poses invert the camera-to-world ones
    R = tr.poses_w2c[:, :, :3]
    assert np.allclose(R, np.swapaxes(tr.rot_c2w, 1, 2), atol=1e-12)
    assert np.allclose(np.einsum("nij,nj->ni", R, tr.centres) + tr.poses_w2c[:, :, 3], 0.0, atol=1e-12)


def test_scene_boxes_follow_their_recipe():
    """20 boxes, footprint 0.3..1.2 m, height 0.5..2.5 m, standing on the ground."""
    w = hd_stream()
    boxes = w.boxes
    assert len(boxes) == 20
    for b in boxes:
        size = b.hi - b.lo
        assert 0.3 <= size[0] <= 1.2 and 0.3 <= size[2] <= 1.2 and 0.5 <= size[1] <= 2.5
        assert b.hi[1] == 1.6          # the ground plane, 1.6 m below the start (y down)
    assert w.intr == (1500.0, 1500.0, 960.0, 540.0) and w.window == 16 and w.smooth_len == 15
