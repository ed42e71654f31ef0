"""Pins of the oracle's sliding-batch ingestion and gravity-locked anchoring (Section 2.2)."""
import math

import numpy as np
import pytest

import oracle as O
from synth import WalkerSpec, walk
from tests.posegen import rot_x, rot_y


def _G(yaw, t, pitch=0.0, roll=0.0):
    """Local-to-world rigid transform of one batch's coordinate frame."""
    G = np.eye(4)
    rz = np.array([[math.cos(roll), -math.sin(roll), 0], [math.sin(roll), math.cos(roll), 0],
                   [0, 0, 1]])
    G[:3, :3] = rot_y(yaw) @ rot_x(pitch) @ rz
    G[:3, 3] = t
    return G


def _batches(world, L, Ov, Gs):
    """Split world poses into batches of L sharing Ov frames, each in its own frame."""
    out, start, b = [], 0, 0
    while True:
        hi = min(start + L, len(world))
        out.append(np.stack([(O.to4x4(world[k]) @ Gs[b])[:3] for k in range(start, hi)]))
        if hi == len(world):
            return out
        start = hi - Ov
        b += 1


def test_anchoring_recovers_yaw_and_translation():
    world = walk(WalkerSpec(n_frames=100, seed=5, turns=True)).poses_w2c
    rng = np.random.default_rng(1)
    Gs = [np.eye(4)] + [_G(rng.uniform(-3, 3), rng.normal(size=3) * 20) for _ in range(20)]
    L, Ov = 20, 4
    p = O.Params(64, 48, window=8, smooth_len=5, pose_frame=O.POSES_BATCH_LOCAL, overlap=Ov)
    st = O.OracleStream(p)
    emitted = [st.push(b, None, (50.0, 50.0, 32.0, 24.0)) for b in _batches(world, L, Ov, Gs)]
    assert emitted[0] == L and all(e == L - Ov for e in emitted[1:-1])
    assert st.n_emitted == 100
    got = np.stack(st.world)
    np.testing.assert_allclose(got, world, rtol=0, atol=1e-10)


def test_gravity_lock_drops_pitch_and_roll():
    world = walk(WalkerSpec(n_frames=40, seed=6)).poses_w2c
    Gs = [np.eye(4), _G(0.4, [3.0, 0.5, -2.0], pitch=0.2, roll=-0.1)]
    p = O.Params(64, 48, window=8, smooth_len=5, pose_frame=O.POSES_BATCH_LOCAL, overlap=3)
    b0, b1 = _batches(world, 25, 3, Gs)
    st = O.OracleStream(p)
    st.push(b0, None, (50.0, 50.0, 32.0, 24.0))
    H = O.anchor_transform(st.world[-1], b1[2])
    # the recovered rotation is a pure yaw about the gravity (y) axis
    R = H[:3, :3]
    assert R[1, 1] == 1.0 and R[0, 1] == R[1, 0] == R[1, 2] == R[2, 1] == 0.0
    assert abs(R[0, 0] * R[2, 2] - R[0, 2] * R[2, 0] - 1.0) < 1e-15
    # ... so the injected pitch/roll survives in the emitted poses ...
    st.push(b1, None, (50.0, 50.0, 32.0, 24.0))
    assert np.max(np.abs(np.stack(st.world[25:]) - world[25:])) > 1e-2
    # ... while the anchor's camera centre lands exactly on its world position
    ca = O.camera_centre(world[24])
    Tl = O.to4x4(b1[2]) @ np.linalg.inv(H)
    np.testing.assert_allclose(O.camera_centre(Tl[:3]), ca, atol=1e-10)


def test_pure_yaw_recovered_exactly_when_no_tilt():
    Ta = np.concatenate([rot_y(0.3) @ rot_x(0.1), np.array([[1.0], [2.0], [3.0]])], 1)
    G = _G(-1.2, [4.0, -1.0, 2.5])
    La = (O.to4x4(Ta) @ G)[:3]
    H = O.anchor_transform(Ta, La)
    np.testing.assert_allclose(H, G, atol=1e-12)


def test_overlap_must_leave_new_frames():
    p = O.Params(64, 48, pose_frame=O.POSES_BATCH_LOCAL, overlap=5)
    st = O.OracleStream(p)
    poses = walk(WalkerSpec(n_frames=10, seed=1)).poses_w2c
    assert st.push(poses[:5], None, (50.0, 50.0, 32.0, 24.0)) == 5   # first batch: all
    with pytest.raises(ValueError):
        st.push(poses[:5], None, (50.0, 50.0, 32.0, 24.0))


def test_bad_anchor_marks_whole_batch_bad():
    world = walk(WalkerSpec(n_frames=30, seed=7)).poses_w2c
    p = O.Params(64, 48, window=4, smooth_len=3, pose_frame=O.POSES_BATCH_LOCAL, overlap=2)
    st = O.OracleStream(p)
    st.push(world[:15], None, (50.0, 50.0, 32.0, 24.0))
    b1 = world[13:].copy()
    b1[1, 0, 0] = 2.0        # the anchor (last shared frame) is not rigid
    st.push(b1, None, (50.0, 50.0, 32.0, 24.0))
    assert not any(st.bad[:15]) and all(st.bad[15:])
