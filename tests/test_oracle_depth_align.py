"""Pins of the oracle's depth alignment across batches (Section 2.2, Fig. 3):
one scale per batch from the overlap frames' depth ratios, applied to the
batch's translations and depth.  A monocular model returns each batch at its
own scale; the alignment must bring every batch back to the first one's."""
import math

import numpy as np

import oracle as O
from synth import WalkerSpec, walk
from tests.posegen import rot_y

K = (50.0, 50.0, 32.0, 24.0)


def test_ratio_is_the_lower_median_of_single_precision_quotients():
    one = np.ones(4, np.float32)
    assert O.depth_scale_ratio(np.array([4, 1, 3, 2], np.float32), one) == 2.0   # not 2.5
    assert O.depth_scale_ratio(np.array([5, 1, 3], np.float32), np.ones(3)) == 3.0
    # invalid depth on either side is left out
    prev = np.array([np.nan, 0.0, -1.0, np.inf, 3.0, 7.0], np.float32)
    cur = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 0.0], np.float32)
    assert O.depth_scale_ratio(prev, cur) == 3.0
    assert O.depth_scale_ratio(np.zeros(3), np.ones(3)) is None
    # each ratio is the IEEE single-precision quotient, not a double one
    r = O.depth_scale_ratio(np.array([1.0]), np.array([3.0]))
    assert r == float(np.float32(1.0) / np.float32(3.0)) and r != 1.0 / 3.0
    # a median: up to half the pixels may be arbitrary outliers
    prev = np.concatenate([np.full(51, 2.0), np.full(49, 1000.0)]).astype(np.float32)
    assert O.depth_scale_ratio(prev, np.ones(100, np.float32)) == 2.0


def _scaled_batches(world, depth, L, Ov, yaws, shifts, scales):
    """World poses and depth split into batches of L sharing Ov frames, batch b
    in its own yaw+translation frame and at its own scale 1/c_b (translations
    and depth divided by c_b), as a monocular model would return them."""
    out, start, b = [], 0, 0
    while True:
        hi = min(start + L, len(world))
        G = np.eye(4)
        G[:3, :3] = rot_y(yaws[b])
        G[:3, 3] = shifts[b]
        P = np.stack([(O.to4x4(world[k]) @ G)[:3] for k in range(start, hi)])
        P[:, :, 3] /= scales[b]
        out.append((P, depth[start:hi] / scales[b]))
        if hi == len(world):
            return out
        start = hi - Ov
        b += 1


def _stream(batches, align, n=80, mode=O.MODE_HEADING):
    p = O.Params(64, 48, window=8, smooth_len=5, mode=mode, pose_frame=O.POSES_BATCH_LOCAL,
                 overlap=4, depth_align=align)
    st = O.OracleStream(p)
    for P, D in batches:
        st.push(P, D, K)
    assert st.n_emitted == n
    return st


def _setup(seed, scale_fn):
    world = walk(WalkerSpec(n_frames=80, seed=seed, turns=True)).poses_w2c
    rng = np.random.default_rng(seed)
    depth = rng.uniform(0.3, 6.0, (80, 48, 64)).astype(np.float32)
    nb = 6
    yaws = [0.0] + list(rng.uniform(-3, 3, nb))
    shifts = [np.zeros(3)] + [rng.normal(size=3) * 5 for _ in range(nb)]
    scales = [1.0] + [scale_fn(rng) for _ in range(nb)]
    return world, depth, yaws, shifts, scales


def test_alignment_recovers_power_of_two_batch_scales_exactly():
    world, depth, yaws, shifts, scales = _setup(3, lambda r: 2.0 ** int(r.integers(-3, 4)))
    aligned = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, scales), True)
    truth = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, [1.0] * 7), False)
    # one scale per batch: c_b itself (the first batch defines the scale);
    # batch 0 emits frames 0..19, batch b >= 1 frames 20 + 16 (b - 1) ..
    for n in range(80):
        b = 0 if n < 20 else 1 + (n - 20) // 16
        assert aligned.scale[n] == scales[b]
    assert np.array_equal(np.stack(aligned.world), np.stack(truth.world))
    for n in (10, 33, 57, 79):
        ia, pa, Ma, Ga = aligned.frame(n)
        it, pt, Mt, Gt = truth.frame(n)
        assert ia == it
        assert np.array_equal(Ma, Mt) and np.array_equal(Ga, Gt)


def test_without_alignment_the_batch_scales_show():
    world, depth, yaws, shifts, scales = _setup(3, lambda r: 2.0 ** int(r.integers(-3, 4)))
    assert any(c != 1.0 for c in scales[1:5])
    raw = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, scales), False)
    truth = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, [1.0] * 7), False)
    diff = [not np.array_equal(raw.frame(n)[3], truth.frame(n)[3]) for n in range(20, 80, 7)]
    assert any(diff)


def test_alignment_of_arbitrary_scales_within_single_precision():
    world, depth, yaws, shifts, scales = _setup(4, lambda r: float(r.uniform(0.4, 2.5)))
    aligned = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, scales), True)
    truth = _stream(_scaled_batches(world, depth, 20, 4, yaws, shifts, [1.0] * 7), False)
    # the recovered scale of each batch is c_b up to the ratios' FP32 rounding
    for n in range(80):
        b = 0 if n < 20 else 1 + (n - 20) // 16
        assert abs(aligned.scale[n] / scales[b] - 1.0) < 4 * 2.0 ** -24 * (b + 1)
    np.testing.assert_allclose(np.stack(aligned.world), np.stack(truth.world), rtol=0, atol=1e-4)
    for n in (30, 60, 79):
        _, _, Ma, Ga = aligned.frame(n)
        _, _, Mt, Gt = truth.frame(n)
        np.testing.assert_allclose(Ma, Mt, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(Ga, Gt, rtol=1e-5, atol=1e-9)


def test_scale_carries_over_when_the_overlap_has_no_depth():
    world, depth, yaws, shifts, scales = _setup(5, lambda r: 2.0)
    batches = _scaled_batches(world, depth, 20, 4, yaws, shifts, scales)
    # the third batch's overlap depth is invalid everywhere: its scale is the
    # second batch's (no ratio); the fourth batch aligns against it again
    P, D = batches[2]
    D = D.copy()
    D[:4] = 0.0
    batches[2] = (P, D)
    st = _stream(batches, True)
    assert st.scale[0] == 1.0 and st.scale[20] == 2.0
    assert st.scale[36] == 2.0        # batch 2 (frames 36..51) kept batch 1's scale
    assert st.scale[52] == 2.0        # batch 3 aligns against batch 2 again: (1/2)/(1/2) = 1
