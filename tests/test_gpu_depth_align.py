"""Depth alignment across batches (MF_FLAG_DEPTH_ALIGN, Section 2.2 Fig. 3)
on the GPU against the FP64 oracle: batch-local batches returned at their
own scales, with a share of the overlap frames' depth replaced by outliers
and invalid values so that the median selection itself is exercised.  The
batch scale is compared exactly (the GPU's FP32 report of it), the records,
motion points and maps within the parity tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from synth import WalkerSpec, walk  # noqa: E402
from tests import parity  # noqa: E402
from tests.test_oracle_depth_align import _scaled_batches  # noqa: E402

pytestmark = pytest.mark.gpu

W, H, OV, L = 160, 120, 4, 24
K = np.array([150.0, 150.0, 80.0, 60.0])
TDT = {"f32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    return m


def _batches(seed, pow2, n=96):
    world = walk(WalkerSpec(n_frames=n, seed=seed, turns=True, accel=1.0)).poses_w2c
    rng = np.random.default_rng(seed)
    depth = rng.uniform(0.3, 6.0, (n, H, W)).astype(np.float32)
    nb = 8
    yaws = [0.0] + list(rng.uniform(-3, 3, nb))
    shifts = [np.zeros(3)] + [rng.normal(size=3) * 5 for _ in range(nb)]
    if pow2:
        scales = [1.0] + [2.0 ** int(rng.integers(-3, 4)) for _ in range(nb)]
    else:
        scales = [1.0] + [float(rng.uniform(0.4, 2.5)) for _ in range(nb)]
    batches = _scaled_batches(world, depth, L, OV, yaws, shifts, scales)
    out = []
    for b, (P, D) in enumerate(batches):
        D = D.copy()
        if b > 0:
            # overlap frames of this batch: ~30 % outliers, some invalid depth
            m = rng.random((OV, H, W))
            D[:OV][m < 0.3] = rng.uniform(0.01, 100.0, int((m < 0.3).sum()))
            D[:OV][(m >= 0.3) & (m < 0.35)] = 0.0
            D[:OV][(m >= 0.35) & (m < 0.37)] = np.nan
        out.append((np.ascontiguousarray(P), D))
    return out, scales


def _run(mf, batches, storage, on_host, reset_after=None):
    """Pushes every batch through one aligned stream; with reset_after = b,
    renders and resets the stream after batch b.  Returns the renders
    concatenated (maps, records, points) and the depth values the kernels read."""
    dev = torch.device("cuda", 0)
    dt = TDT[storage]
    s = mf.MotionFocusStream(W, H, window=8, smooth_len=5, mode="heading", pose_frame="batch_local",
                             overlap=OV, depth_dtype=dt, map_dtype=dt, device=dev, depth_align=True,
                             max_pending=512)
    seen, outs, keep = [], [], []
    for b, (P, D) in enumerate(batches):
        Dt = torch.from_numpy(D).to(dt)
        seen.append(Dt.to(torch.float64).numpy())          # the values the kernels read
        # device inputs are read when their frames render: keep them alive
        inputs = (P, Dt) if on_host else (torch.from_numpy(P).to(dev), Dt.to(dev))
        keep.append(inputs)
        s.push(inputs[0], inputs[1], K)
        if reset_after is not None and b == reset_after:
            outs.append(s.get_maps())
            mf.mf_reset_stream(s.handle)
    outs.append(s.get_maps())
    s.close()
    M = np.concatenate([o[0].double().cpu().numpy() for o in outs])
    G = np.concatenate([o[1].double().cpu().numpy() for o in outs])
    info = np.concatenate([o[2] for o in outs])
    pts = np.concatenate([o[3] for o in outs])
    return M, G, info, pts, seen


def _oracle(batches_seen):
    ref = O.OracleStream(O.Params(W, H, window=8, smooth_len=5, mode=O.MODE_HEADING,
                                  pose_frame=O.POSES_BATCH_LOCAL, overlap=OV, depth_align=True))
    for P, D in batches_seen:
        ref.push(P, D, K)
    return ref


@pytest.mark.parametrize("pow2,storage,on_host", [(True, "f32", False), (False, "f32", False),
                                                  (False, "f32", True), (False, "bf16", False)])
def test_depth_alignment_matches_oracle(mf, pow2, storage, on_host):
    batches, scales = _batches(21 if pow2 else 22, pow2)
    M, G, info, pts, seen = _run(mf, batches, storage, on_host)
    ref = _oracle([(P, D) for (P, _), D in zip(batches, seen)])
    assert len(info) == ref.n_emitted == 96
    intr = O.compensated_intrinsics(K, ref.p)
    # the selected median, hence the batch scale, is the oracle's exactly
    assert np.array_equal(info["depth_scale"], np.array(ref.scale, dtype=np.float32))
    assert len(set(ref.scale)) > 3
    for n in range(ref.n_emitted):
        rinfo, rp, Mr, Gr = ref.frame(n)
        parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}", size=(W, H))
        parity.check_map(M[n], Mr, storage, where=f"M frame {n}")
        parity.check_map(G[n], Gr, storage, where=f"G frame {n}")
    if pow2:
        # power-of-two batch scales are recovered exactly: batch b has c_b
        for n in range(96):
            b = 0 if n < L else 1 + (n - L) // (L - OV)
            assert ref.scale[n] == scales[b]


def test_reset_starts_a_first_batch_again(mf):
    batches, _ = _batches(23, False, n=64)
    M, G, info, pts, seen = _run(mf, batches[:3] + batches[:2], "f32", False, reset_after=2)
    # after the reset, the first two batches again: scale 1, then the same
    # ratio as the first time
    assert len(info) == (L + 2 * (L - OV)) + (L + (L - OV))
    first = info[:L + (L - OV)]
    again = info[-(L + (L - OV)):]
    assert np.array_equal(M[:L + (L - OV)], M[-(L + (L - OV)):])
    assert np.array_equal(first["depth_scale"], again["depth_scale"])
    assert first["depth_scale"][0] == 1.0 and first["depth_scale"][-1] != 1.0


def test_depth_alignment_needs_batch_local_streams(mf):
    dev = torch.device("cuda", 0)
    with pytest.raises(mf.MFError) as e:
        mf.MotionFocusStream(64, 48, window=8, smooth_len=5, device=dev, depth_align=True)
    assert e.value.status == mf.MF_ERR_INVALID_ARG
    eng = mf.MotionFocusEngine(max_streams=2, max_tick_frames=16, max_stream_frames=8, device=dev)
    d = mf.mf_stream_desc_init(width=64, height=48, window=8, smooth_len=5,
                               pose_frame=mf.MF_POSES_BATCH_LOCAL, overlap=2,
                               flags=mf.MF_FLAG_DEPTH_ALIGN)
    with pytest.raises(mf.MFError) as e:
        mf.mf_engine_add_stream(eng.handle, d)
    assert e.value.status == mf.MF_ERR_INVALID_ARG
    eng.close()
