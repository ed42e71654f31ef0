"""Stream snapshot and restore: a stream moved mid-sequence into a freshly
opened stream (another CUDA stream) continues exactly as the original --
the same later pushes give bit-identical maps and records -- for world
poses and for batch-local batches with depth alignment; a mismatched
descriptor, pending frames or a used stream are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import small_stream  # noqa: E402
from tests.test_gpu_depth_align import H, K as K_ALIGN, OV, W, _batches  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    return m


def _get(s):
    M, G, info, pts = s.get_maps()
    return M.cpu().numpy(), G.cpu().numpy(), info, pts


def test_world_stream_moves_mid_sequence(mf):
    dev = torch.device("cuda", 0)
    w = small_stream(seed=31, n_frames=80, window=12, smooth_len=9)
    P = torch.from_numpy(w.poses).to(dev)
    D = torch.from_numpy(w.depth_stack(0, 80)).to(dev)
    kw = dict(window=12, smooth_len=9, mode="heading", device=dev)
    a = mf.MotionFocusStream(320, 240, **kw)
    a.push(P[:37], D[:37], w.K())
    with pytest.raises(mf.MFError) as e:        # frames pending
        a.snapshot()
    assert e.value.status == mf.MF_ERR_NOT_READY
    _get(a)
    blob = a.snapshot()
    b = mf.MotionFocusStream(320, 240, cuda_stream=torch.cuda.Stream(dev), **kw)
    b.restore(blob)
    for s in (a, b):
        s.push(P[37:], D[37:], w.K())
    ra, rb = _get(a), _get(b)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    assert rb[2]["frame_index"][0] == 37 and rb[2]["n_valid"].sum() > 0
    with pytest.raises(mf.MFError) as e:        # b has taken pushes
        b.restore(blob)
    assert e.value.status == mf.MF_ERR_NOT_READY
    c = mf.MotionFocusStream(320, 240, window=8, smooth_len=9, mode="heading", device=dev)
    with pytest.raises(mf.MFError) as e:        # another window
        c.restore(blob)
    assert e.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as e:        # damaged
        mf.MotionFocusStream(320, 240, **kw).restore(blob[:-8])
    assert e.value.status == mf.MF_ERR_INVALID_ARG
    for s in (a, b, c):
        s.close()


def test_aligned_batch_local_stream_moves_between_batches(mf):
    dev = torch.device("cuda", 0)
    batches, _ = _batches(24, False, n=96)
    kw = dict(window=8, smooth_len=5, mode="heading", pose_frame="batch_local", overlap=OV,
              depth_align=True, device=dev, max_pending=512)
    keep = [(torch.from_numpy(P).to(dev), torch.from_numpy(D).to(dev)) for P, D in batches]
    a = mf.MotionFocusStream(W, H, **kw)
    for P, D in keep[:2]:
        a.push(P, D, K_ALIGN)
    _get(a)
    b = mf.MotionFocusStream(W, H, **kw)
    b.restore(a.snapshot())
    for s in (a, b):
        for P, D in keep[2:]:
            s.push(P, D, K_ALIGN)
    ra, rb = _get(a), _get(b)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    assert len(set(rb[2]["depth_scale"].tolist())) > 1    # later batches realigned
    a.close()
    b.close()
