"""Failure detection with faults made on the host (mf_set_fault): an
allocation that fails, a pose that is no rotation, a serving push that is
lost, an admission that is refused, a device wait reported as run out, and a
stream closed with its work in flight.  No test makes a GPU fault, trap or
hang; each checks the status the library reports and that the CUDA context
stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from synth import small_stream  # noqa: E402
from tests import parity  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    yield m
    m.mf_set_fault(None)


@pytest.fixture(autouse=True)
def clear_rules(mf):
    mf.mf_set_fault(None)
    yield
    mf.mf_set_fault(None)


def _usable(mf):
    """A fresh stream still renders a small push correctly."""
    dev = torch.device("cuda", 0)
    w = small_stream(n_frames=24, smooth_len=7)
    s = mf.MotionFocusStream(w.width, w.height, window=8, smooth_len=7, mode="heading", device=dev)
    s.push(torch.from_numpy(w.poses).to(dev), torch.from_numpy(w.depth_stack(0, 24)).to(dev), w.K())
    M, G, info, _ = s.get_maps()
    s.close()
    assert info["n_valid"].sum() > 0 and torch.isfinite(M).all()


def test_allocation_failure_is_reported(mf):
    dev = torch.device("cuda", 0)
    mf.mf_set_fault("alloc_fail@1")
    with pytest.raises(mf.MFError) as e:
        mf.MotionFocusStream(64, 48, window=8, smooth_len=5, device=dev)
    assert e.value.status == mf.MF_ERR_OOM
    mf.mf_set_fault("alloc_fail")
    with pytest.raises(mf.MFError) as e:
        mf.MotionFocusEngine(max_streams=2, max_tick_frames=16, max_stream_frames=8, device=dev)
    assert e.value.status == mf.MF_ERR_OOM
    mf.mf_set_fault(None)
    _usable(mf)


def test_bad_pose_is_flagged_per_frame(mf):
    """The 10th host pose is corrupted on its way to the device: its frame
    reports MF_FRAME_BAD_POSE and every frame matches the oracle run on the
    same corrupted poses."""
    dev = torch.device("cuda", 0)
    w = small_stream(seed=7, n_frames=40, smooth_len=5)
    depth = w.depth_stack(0, 40)
    mf.mf_set_fault("bad_pose@10")
    s = mf.MotionFocusStream(w.width, w.height, window=8, smooth_len=5, mode="heading", device=dev)
    s.push(np.ascontiguousarray(w.poses), torch.from_numpy(depth).to(dev), w.K())
    M, G, info, pts = s.get_maps()
    s.close()
    bad = np.array(w.poses)
    bad[9, 0, 0] *= 2.0
    ref = O.OracleStream(O.Params(w.width, w.height, window=8, smooth_len=5, mode=O.MODE_HEADING))
    ref.push(bad, depth.astype(np.float64), w.K())
    intr = O.compensated_intrinsics(w.K(), ref.p)
    assert info["status"][9] == mf.MF_FRAME_BAD_POSE
    Mh = M.double().cpu().numpy()
    for n in range(40):
        rinfo, rp, Mr, _ = ref.frame(n)
        parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}", size=(w.width, w.height))
        parity.check_map(Mh[n], Mr, where=f"M frame {n}")


def test_lost_serving_push_is_detected(mf):
    """The second push is accepted and lost: drain gives up with
    MF_ERR_TIMEOUT and frames_done falls short by that push's frames."""
    dev = torch.device("cuda", 0)
    w = small_stream(seed=8, n_frames=30, smooth_len=5)
    srv = mf.MotionFocusServer(max_streams=2, max_tick_frames=64, max_stream_frames=16, tick_us=50,
                               device=dev)
    slot = srv.add_stream(w.width, w.height, window=8, smooth_len=5)
    D = torch.from_numpy(w.depth_stack(0, 30)).to(dev)
    M = torch.zeros((30, w.height, w.width), device=dev)
    mf.mf_set_fault("drop_push@2")
    for lo in range(0, 30, 10):
        srv.submit(slot, w.poses[lo:lo + 10], D[lo:lo + 10], w.K(), M[lo:lo + 10])
    with pytest.raises(mf.MFError) as e:
        srv.drain(timeout_ns=500_000_000)
    assert e.value.status == mf.MF_ERR_TIMEOUT
    assert srv.frames_done(slot) == 20
    assert M[10:20].abs().sum() == 0          # the lost push never rendered
    srv.close()
    _usable(mf)


def test_refused_admission(mf):
    dev = torch.device("cuda", 0)
    eng = mf.MotionFocusEngine(max_streams=4, max_tick_frames=16, max_stream_frames=8, device=dev)
    mf.mf_set_fault("admission_full@2")
    eng.add_stream(64, 48, window=8, smooth_len=5)
    with pytest.raises(mf.MFError) as e:
        eng.add_stream(64, 48, window=8, smooth_len=5)
    assert e.value.status == mf.MF_ERR_ADMISSION
    eng.add_stream(64, 48, window=8, smooth_len=5)   # only the second was refused
    assert eng.stats().streams == 2
    eng.close()


def test_device_wait_run_out_is_reported_once(mf):
    """A completed wait reports a device wait that ran out (here injected on
    the host, through the same fault word a map kernel sets) as
    MF_ERR_TIMEOUT, once; the stream then works on."""
    dev = torch.device("cuda", 0)
    w = small_stream(seed=9, n_frames=24, smooth_len=7)
    s = mf.MotionFocusStream(w.width, w.height, window=8, smooth_len=7, device=dev)
    s.push(torch.from_numpy(w.poses).to(dev), torch.from_numpy(w.depth_stack(0, 24)).to(dev), w.K())
    s.get_maps()
    mf.mf_set_fault("wait_timeout@1")
    with pytest.raises(mf.MFError) as e:
        mf.mf_sync(s.handle)
    assert e.value.status == mf.MF_ERR_TIMEOUT
    mf.mf_sync(s.handle)                      # reported once
    s.close()
    _usable(mf)


def test_close_with_work_in_flight(mf):
    """Closing a stream right after enqueueing a large push and render waits
    for its work and releases everything; the device stays usable."""
    dev = torch.device("cuda", 0)
    w = small_stream(seed=10, n_frames=64)
    D = torch.from_numpy(w.depth_stack(0, 64)).to(dev)
    for _ in range(3):
        s = mf.MotionFocusStream(w.width, w.height, window=8, smooth_len=15, device=dev)
        s.push(torch.from_numpy(w.poses).to(dev), D, w.K())
        M = torch.empty((64, w.height, w.width), device=dev)
        mf.mf_get_maps(s.handle, 64, M, None, None, None)
        s.close()
    torch.cuda.synchronize()
    _usable(mf)
