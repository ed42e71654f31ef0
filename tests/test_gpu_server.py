"""The serving loop: continuous batching gives the engine's results, accepts
pushes from several threads at once, and reports per-frame latency."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.test_gpu_engine import STREAMS, _inputs, _run_engine  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    return m


def _serve(mf, specs, chunk=7, threads=1):
    dev = torch.device("cuda", 0)
    srv = mf.MotionFocusServer(max_streams=8, max_tick_frames=512, max_stream_frames=16,
                               tick_us=100, device=dev)
    state = []
    for spec in specs:
        width, height, window, smooth_len, mode, seed, frames = spec
        poses, depth, K = _inputs(spec)
        slot = srv.add_stream(width, height, window=window, smooth_len=smooth_len, mode=mode)
        state.append(dict(slot=slot, poses=poses, depth=torch.from_numpy(depth).to(dev), K=K,
                          M=torch.zeros((frames, height, width), device=dev),
                          G=torch.zeros((frames, height, width), device=dev),
                          info=torch.zeros(frames * 64, dtype=torch.uint8, device=dev),
                          frames=frames))
    torch.cuda.synchronize()

    def feed(sts):
        for s in sts:
            for lo in range(0, s["frames"], chunk):
                hi = min(s["frames"], lo + chunk)
                srv.submit(s["slot"], s["poses"][lo:hi], s["depth"][lo:hi], s["K"],
                           s["M"][lo:hi], s["G"][lo:hi], s["info"][lo * 64:hi * 64])

    groups = [state[i::threads] for i in range(threads)]
    ths = [threading.Thread(target=feed, args=(g,)) for g in groups]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    srv.drain()
    for s in state:
        assert srv.frames_done(s["slot"]) == s["frames"]
    lat = srv.latency()
    st = srv.stats()
    for s in state:
        srv.remove_stream(s["slot"])
    out = [(s["M"].cpu().numpy(), s["G"].cpu().numpy(),
            s["info"].cpu().numpy().view(mf.FRAME_INFO_DTYPE)) for s in state]
    srv.close()
    return out, lat, st


def test_server_results_equal_engine(mf):
    eng, _ = _run_engine(mf, STREAMS)
    srv, lat, st = _serve(mf, STREAMS)
    for a, b in zip(eng, srv):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert lat.frames == sum(s[6] for s in STREAMS)
    assert 0.0 < lat.p50_ms <= lat.p99_ms <= lat.max_ms
    assert st.frames == lat.frames and st.graph_launches == st.ticks


def test_server_concurrent_submitters(mf):
    eng, _ = _run_engine(mf, STREAMS)
    srv, lat, st = _serve(mf, STREAMS, threads=3)
    for a, b in zip(eng, srv):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert lat.frames == sum(s[6] for s in STREAMS)


def test_server_queue_limit_and_unknown_stream(mf):
    dev = torch.device("cuda", 0)
    srv = mf.MotionFocusServer(max_streams=2, max_tick_frames=64, max_stream_frames=8,
                               tick_us=10_000_000, queue_limit=2, device=dev)
    s = srv.add_stream(64, 48, window=4, smooth_len=3)
    P = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), (4, 1, 1))
    K = (50.0, 50.0, 32.0, 24.0)
    srv.submit(s, P, None, K)
    srv.submit(s, P, None, K)
    with pytest.raises(mf.MFError) as e:
        srv.submit(s, P, None, K)                # the queue holds two pushes
    assert e.value.status == mf.MF_ERR_NOT_READY
    with pytest.raises(mf.MFError) as e:
        srv.submit(1, P, None, K)                # slot 1 was never admitted
    assert e.value.status == mf.MF_ERR_INVALID_ARG
    srv.close()                                  # stops with queued work: no hang


def test_latency_probe_stamps_after_the_work(mf):
    """mf_probe_stamp: the completion stamp of the plain per-stream path.  A
    stamp enqueued behind a stream's map rendering completes after it, and
    each frame's latency runs from its own arrival time."""
    dev = torch.device("cuda", 0)
    spec = STREAMS[0]
    width, height, window, smooth_len, mode, seed, frames = spec
    poses, depth, K = _inputs(spec)
    st = torch.cuda.Stream(dev)
    s = mf.MotionFocusStream(width, height, window=window, smooth_len=smooth_len, mode=mode,
                             device=dev, cuda_stream=st)
    p = mf._mf.mf_probe_open()
    D = torch.from_numpy(depth).to(dev)
    torch.cuda.synchronize()
    t_before = mf.mf_clock_ns()
    arrivals = np.array([t_before - 1_000_000 * k for k in range(frames)], dtype=np.int64)
    s.push(torch.from_numpy(poses).to(dev), D, K)
    M, G, info, _ = s.get_maps()
    mf._mf.mf_probe_stamp(p, st.cuda_stream, arrivals)
    st.synchronize()
    t_after = mf.mf_clock_ns()
    # the host function may still be running just after the stream's work
    for _ in range(1000):
        lat = mf._mf.mf_probe_latency(p)
        if lat.frames == frames:
            break
        torch.cuda.synchronize()
    assert lat.frames == frames
    span_ms = (t_after - t_before) * 1e-6
    # frame k arrived k ms before t_before: its latency is k ms plus the work
    assert 0.0 < lat.p50_ms and lat.max_ms <= (frames - 1) + span_ms + 50.0
    assert lat.max_ms >= frames - 1
    empty = mf._mf.mf_probe_latency(p, reset=True)
    assert empty.frames == frames
    assert mf._mf.mf_probe_latency(p).frames == 0
    mf._mf.mf_probe_close(p)
    s.close()
