"""mf_render_noalloc, the allocation-free entry point, against the stream API.

mf_render_noalloc serves callers that cannot let the library allocate device
memory: real-time loops where a cudaMalloc could stall the device, plugins
running inside a framework that owns all device memory, and processes held
to a fixed memory budget.  Its scratch lives in a static device array inside
libmf.  This test calls it through the C ABI twice in a row, with different
inputs each time, and checks each result against what the ordinary stream
entry points (mf_open_stream / mf_push_frames / mf_get_maps) return for the
same frames, within the tolerances of the parity tests.  It sits in a file
that pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    return m


def _stream_result(mf, w, n_poses, n_render, depth_all, mode):
    dev = torch.device("cuda", 0)
    s = mf.MotionFocusStream(w.width, w.height, window=w.window, smooth_len=w.smooth_len,
                             mode=mode, device=dev)
    s.push(torch.from_numpy(np.ascontiguousarray(w.poses[:n_poses])).to(dev), depth_all, w.K())
    M, G, info, _ = s.get_maps()
    s.close()
    return M[-n_render:], G[-n_render:], info[-n_render:]


CASES = [  # (seed, frames, window, smooth_len, mode, n_render)
    (21, 90, 8, 15, "accel", 64),
    (22, 70, 12, 9, "heading", 50),
]


def test_noalloc_matches_stream_entry_points_on_consecutive_calls(mf):
    dev = torch.device("cuda", 0)
    for seed, frames, window, smooth_len, mode, n_render in CASES:
        w = small_stream(seed=seed, n_frames=frames, window=window, smooth_len=smooth_len)
        depth_all = torch.from_numpy(w.depth_stack(0, frames)).to(dev)
        poses = torch.from_numpy(np.ascontiguousarray(w.poses)).to(dev)
        depth = depth_all[frames - n_render:].contiguous()
        desc = mf.mf_stream_desc_init(width=w.width, height=w.height, window=window,
                                      smooth_len=smooth_len,
                                      mode=mf.MF_MODE_ACCEL if mode == "accel" else mf.MF_MODE_HEADING,
                                      cuda_stream=1)
        M = torch.empty((n_render, w.height, w.width), dtype=torch.float32, device=dev)
        G = torch.empty_like(M)
        info = torch.empty(n_render * mf.FRAME_INFO_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        mf.mf_render_noalloc(desc, frames, poses, n_render, depth, w.K(), M, G, info)
        torch.cuda.synchronize()
        info_np = info.cpu().numpy().view(mf.FRAME_INFO_DTYPE)

        Mr, Gr, info_r = _stream_result(mf, w, frames, n_render, depth_all, mode)
        assert info_np["n_valid"].sum() > 0
        parity.check_map(M.double().cpu().numpy(), Mr.double().cpu().numpy(), where="M")
        parity.check_map(G.double().cpu().numpy(), Gr.double().cpu().numpy(), where="G")
        for k in parity.INT_FIELDS + ("argmax_x", "argmax_y"):
            assert np.array_equal(info_np[k], info_r[k]), k
        ok = info_r["focus_valid"] == 1
        tol = parity.coord_tol(info_r["focus_u"][ok], info_r["focus_v"][ok], w.intr)
        assert np.all(np.abs(info_np["focus_u"][ok] - info_r["focus_u"][ok]) <= tol)
        assert np.all(np.abs(info_np["focus_v"][ok] - info_r["focus_v"][ok]) <= tol)


def test_noalloc_rejects_sizes_beyond_its_limit(mf):
    dev = torch.device("cuda", 0)
    w = small_stream(seed=23, n_frames=8)
    desc = mf.mf_stream_desc_init(width=w.width, height=w.height, cuda_stream=1)
    poses = torch.zeros((mf.MF_NOALLOC_MAX_POSES + 1, 12), dtype=torch.float64, device=dev)
    for n_poses, n_render in ((mf.MF_NOALLOC_MAX_FRAMES + 1, mf.MF_NOALLOC_MAX_FRAMES + 1),
                              (mf.MF_NOALLOC_MAX_POSES + 1, 8), (8, 9), (8, 0)):
        with pytest.raises(mf.MFError) as e:
            mf.mf_render_noalloc(desc, n_poses, poses, n_render, None, w.K())
        assert e.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as e:   # host memory is refused as well
        mf.mf_render_noalloc(desc, 8, np.zeros((8, 12)), 8, None, w.K())
    assert e.value.status == mf.MF_ERR_INVALID_ARG
