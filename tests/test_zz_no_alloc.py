"""mf_render_noalloc, the allocation-free entry point, against the stream API.

mf_render_noalloc serves callers that cannot let the library allocate device
memory: real-time loops where a cudaMalloc could stall the device, plugins
running inside a framework that owns all device memory, and processes held
to a fixed memory budget.  Its scratch lives in a static device array inside
libmf.  This test calls it through the C ABI twice in a row, with different
inputs each time, and checks each result against what the ordinary stream
entry points (mf_open_stream / mf_push_frames / mf_get_maps) return for the
same frames, within the tolerances of the parity tests; further cases run
the map maximum as Z (two persistent passes over the one shared work
counter), the tensor-core map kernel and 16-bit storage through it, each
twice in a row on one CUDA stream, and one case is compared with the FP64
oracle directly.  It sits in a file that pytest collects last.
"""
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
    return m


def _stream_result(mf, w, n_poses, n_render, depth_all, mode, dtype=torch.float32,
                   normalize="count", map_kernel="auto"):
    dev = torch.device("cuda", 0)
    s = mf.MotionFocusStream(w.width, w.height, window=w.window, smooth_len=w.smooth_len,
                             mode=mode, device=dev, depth_dtype=dtype, map_dtype=dtype,
                             normalize=normalize, map_kernel=map_kernel)
    s.push(torch.from_numpy(np.ascontiguousarray(w.poses[:n_poses])).to(dev), depth_all, w.K())
    M, G, info, _ = s.get_maps()
    s.close()
    return M[-n_render:], G[-n_render:], info[-n_render:]


MF_DT = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
STORAGE = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}


def _noalloc(mf, w, frames, n_render, poses, depth, mode, dtype=torch.float32, normalize="count",
             map_kernel="auto", cuda_stream=1):
    """One mf_render_noalloc call into fresh output buffers (enqueued only)."""
    dev = torch.device("cuda", 0)
    flags = {"auto": 0, "cuda_cores": mf.MF_FLAG_MAP_CUDA_CORES,
             "tensor_cores": mf.MF_FLAG_MAP_TENSOR_CORES}[map_kernel]
    desc = mf.mf_stream_desc_init(width=w.width, height=w.height, window=w.window,
                                  smooth_len=w.smooth_len,
                                  mode=mf.MF_MODE_ACCEL if mode == "accel" else mf.MF_MODE_HEADING,
                                  depth_dtype=MF_DT[dtype], map_dtype=MF_DT[dtype], flags=flags,
                                  normalize=mf.MF_NORM_MAX if normalize == "max" else mf.MF_NORM_COUNT,
                                  cuda_stream=cuda_stream)
    M = torch.empty((n_render, w.height, w.width), dtype=dtype, device=dev)
    G = torch.empty_like(M)
    info = torch.empty(n_render * mf.FRAME_INFO_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    mf.mf_render_noalloc(desc, frames, poses, n_render, depth, w.K(), M, G, info)
    return M, G, info


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


# (seed, frames, window, smooth_len, mode, n_render, storage dtype, Z, map kernel)
VARIANTS = [
    (31, 80, 8, 15, "heading", 60, torch.float32, "max", "cuda_cores"),
    (32, 72, 16, 9, "accel", 48, torch.float32, "count", "tensor_cores"),
    (33, 64, 12, 15, "heading", 40, torch.bfloat16, "count", "cuda_cores"),
    (34, 66, 8, 7, "heading", 50, torch.bfloat16, "max", "tensor_cores"),
]


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"{STORAGE[v[6]]}-{v[7]}-{v[8]}")
def test_noalloc_variants_back_to_back_on_one_stream(mf, variant):
    """Two calls in a row on one CUDA stream (the second with other inputs,
    no synchronisation between them), each against the stream entry points
    with the same storage type, normalisation and map kernel: the shared
    scratch carries nothing from one call into the next."""
    seed, frames, window, smooth_len, mode, n_render, dt, normalize, kernel = variant
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(dev)
    runs = []
    for k in range(2):
        w = small_stream(seed=seed + 100 * k, n_frames=frames, window=window, smooth_len=smooth_len)
        depth_all = torch.from_numpy(w.depth_stack(0, frames)).to(dev).to(dt)
        poses = torch.from_numpy(np.ascontiguousarray(w.poses)).to(dev)
        depth = depth_all[frames - n_render:].contiguous()
        with torch.cuda.stream(st):
            out = _noalloc(mf, w, frames, n_render, poses, depth, mode, dt, normalize, kernel,
                           cuda_stream=st.cuda_stream)
        runs.append((w, depth_all, poses, depth, out))
    st.synchronize()
    for w, depth_all, poses, depth, (M, G, info) in runs:
        info_np = info.cpu().numpy().view(mf.FRAME_INFO_DTYPE)
        Mr, Gr, info_r = _stream_result(mf, w, frames, n_render, depth_all, mode, dt, normalize, kernel)
        assert info_np["n_valid"].sum() > 0
        # the same kernels on the same records: maps within the map tolerance
        # of the storage type (a rounding step apart at most)
        parity.check_map(M.double().cpu().numpy(), Mr.double().cpu().numpy(), STORAGE[dt], where="M")
        parity.check_map(G.double().cpu().numpy(), Gr.double().cpu().numpy(), STORAGE[dt], where="G")
        for k in parity.INT_FIELDS:
            assert np.array_equal(info_np[k], info_r[k]), k
        mm, mr = info_np["map_max"].astype(np.float64), info_r["map_max"].astype(np.float64)
        assert np.all(np.abs(mm - mr) <= 1e-5 * np.abs(mr) + 1e-10)


def test_noalloc_matches_the_oracle(mf):
    """One allocation-free call against the FP64 oracle directly: records
    exactly, focus and maps within the parity tests' tolerances."""
    dev = torch.device("cuda", 0)
    frames, n_render = 96, 70
    w = small_stream(seed=41, n_frames=frames, window=16, smooth_len=11)
    depth_all = w.depth_stack(0, frames)
    poses = torch.from_numpy(np.ascontiguousarray(w.poses)).to(dev)
    depth = torch.from_numpy(np.ascontiguousarray(depth_all[frames - n_render:])).to(dev)
    M, G, info = _noalloc(mf, w, frames, n_render, poses, depth, "heading")
    torch.cuda.synchronize()
    info_np = info.cpu().numpy().view(mf.FRAME_INFO_DTYPE)
    ref = O.OracleStream(O.Params(w.width, w.height, window=16, smooth_len=11, mode=O.MODE_HEADING))
    ref.push(w.poses, depth_all.astype(np.float64), w.K())
    intr = O.compensated_intrinsics(w.K(), ref.p)
    Mh, Gh = M.double().cpu().numpy(), G.double().cpu().numpy()
    for j in range(n_render):
        n = frames - n_render + j
        rinfo, rp, Mr, Gr = ref.frame(n)
        parity.check_frame(info_np[j], None, rinfo, rp, intr, where=f"frame {n}",
                           size=(w.width, w.height))
        parity.check_map(Mh[j], Mr, where=f"M frame {n}")
        parity.check_map(Gh[j], Gr, where=f"G frame {n}")
        parity.check_argmax(info_np[j], Mr, rinfo["n_valid"], where=f"argmax {n}")
    assert info_np["n_valid"].sum() > 0


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
