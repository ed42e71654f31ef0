"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from synth import WalkerSpec, hd_stream, small_stream, walk  # noqa: E402
from tests import parity  # noqa: E402
from tests.posegen import rot_x, rot_y, trajectory  # noqa: E402

pytestmark = pytest.mark.gpu

TDT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    return m


def _mode(name):
    return O.MODE_ACCEL if name == "accel" else O.MODE_HEADING


def run_both(mf, poses, depth, K, width, height, window=8, smooth_len=15, mode="accel",
             storage="f32", pushes=None, pose_frame="world", overlap=0, calib=None,
             on_host=False, get_chunks=None, normalize="count", map_kernel="auto"):
    """Run the same pushes through the GPU stream and the oracle."""
    dev = torch.device("cuda", 0)
    dt = TDT[storage]
    s = mf.MotionFocusStream(width, height, window=window, smooth_len=smooth_len, mode=mode,
                             pose_frame=pose_frame, overlap=overlap, depth_dtype=dt, map_dtype=dt,
                             calib=calib, device=dev, normalize=normalize, map_kernel=map_kernel)
    p = O.Params(width, height, window=window, smooth_len=smooth_len, mode=_mode(mode),
                 pose_frame=O.POSES_BATCH_LOCAL if pose_frame == "batch_local" else O.POSES_WORLD,
                 overlap=overlap, calib_width=calib[0] if calib else 0,
                 calib_height=calib[1] if calib else 0, normalize=normalize)
    ref = O.OracleStream(p)
    pushes = pushes or [(0, len(poses))]
    keep = []
    for lo, hi in pushes:
        P = np.ascontiguousarray(poses[lo:hi])
        D = None
        D64 = None
        if depth is not None:
            Dt = torch.from_numpy(np.ascontiguousarray(depth[lo:hi])).to(dt)
            D64 = Dt.to(torch.float64).numpy()          # the values the kernel reads
            D = Dt if on_host else Dt.to(dev)
        Pt = P if on_host else torch.from_numpy(P).to(dev)
        keep.append((Pt, D))
        s.push(Pt, D, K)
        ref.push(P, D64, K)
    outs = []
    if get_chunks:
        for c in get_chunks:
            outs.append(s.get_maps(c))
    outs.append(s.get_maps())
    M = torch.cat([o[0] for o in outs if o[0] is not None]).float().cpu().numpy()
    G = torch.cat([o[1] for o in outs if o[1] is not None]).float().cpu().numpy()
    info = np.concatenate([o[2] for o in outs])
    pts = np.concatenate([o[3] for o in outs if o[3] is not None])
    s.close()
    return M, G, info, pts, ref


def compare_all(M, G, info, pts, ref, K, storage="f32", maps=True):
    assert len(info) == ref.n_emitted
    intr = O.compensated_intrinsics(K, ref.p)
    worst = 0.0
    for n in range(ref.n_emitted):
        rinfo, rp, Mr, Gr = ref.frame(n, full_maps=maps)
        parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}",
                           size=(ref.p.width, ref.p.height))
        if maps:
            worst = max(worst, parity.check_map(M[n], Mr, storage, f"M frame {n}")[0])
            if Gr is not None:
                parity.check_map(G[n], Gr, storage, f"G frame {n}")
            else:
                assert not G[n].any()
            if storage == "f32":
                parity.check_argmax(info[n], Mr, rinfo["n_valid"], where=f"argmax {n}")
    return worst


# ---------------------------------------------------------------- configs --
KERNELS = ["cuda_cores", "tensor_cores"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("mode", ["accel", "heading"])
def test_small_stream_parity(mf, mode, kernel):
    """320x240, 64 frames, window 8 (3 x 4 tiles with ragged right/bottom edges)."""
    w = small_stream()
    M, G, info, pts, ref = run_both(mf, w.poses, w.depth_stack(0, 64), w.K(), 320, 240,
                                    window=8, smooth_len=15, mode=mode, map_kernel=kernel)
    compare_all(M, G, info, pts, ref, w.K())
    assert info["n_valid"].sum() > 300


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_small_stream_16bit_storage(mf, storage, kernel):
    w = small_stream()
    M, G, info, pts, ref = run_both(mf, w.poses, w.depth_stack(0, 64), w.K(), 320, 240,
                                    mode="heading", storage=storage, map_kernel=kernel)
    compare_all(M, G, info, pts, ref, w.K(), storage=storage)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_storage_error_report(mf, storage):
    """Per-output error of 16-bit storage against the FP64 oracle (printed).

    The bound is the storage format's rounding on top of the FP32 tolerance.
    """
    import json
    w = small_stream()
    stats = {}
    for mode in ("accel", "heading"):
        M, G, info, pts, ref = run_both(mf, w.poses, w.depth_stack(0, 64), w.K(), 320, 240,
                                        mode=mode, storage=storage)
        errs = {"M": [], "G": []}
        rels = {"M": [], "G": []}
        for n in range(ref.n_emitted):
            _, _, Mr, Gr = ref.frame(n)
            for key, got, r in (("M", M[n], Mr), ("G", G[n], Gr)):
                e = np.abs(got.astype(np.float64) - r)
                errs[key].append(e)
                big = r > 1e-6
                rels[key].append(e[big] / r[big])
                assert np.all(e <= parity.map_tol(r, storage)), (mode, key, n)
        for key in ("M", "G"):
            e = np.concatenate([x.ravel() for x in errs[key]])
            rr = np.concatenate([x.ravel() for x in rels[key]])
            stats[f"{mode}_{key}"] = {"max_abs": float(e.max()), "mean_abs": float(e.mean()),
                                      "max_rel": float(rr.max()), "mean_rel": float(rr.mean())}
    print("\nSTORAGE_ERROR", storage, json.dumps(stats))


def _accelerating_walk(n, width=320, seed=0):
    """Forward acceleration with sway: ACCEL points land inside the frame."""
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    for k in range(n):
        t = k / 30.0
        cs.append(np.array([0.05 * math.sin(2.0 * t), 0.02 * math.sin(3.1 * t),
                            1.0 * t + 0.6 * t * t]) + rng.normal(0, 1e-4, 3))
        rs.append(rot_y(0.2 * math.sin(1.3 * t)) @ rot_x(0.05 * math.sin(4 * t)))
    return trajectory(cs, rs)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("window,smooth_len", [(8, 3), (16, 15), (32, 33), (5, 7), (1, 3),
                                               (24, 9)])
def test_windows_in_frame_accel(mf, window, smooth_len, kernel):
    poses = _accelerating_walk(80)
    rng = np.random.default_rng(1)
    depth = rng.uniform(0.2, 5.0, (80, 240, 320)).astype(np.float32)
    K = np.array([260.0, 260.0, 160.0, 120.0])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, 320, 240, window=window,
                                    smooth_len=smooth_len, mode="accel", map_kernel=kernel)
    compare_all(M, G, info, pts, ref, K)
    assert info["n_valid"][-1] == window and M[-1].max() > 0.05


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("window,normalize", [(24, "count"), (32, "count"), (20, "max")])
def test_windows_above_16_with_16bit_storage(mf, storage, window, normalize):
    """16-bit maps of 17..32-point windows (the 32-point map path), ACCEL points
    in view, both normalisations; a width whose last strip leaves the frame."""
    poses = _accelerating_walk(80)
    rng = np.random.default_rng(2)
    depth = rng.uniform(0.2, 5.0, (80, 240, 330)).astype(np.float32)
    K = np.array([260.0, 260.0, 165.0, 120.0])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, 330, 240, window=window, smooth_len=15,
                                    mode="accel", storage=storage, normalize=normalize)
    if normalize == "count":
        compare_all(M, G, info, pts, ref, K, storage=storage)
    else:
        intr = O.compensated_intrinsics(K, ref.p)
        cst = O.OracleStream(O.Params(330, 240, window=window, smooth_len=15))
        cst.push(poses, torch.from_numpy(depth).to(TDT[storage]).double().numpy(), K)
        for n in range(ref.n_emitted):
            rinfo, rp, Mr, Gr = ref.frame(n)
            parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}", size=(330, 240))
            mx = cst.frame(n)[2].max()
            if rinfo["n_valid"] == 0 or abs(mx - O.NORM_FLOOR) <= 4 * parity.MAP_RTOL * O.NORM_FLOOR:
                continue
            div = mx if mx >= O.NORM_FLOOR else None
            parity.check_map(M[n], Mr, storage, where=f"M frame {n}", divisor=div)
            parity.check_map(G[n], Gr, storage, where=f"G frame {n}", divisor=div)
    assert info["n_valid"][-1] == window and M[-1].max() > 0.05


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("width,height", [(333, 197), (130, 70), (4, 3), (1, 1), (129, 65),
                                          (257, 129)])
def test_ragged_and_tiny_frames(mf, width, height, kernel):
    poses = _accelerating_walk(30)
    rng = np.random.default_rng(2)
    depth = rng.uniform(0.2, 5.0, (30, height, width)).astype(np.float32)
    K = np.array([0.8 * width + 1, 0.8 * width + 1, (width - 1) / 2, (height - 1) / 2])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, width, height, window=6,
                                    smooth_len=5, mode="heading", map_kernel=kernel)
    compare_all(M, G, info, pts, ref, K)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("width,height", [(16384, 6), (6, 16384)])
def test_largest_dimension(mf, width, height, kernel):
    """Frames at MF_MAX_DIM in one dimension: 256 column strips of the
    tensor-core kernel, 16 groups of strips / 64 bands of the CUDA cores."""
    poses = _accelerating_walk(12)
    rng = np.random.default_rng(3)
    depth = rng.uniform(0.2, 5.0, (12, height, width)).astype(np.float32)
    f = 0.8 * max(width, height)
    K = np.array([f, f, (width - 1) / 2, (height - 1) / 2])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, width, height, window=6,
                                    smooth_len=5, mode="heading", map_kernel=kernel)
    compare_all(M, G, info, pts, ref, K)
    assert info["n_valid"].sum() > 0


@pytest.mark.parametrize("kernel", KERNELS)
def test_calibration_rescale(mf, kernel):
    """Intrinsics at twice the map resolution; no depth pushed (G = 0)."""
    poses = _accelerating_walk(40)
    K = np.array([520.0, 520.0, 319.5, 239.5])
    M, G, info, pts, ref = run_both(mf, poses, None, K, 320, 240, window=8, smooth_len=5,
                                    mode="heading", calib=(640, 480), map_kernel=kernel)
    compare_all(M, G, info, pts, ref, K)


@pytest.mark.parametrize("mode,storage,kernel", [
    ("accel", "f32", "cuda_cores"), ("heading", "f32", "cuda_cores"),
    ("heading", "bf16", "cuda_cores"), ("accel", "f16", "cuda_cores"),
    ("heading", "f32", "tensor_cores"), ("accel", "bf16", "tensor_cores")])
def test_max_normalised_maps(mf, mode, storage, kernel):
    """Z = the map maximum: each frame's maps divided by its FP32 maximum
    (CUDA cores: a max-only pass, then a pass that renders the scaled map;
    tensor cores: the map, then an in-place division)."""
    w = small_stream()
    M, G, info, pts, ref = run_both(mf, w.poses, w.depth_stack(0, 64), w.K(), 320, 240,
                                    window=8, smooth_len=15, mode=mode, storage=storage,
                                    normalize="max", map_kernel=kernel)
    assert len(info) == ref.n_emitted
    cref = O.Params(320, 240, window=8, smooth_len=15, mode=_mode(mode))
    cst = O.OracleStream(cref)
    cst.push(w.poses, w.depth_stack(0, 64), w.K())
    intr = O.compensated_intrinsics(w.K(), ref.p)
    normalised = kept = ambiguous = 0
    for n in range(ref.n_emitted):
        rinfo, rp, Mr, Gr = ref.frame(n)
        parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}", size=(320, 240))
        if rinfo["n_valid"] == 0:
            assert not M[n].any() and not G[n].any() and info[n]["map_max"] == 0.0
            continue
        mx = cst.frame(n)[2].max()            # the count map's maximum
        # each side compares its own maximum with the floor: inside the band
        # where FP32 and FP64 maxima may fall on opposite sides, both are valid
        if abs(mx - O.NORM_FLOOR) <= 4 * parity.MAP_RTOL * O.NORM_FLOOR:
            ambiguous += 1
            continue
        if mx < O.NORM_FLOOR:                 # left count-normalised
            kept += 1
            parity.check_map(M[n], Mr, storage, f"M frame {n}")
            parity.check_map(G[n], Gr, storage, f"G frame {n}")
            assert abs(float(info[n]["map_max"]) - mx) <= parity.MAP_RTOL * mx + parity.MAP_ATOL
            continue
        normalised += 1
        parity.check_map(M[n], Mr, storage, f"M frame {n}", divisor=mx)
        parity.check_map(G[n], Gr, storage, f"G frame {n}", divisor=mx)
        assert info[n]["map_max"] == 1.0
        x, y = int(info[n]["argmax_x"]), int(info[n]["argmax_y"])
        assert Mr[y, x] >= 1.0 - 4 * parity.MAP_RTOL
        if storage == "f32":
            assert M[n][y, x] == 1.0 and M[n].max() == 1.0
    print(f"\nNORM_MAX {mode} {storage}: normalised {normalised}, kept {kept}, "
          f"ambiguous {ambiguous}")
    assert normalised > 10 and ambiguous <= 1


# ------------------------------------------------------------ edge cases --
def test_degenerate_constant_velocity_is_empty(mf):
    cs = [np.array([0.01 * k, 0.0, 0.05 * k]) for k in range(40)]
    poses = trajectory(cs, [rot_y(0.3)] * 40)
    depth = np.ones((40, 48, 64), np.float32)
    K = np.array([50.0, 50.0, 32.0, 24.0])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, 64, 48, window=8, smooth_len=15)
    assert np.all(info["n_valid"] == 0) and np.all(info["status"] == O.FRAME_EMPTY)
    assert not M.any() and not G.any()
    assert np.all(info["argmax_x"] == -1)


@pytest.mark.parametrize("kernel", KERNELS)
def test_bad_pose_and_invalid_depth(mf, kernel):
    poses = _accelerating_walk(30)
    poses[12, 0, 0] = 1.01
    depth = np.full((30, 48, 64), 2.0, np.float32)
    depth[:, 0, :] = 0.0
    depth[:, 1, :] = np.nan
    depth[:, 2, :] = np.inf
    depth[:, 3, :] = -1.0
    depth[:, 4, :] = 0.5
    depth[:, 5, :] = -np.inf
    depth[:, 6, :] = -0.0
    depth[:, 7, 0::2] = np.float32(2.0 ** -149)      # positive denormals: finite D > 0
    depth[:, 7, 1::2] = np.float32(3.0 * 2.0 ** -140)
    depth[:, 8, 0::2] = -np.float32(2.0 ** -149)     # negative denormals
    depth[:, 8, 1::2] = np.float32(2.0 ** 127)       # near the top of the range
    K = np.array([50.0, 50.0, 32.0, 24.0])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, 64, 48, window=4, smooth_len=3,
                                    map_kernel=kernel)
    compare_all(M, G, info, pts, ref, K)
    assert info["status"][12] == O.FRAME_BAD_POSE and info["valid_mask"][13] == 0b0011
    assert not G[:, :4].any() and np.array_equal(G[:, 4], M[:, 4])
    assert not G[:, 5:7].any() and not G[:, 8, 0::2].any()
    assert np.array_equal(G[:, 7], M[:, 7])          # min(1, d0 / D) = 1 for denormal D > 0


def test_host_pointers_match_device_pointers(mf):
    w = small_stream(n_frames=40)
    d = w.depth_stack(0, 40)
    a = run_both(mf, w.poses, d, w.K(), 320, 240, mode="heading")
    b = run_both(mf, w.poses, d, w.K(), 320, 240, mode="heading", on_host=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def _transfer_case(mf, storage="f32", normalize="count", n=100, width=640, height=480):
    """Poses, depth and intrinsics of a 640x480 heading stream (points in view)."""
    poses = _accelerating_walk(n, width=width)
    rng = np.random.default_rng(7)
    depth = rng.uniform(0.2, 5.0, (n, height, width)).astype(np.float32)
    depth[:, :3, :] = 0.0
    K = np.array([0.8 * width, 0.8 * width, (width - 1) / 2, (height - 1) / 2])
    return poses, torch.from_numpy(depth).to(TDT[storage]), K


def _render(mf, poses, depth, K, pushes, gets, storage="f32", normalize="count", where="device",
            reset_after_first=False):
    """Push/get through the C ABI with inputs and outputs in `where` memory:
    "device", "pinned" (page-locked host) or "pageable" (plain host)."""
    dev = torch.device("cuda", 0)
    dt = TDT[storage]
    n, height, width = depth.shape
    s = mf.MotionFocusStream(width, height, window=8, smooth_len=7, mode="heading",
                             depth_dtype=dt, map_dtype=dt, device=dev, normalize=normalize)
    if where == "device":
        D = depth.to(dev)
        P = torch.from_numpy(poses).to(dev)
        M = torch.empty((n, height, width), dtype=dt, device=dev)
        info = torch.empty(n * 64, dtype=torch.uint8, device=dev)
    else:
        pin = where == "pinned"
        D = depth.clone().pin_memory() if pin else depth.clone()
        P = np.ascontiguousarray(poses)
        M = torch.empty((n, height, width), dtype=dt, pin_memory=pin)
        info = torch.empty(n * 64, dtype=torch.uint8, pin_memory=pin)
    G = torch.empty_like(M)
    if reset_after_first:
        lo, hi = pushes[0]
        mf._mf.mf_push_frames(s.handle, hi - lo, P[lo:hi], D[lo:hi], K)
        mf._mf.mf_reset_stream(s.handle)
    done = 0
    gi = iter(gets)
    for lo, hi in pushes:
        mf._mf.mf_push_frames(s.handle, hi - lo, P[lo:hi], D[lo:hi], K)
        want = next(gi, None)
        if want:
            got = mf._mf.mf_get_maps(s.handle, want, M[done:], G[done:], info[done * 64:], None)
            assert got == want
            done += got
    while done < n - 0:
        got = mf._mf.mf_get_maps(s.handle, n - done, M[done:], G[done:], info[done * 64:], None)
        if got == 0:
            break
        done += got
    torch.cuda.synchronize()
    s.close()
    return (M.float().cpu().numpy(), G.float().cpu().numpy(),
            info.cpu().numpy().view(mf._mf.FRAME_INFO_DTYPE), done)


@pytest.mark.parametrize("storage,normalize", [("f32", "count"), ("bf16", "max")])
def test_host_transfers_in_pieces_match_device_path(mf, storage, normalize):
    """Pinned and pageable host inputs and outputs go through upload pieces,
    a ring of output pieces and two copy streams; every output must equal the
    all-device path bit for bit.  640x480 gives 34-frame pieces; the pushes
    and gets below cut across them, wrap and grow the depth staging ring and
    reuse the output ring many times."""
    poses, depth, K = _transfer_case(mf, storage)
    ref = _render(mf, poses, depth, K, [(0, 100)], [], storage, normalize, "device")
    assert ref[3] == 100 and ref[2]["n_valid"].sum() > 400
    cases = [
        ("pinned", [(0, 100)], [45, 30]),
        ("pinned", [(0, 50), (50, 100)], [45, 0]),
        ("pinned", [(0, 20), (20, 90), (90, 100)], [7, 70, 0]),
        ("pageable", [(0, 60), (60, 100)], [33, 0]),
    ]
    for where, pushes, gets in cases:
        got = _render(mf, poses, depth, K, pushes, gets, storage, normalize, where)
        assert got[3] == 100, (where, pushes)
        for a, b, name in zip(ref[:3], got[:3], ("M", "G", "info")):
            assert np.array_equal(a, b), (where, pushes, gets, name)


def test_reset_with_uploads_in_flight(mf):
    """A reset drops pending pinned uploads; the next pushes reuse the
    staging ring (after growing it) without reading stale planes."""
    poses, depth, K = _transfer_case(mf)
    ref = _render(mf, poses, depth, K, [(0, 100)], [], where="device")
    got = _render(mf, poses, depth, K, [(0, 30), (30, 100)], [0], where="pinned",
                  reset_after_first=True)
    # the dropped push held frames 0..29; after the reset frames restart at 0
    assert got[3] == 100
    for a, b in zip(ref[:3], got[:3]):
        assert np.array_equal(a, b)


def test_split_pushes_and_partial_gets(mf):
    """Frame accounting across pushes and partial mf_get_maps calls."""
    w = small_stream(n_frames=60)
    d = w.depth_stack(0, 60)
    whole = run_both(mf, w.poses, d, w.K(), 320, 240, mode="heading")
    split = run_both(mf, w.poses, d, w.K(), 320, 240, mode="heading",
                     pushes=[(0, 1), (1, 17), (17, 18), (18, 60)], get_chunks=[5, 1, 20])
    for a, b in zip(whole[:4], split[:4]):
        assert np.array_equal(a, b)


def test_batch_local_anchoring(mf):
    """Section 2.2: batches in their own yaw+translation frames, overlap 4."""
    world = walk(WalkerSpec(n_frames=90, seed=9, turns=True)).poses_w2c
    rng = np.random.default_rng(3)
    L, Ov = 24, 4
    batches, start, b = [], 0, 0
    local = []
    while True:
        hi = min(start + L, 90)
        G = np.eye(4)
        if b:
            G[:3, :3] = rot_y(rng.uniform(-3, 3)) @ rot_x(0.1 * rng.normal())
            G[:3, 3] = rng.normal(size=3) * 10
        local.append(np.stack([(O.to4x4(world[k]) @ G)[:3] for k in range(start, hi)]))
        batches.append((sum(len(x) for x in local[:-1]), sum(len(x) for x in local)))
        if hi == 90:
            break
        start = hi - Ov
        b += 1
    poses = np.concatenate(local)
    depth = np.ones((len(poses), 48, 64), np.float32) * 3.0
    K = np.array([50.0, 50.0, 32.0, 24.0])
    M, G, info, pts, ref = run_both(mf, poses, depth, K, 64, 48, window=8, smooth_len=7,
                                    mode="heading", pushes=batches, pose_frame="batch_local",
                                    overlap=Ov)
    assert len(info) == 90
    compare_all(M, G, info, pts, ref, K)


def test_not_ready_and_empty_gets(mf):
    dev = torch.device("cuda", 0)
    s = mf.MotionFocusStream(16, 8, window=2, smooth_len=3, max_pending=10, device=dev)
    P = torch.from_numpy(_accelerating_walk(12)).to(dev)
    assert s.get_maps()[2].shape == (0,)
    s.push(P[:6], None, (10.0, 10.0, 8.0, 4.0))
    with pytest.raises(mf.MFError) as e:
        s.push(P[6:12], None, (10.0, 10.0, 8.0, 4.0))
    assert e.value.status == mf.MF_ERR_NOT_READY
    M, G, info, pts = s.get_maps(4)
    assert len(info) == 4 and s.pending() == 2
    s.push(P[6:12], None, (10.0, 10.0, 8.0, 4.0))
    assert s.pending() == 8 and not G.any()
    s.close()


def test_translation_scale_invariance_bit_exact_on_gpu(mf):
    poses = _accelerating_walk(50)
    scaled = poses.copy()
    scaled[:, :, 3] *= 2.0 ** 7
    depth = np.ones((50, 64, 96), np.float32)
    K = np.array([80.0, 80.0, 48.0, 32.0])
    a = run_both(mf, poses, depth, K, 96, 64, window=8, smooth_len=9)
    b = run_both(mf, scaled, depth, K, 96, 64, window=8, smooth_len=9)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


def test_world_frame_change_and_mirror_symmetry_on_gpu(mf):
    """Two symmetries of the method, checked on the CUDA path itself: a rigid
    change of the world frame (T_t -> T_t G) leaves every output unchanged, and
    mirroring the world about the camera's y-z plane (R -> S R S, t -> S t,
    S = diag(-1, 1, 1)) mirrors the maps about the principal point's column
    (cx = (W-1)/2), both within the map tolerance."""
    poses = _accelerating_walk(60)
    depth = np.ones((60, 64, 96), np.float32)
    K = np.array([80.0, 80.0, 47.5, 31.5])
    base = run_both(mf, poses, depth, K, 96, 64, window=8, smooth_len=9, mode="accel")
    G = np.eye(4)
    G[:3, :3] = rot_y(0.7) @ rot_x(-0.3)
    G[:3, 3] = [12.0, -3.0, 40.0]
    moved = np.stack([(O.to4x4(T) @ G)[:3] for T in poses])
    Sm = np.diag([-1.0, 1.0, 1.0])
    mirrored = poses.copy()
    mirrored[:, :, :3] = Sm @ poses[:, :, :3] @ Sm
    mirrored[:, :, 3] = poses[:, :, 3] @ Sm
    a = run_both(mf, moved, depth, K, 96, 64, window=8, smooth_len=9, mode="accel")
    m = run_both(mf, mirrored, depth, K, 96, 64, window=8, smooth_len=9, mode="accel")
    assert base[2]["n_valid"].sum() > 100
    for n in range(60):
        parity.check_map(a[0][n], base[0][n].astype(np.float64), where=f"world frame M {n}")
        parity.check_map(m[0][n][:, ::-1], base[0][n].astype(np.float64), where=f"mirror M {n}")
        parity.check_map(m[1][n][:, ::-1], base[1][n].astype(np.float64), where=f"mirror G {n}")
    for k in ("n_valid", "valid_mask", "status"):
        assert np.array_equal(a[2][k], base[2][k]) and np.array_equal(m[2][k], base[2][k])


def test_streams_alone_and_interleaved_identical(mf):
    dev = torch.device("cuda", 0)
    wa, wb = small_stream(seed=11, n_frames=30), small_stream(seed=12, n_frames=30)
    da, db = (torch.from_numpy(w.depth_stack(0, 30)).to(dev) for w in (wa, wb))
    pa, pb = (torch.from_numpy(w.poses).to(dev) for w in (wa, wb))

    def alone(p, d, K):
        s = mf.MotionFocusStream(320, 240, mode="heading", device=dev)
        s.push(p, d, K)
        r = s.get_maps()
        s.close()
        return r

    ra, rb = alone(pa, da, wa.K()), alone(pb, db, wb.K())
    sa = mf.MotionFocusStream(320, 240, mode="heading", device=dev)
    sb = mf.MotionFocusStream(320, 240, mode="heading", device=dev)
    for lo, hi in ((0, 10), (10, 30)):
        sa.push(pa[lo:hi], da[lo:hi], wa.K())
        sb.push(pb[lo:hi], db[lo:hi], wb.K())
    xa, xb = sa.get_maps(), sb.get_maps()
    for r, x in ((ra, xa), (rb, xb)):
        assert torch.equal(r[0], x[0]) and torch.equal(r[1], x[1])
        assert np.array_equal(r[2], x[2])
    sa.close()
    sb.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_streams_rendering_concurrently_identical(mf, kernel):
    """Two streams whose map launches run at the same time on their own CUDA
    streams (each stream owns its work counter) render exactly the maps each
    renders alone."""
    dev = torch.device("cuda", 0)
    ws = [hd_stream(seed=s, n_frames=64) for s in (3, 4)]
    rings = [torch.from_numpy(np.stack([w.depth(k) for k in range(w.ring)])).to(dev) for w in ws]
    idx = torch.tensor([k % ws[0].ring for k in range(64)], device=dev)
    depths = [r[idx].contiguous() for r in rings]
    poses = [torch.from_numpy(w.poses).to(dev) for w in ws]
    torch.cuda.synchronize(dev)  # inputs are ready before other CUDA streams read them

    def open_stream(cs):
        return mf.MotionFocusStream(1920, 1080, window=16, smooth_len=15, mode="heading", device=dev,
                                    cuda_stream=cs, map_kernel=kernel)

    alone = []
    for w, p, d in zip(ws, poses, depths):
        s = open_stream(torch.cuda.Stream(dev))
        s.push(p, d, w.K())
        alone.append(s.get_maps())
        s.close()
    torch.cuda.synchronize(dev)
    streams = [open_stream(torch.cuda.Stream(dev)) for _ in ws]
    for s, w, p, d in zip(streams, ws, poses, depths):
        s.push(p, d, w.K())
    outs = []
    for s in streams:  # enqueue both renders before waiting for either
        M = torch.empty((64, 1080, 1920), device=dev)
        G = torch.empty_like(M)
        info = torch.empty(64 * mf._mf.FRAME_INFO_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            assert mf._mf.mf_get_maps(s.handle, 64, M, G, info, None) == 64
        outs.append((M, G, info))
    for s in streams:
        s.torch_stream.synchronize()
        s.close()
    for a, (M, G, info) in zip(alone, outs):
        assert torch.equal(a[0], M) and torch.equal(a[1], G)
        assert np.array_equal(a[2], info.cpu().numpy().view(mf._mf.FRAME_INFO_DTYPE))


# ---------------------------------------------------------- full workload --
# (kernel, storage, workload): the benchmark's default frames (config 2,
# ACCEL on a constant-speed walker: its points are mostly out of view), its
# HEADING leg (every point in view, every unit computes) and ACCEL on a
# walker that speeds up and slows down (the paper's default mode with points
# in view).  The last value is the least fraction of sampled reference map
# values above 1e-3 that each workload must show, so that no comparison of
# (nearly) all-zero maps can pass.
HD_CASES = [("cuda_cores", "f32", "accel"), ("tensor_cores", "f32", "accel"),
            ("tensor_cores", "bf16", "accel"), ("cuda_cores", "f32", "heading"),
            ("cuda_cores", "bf16", "heading"), ("cuda_cores", "f16", "heading"),
            ("cuda_cores", "f32", "accel_in_view"), ("cuda_cores", "bf16", "accel_in_view")]
HD_NONZERO = {"accel": 0.1, "heading": 0.4, "accel_in_view": 0.4}


def hd_workload(name):
    return hd_stream(accel=1.5) if name == "accel_in_view" else hd_stream()


@pytest.mark.parametrize("kernel,storage,workload", HD_CASES)
def test_hd_stream_full_size_sampled(mf, kernel, storage, workload):
    """1920x1080 x 900 frames, window 16: one push and one get of all frames
    (the launch configuration the benchmark times).  Every frame's integers,
    focus and motion points are checked; maps on 256 sampled pixels per frame
    plus each frame's argmax, and three whole frames."""
    w = hd_workload(workload)
    mode = "heading" if workload == "heading" else "accel"
    dev = torch.device("cuda", 0)
    dt = TDT[storage]
    ring = torch.from_numpy(np.stack([w.depth(k) for k in range(w.ring)])).to(dev).to(dt)
    idx = torch.tensor([k % w.ring for k in range(w.n_frames)], device=dev)
    depth = ring[idx].contiguous()
    s = mf.MotionFocusStream(w.width, w.height, window=w.window, smooth_len=w.smooth_len,
                             device=dev, depth_dtype=dt, map_dtype=dt, map_kernel=kernel, mode=mode)
    s.push(torch.from_numpy(w.poses).to(dev), depth, w.K())
    M, G, info, pts = s.get_maps()
    s.close()
    del depth
    ref = O.OracleStream(O.Params(w.width, w.height, window=w.window, smooth_len=w.smooth_len,
                                  mode=_mode(mode)))
    ref.push(w.poses, None, w.K())
    intr = O.compensated_intrinsics(w.K(), ref.p)
    rng = np.random.default_rng(5)
    frames = range(w.n_frames)
    ys = rng.integers(0, w.height, 256)
    xs = rng.integers(0, w.width, 256)
    yt, xt = torch.from_numpy(ys).to(dev), torch.from_numpy(xs).to(dev)
    Ms = M[:, yt, xt].double().cpu().numpy()
    Gs = G[:, yt, xt].double().cpu().numpy()
    ringh = ring.double().cpu().numpy()
    refs = []
    for n in frames:
        rinfo, rp, _, _ = ref.frame(n, full_maps=False)
        parity.check_frame(info[n], pts[n], rinfo, rp, intr, where=f"frame {n}",
                           size=(w.width, w.height))
        Mr = O.focus_map(rp, w.width, w.height, xs, ys)
        refs.append(Mr)
        parity.check_map(Ms[n], Mr, storage, where=f"M frame {n}")
        Gr = O.guided_depth(Mr, ringh[n % w.ring][ys, xs], 1.0)
        parity.check_map(Gs[n], Gr, storage, where=f"G frame {n}")
        if rinfo["n_valid"]:
            ax, ay = int(info[n]["argmax_x"]), int(info[n]["argmax_y"])
            m_at = O.focus_map(rp, w.width, w.height, np.array([ax]), np.array([ay]))[0]
            assert abs(float(info[n]["map_max"]) - m_at) <= 1e-5 * m_at + 1e-10
            if storage == "f32":
                assert float(M[n, ay, ax]) == float(info[n]["map_max"])
    assert info["n_valid"].sum() > 5000
    got = parity.assert_not_vacuous(np.concatenate(refs), HD_NONZERO[workload], where=workload)
    print(f"\nHD_SAMPLED {kernel} {storage} {workload}: {got:.3f} of sampled values > 1e-3")
    # three whole frames against the full FP64 map (values and argmax)
    for n in (100, 451, 899):
        rinfo, rp, _, _ = ref.frame(n, full_maps=False)
        Mr = O.focus_map(rp, w.width, w.height)
        parity.check_map(M[n].double().cpu().numpy(), Mr, storage, where=f"full M frame {n}")
        if storage == "f32":
            parity.check_argmax(info[n], Mr, rinfo["n_valid"], where=f"argmax {n}")
        Gr = O.guided_depth(Mr, ringh[n % w.ring], 1.0)
        parity.check_map(G[n].double().cpu().numpy(), Gr, storage, where=f"full G frame {n}")


@pytest.mark.parametrize("window,storage,normalize", [
    (16, "f32", "count"), (8, "f32", "count"), (24, "f32", "count"), (16, "bf16", "count"),
    (24, "f16", "count"), (16, "f32", "max")])
def test_default_kernel_is_the_cuda_core_kernel(mf, window, storage, normalize):
    """With no kernel flag the library runs the CUDA-core map kernel (the map
    is HBM-bound work), and its maps are the forced kernel's, bit for bit
    (mf_stats.last_map_kernel reports which one ran)."""
    w = small_stream()
    dev = torch.device("cuda", 0)
    dt = TDT[storage]
    poses = torch.from_numpy(np.ascontiguousarray(w.poses[:48])).to(dev)
    depth = torch.from_numpy(np.ascontiguousarray(w.depth_stack(0, 48))).to(dt).to(dev)
    out = {}
    for kernel in ("auto", "cuda_cores"):
        s = mf.MotionFocusStream(320, 240, window=window, smooth_len=15, depth_dtype=dt, map_dtype=dt,
                                 device=dev, normalize=normalize, map_kernel=kernel)
        s.push(poses, depth, w.K())
        M, G, info, _ = s.get_maps()
        assert int(s.stats().last_map_kernel) == mf._mf.MF_FLAG_MAP_CUDA_CORES, kernel
        out[kernel] = (M.cpu(), G.cpu(), info)
        s.close()
    assert torch.equal(out["auto"][0], out["cuda_cores"][0]) and torch.equal(out["auto"][1], out["cuda_cores"][1])
    assert np.array_equal(out["auto"][2], out["cuda_cores"][2])
