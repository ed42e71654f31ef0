"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form
(principal point, fx*tan(theta)), a property that the least-squares fit or
Eq. 7 must have, an invariant, or a degenerate case.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.posegen import rot_x, rot_y, trajectory

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run(poses, p, K=(260.0, 260.0, 160.0, 120.0), depth=None):
    st = O.OracleStream(p)
    st.push(poses, depth, K)
    return st


# --------------------------------------------------------------- Eqs. 2-3 --
def test_stencils_reduce_to_paper_differences():
    """Golden: K=3 ACCEL is Eq. 3's (1,-2,1); K=2 HEADING is Eq. 2's (1,-1)."""
    with open(os.path.join(GOLDEN, "stencils.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for mode, k, *w in rows:
        m = O.MODE_ACCEL if mode == "ACCEL" else O.MODE_HEADING
        assert O.ls_weights_exact(int(k), m) == [Fraction(x) for x in w]
        assert list(O.ls_weights(int(k), m)) == [float(x) for x in w]


@pytest.mark.parametrize("K", list(range(3, 34)))
def test_stencil_moments_and_least_squares_shape(K):
    """The fit reproduces quadratics exactly and its weights are a quadratic in tau.

    Moment conditions sum_k w_k tau_k^e = (0, 0, 2) (ACCEL) / (0, 1, 0)
    (HEADING) state that any exact quadratic trajectory yields its true
    second / first derivative; weights lying in the span of (1, tau, tau^2)
    is the normal-equation (minimum-norm) condition.  Together they fix the
    least-squares weights uniquely.
    """
    taus = [Fraction(-k) for k in range(K)]
    for mode, want in ((O.MODE_ACCEL, (0, 0, 2)), (O.MODE_HEADING, (0, 1, 0))):
        w = O.ls_weights_exact(K, mode)
        for e in range(3):
            assert sum(wk * t ** e for wk, t in zip(w, taus)) == want[e]
        # third finite differences of w over tau vanish <=> w is quadratic in tau
        for k in range(K - 3):
            assert w[k] - 3 * w[k + 1] + 3 * w[k + 2] - w[k + 3] == 0


def test_stencil_rejects_underdetermined():
    with pytest.raises(ValueError):
        O.ls_weights_exact(2, O.MODE_ACCEL)
    with pytest.raises(ValueError):
        O.ls_weights_exact(1, O.MODE_HEADING)


# ------------------------------------------------------------------ Eq. 1 --
def test_camera_centre_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(20):
        r = rot_y(rng.uniform(-3, 3)) @ rot_x(rng.uniform(-1, 1))
        c = rng.normal(size=3) * 10
        T = trajectory([c], [r])[0]
        assert np.allclose(O.camera_centre(T), c, rtol=0, atol=1e-12)


def test_rigid_check():
    T = trajectory([np.zeros(3)])[0]
    assert O.is_rigid(T)
    T2 = T.copy()
    T2[0, 0] = 1.0 + 1e-5
    assert not O.is_rigid(T2)
    T3 = T.copy()
    T3[1, 3] = np.nan
    assert not O.is_rigid(T3)


# -------------------------------------------------------------- Eqs. 4-6 --
def _const_velocity(n, vel, rot=np.eye(3), start=(0.0, 0.0, 0.0)):
    cs = [np.asarray(start) + k * np.asarray(vel, dtype=np.float64) for k in range(n)]
    return trajectory(cs, [rot] * n)


@pytest.mark.parametrize("K", [2, 3, 7, 15])
def test_heading_forward_motion_hits_principal_point(K):
    p = O.Params(320, 240, window=8, smooth_len=K, mode=O.MODE_HEADING)
    st = run(_const_velocity(40, (0, 0, 0.05)), p)
    pts = st.points(39)
    assert pts.n_valid == 8
    assert np.all(pts.u == 160.0) and np.all(pts.v == 120.0)
    fv, u, v, x, y = O.focus_pixel(pts, 320, 240)
    assert (fv, u, v, x, y) == (1, 160.0, 120.0, 160, 120)


@pytest.mark.parametrize("K", [3, 5, 15])
def test_accel_forward_acceleration_hits_principal_point(K):
    p = O.Params(320, 240, window=8, smooth_len=K, mode=O.MODE_ACCEL)
    cs = [np.array([0.0, 0.0, 0.5 * 0.01 * k * k]) for k in range(40)]
    st = run(trajectory(cs), p)
    pts = st.points(39)
    assert pts.n_valid == 8
    np.testing.assert_allclose(pts.u, 160.0, atol=1e-9)
    np.testing.assert_allclose(pts.v, 120.0, atol=1e-9)
    # the constant second difference (Eq. 3) is 0.01 m/frame^2 along z
    np.testing.assert_allclose(pts.d_cam[:, 2], 0.01, rtol=1e-9)


@pytest.mark.parametrize("theta_deg", [-30.0, -7.5, 4.0, 20.0])
def test_yawed_camera_moves_focus_by_fx_tan_theta(theta_deg):
    """Camera yawed by theta, moving along world +z: u = cx - fx tan(theta)."""
    th = math.radians(theta_deg)
    p = O.Params(320, 240, window=4, smooth_len=3, mode=O.MODE_HEADING)
    st = run(_const_velocity(20, (0, 0, 0.05), rot=rot_y(th)), p)
    pts = st.points(19)
    np.testing.assert_allclose(pts.u, 160.0 - 260.0 * math.tan(th), atol=1e-9)
    np.testing.assert_allclose(pts.v, 120.0, atol=1e-9)


@pytest.mark.parametrize("phi_deg", [-10.0, 3.0, 12.0])
def test_pitched_camera_moves_focus_by_fy_tan_phi(phi_deg):
    """Camera pitched by phi about x (y down), moving along +z: v = cy + fy tan(phi)."""
    ph = math.radians(phi_deg)
    p = O.Params(320, 240, window=4, smooth_len=3, mode=O.MODE_HEADING)
    st = run(_const_velocity(20, (0, 0, 0.05), rot=rot_x(ph)), p)
    pts = st.points(19)
    np.testing.assert_allclose(pts.v, 120.0 + 260.0 * math.tan(ph), atol=1e-9)
    np.testing.assert_allclose(pts.u, 160.0, atol=1e-9)


def test_intrinsics_rescaled_to_map_resolution():
    """K calibrated at 640x480, map at 320x240: the principal ray lands on (cx', cy')."""
    p = O.Params(320, 240, window=4, smooth_len=3, mode=O.MODE_HEADING,
                 calib_width=640, calib_height=480)
    st = run(_const_velocity(20, (0, 0, 0.05)), p, K=(520.0, 520.0, 319.5, 239.5))
    pts = st.points(19)
    assert np.all(pts.u == 159.5) and np.all(pts.v == 119.5)
    # a yawed camera checks that fx is halved as well
    st = run(_const_velocity(20, (0, 0, 0.05), rot=rot_y(0.1)), p, K=(520.0, 520.0, 319.5, 239.5))
    np.testing.assert_allclose(st.points(19).u, 159.5 - 260.0 * math.tan(0.1), atol=1e-9)


# ------------------------------------------------------------- degenerate --
def test_accel_constant_velocity_is_empty():
    p = O.Params(64, 48, window=8, smooth_len=15, mode=O.MODE_ACCEL)
    st = run(_const_velocity(60, (0.01, -0.002, 0.045), rot=rot_y(0.3), start=(5, 1, -3)), p,
             K=(50.0, 50.0, 32.0, 24.0), depth=np.ones((60, 48, 64)))
    for n in (20, 40, 59):
        info, pts, M, G = st.frame(n)
        assert info["n_valid"] == 0 and info["status"] == O.FRAME_EMPTY
        assert info["argmax_x"] == -1 and info["map_max"] == 0.0
        assert not M.any() and not G.any()


def test_stationary_camera_is_empty():
    rots = [rot_y(0.05 * k) @ rot_x(0.01 * k) for k in range(30)]
    cs = [np.array([3.0, -1.0, 7.0])] * 30
    for mode in (O.MODE_ACCEL, O.MODE_HEADING):
        p = O.Params(64, 48, window=8, smooth_len=5, mode=mode)
        st = run(trajectory(cs, rots), p, K=(50.0, 50.0, 32.0, 24.0))
        for n in range(30):
            assert st.points(n).n_valid == 0


@pytest.mark.parametrize("W,K", [(8, 15), (4, 3), (1, 2), (32, 33)])
def test_short_history_gives_fewer_points(W, K):
    mode = O.MODE_HEADING if K == 2 else O.MODE_ACCEL
    cs = [np.array([0.0, 0.0, 0.05 * k + 0.001 * k * k]) for k in range(W + K + 5)]
    p = O.Params(64, 48, window=W, smooth_len=K, mode=mode)
    st = run(trajectory(cs), p, K=(50.0, 50.0, 32.0, 24.0))
    for n in range(W + K + 5):
        want = max(0, min(W, n - K + 2))
        pts = st.points(n)
        assert pts.n_valid == want
        # the valid slots are the newest ones
        assert pts.valid_mask == ((1 << want) - 1) << (W - want)


def test_bad_pose_frame_and_windows():
    cs = [np.array([0.0, 0.0, 0.05 * k + 0.001 * k * k]) for k in range(30)]
    poses = trajectory(cs)
    poses[12, 0, 0] = 1.01  # not a rotation
    p = O.Params(64, 48, window=4, smooth_len=3)
    st = run(poses, p, K=(50.0, 50.0, 32.0, 24.0))
    assert st.points(12).status == O.FRAME_BAD_POSE
    # slot s of frame n is point i = n - 3 + s, fitted on poses i-2..i; only
    # the points whose 3-sample fit avoids frame 12 stay valid
    assert st.points(13).valid_mask == 0b0011
    assert st.points(14).valid_mask == 0b0001
    assert st.points(15).valid_mask == 0b1000
    assert st.points(17).valid_mask == 0b1110


# ------------------------------------------------------------------ Eq. 7 --
def _single_point_frame():
    """HEADING, K=2: frame 1 has exactly one valid point (the newest)."""
    th, ph = 0.07, -0.04
    p = O.Params(48, 36, window=4, smooth_len=2, mode=O.MODE_HEADING)
    st = run(_const_velocity(2, (0, 0, 0.05), rot=rot_y(th) @ rot_x(ph)), p,
             K=(40.0, 40.0, 23.5, 17.5), depth=np.full((2, 36, 48), 2.0))
    return st


def test_single_point_map_closed_form_and_argmax():
    st = _single_point_frame()
    info, pts, M, G = st.frame(1)
    assert info["n_valid"] == 1
    s = 3
    # one point: s = 1, sigma = sigma_rel * fx
    assert pts.s[s] == 1.0 and pts.sigma[s] == 0.1 * 40.0
    u, v = pts.u[s], pts.v[s]
    x, y = 10, 20
    want = math.exp(-((x - u) ** 2 + (y - v) ** 2) / (2 * 4.0 ** 2))
    assert abs(M[y, x] - want) <= 1e-15
    # argmax is the pixel nearest (u, v)
    assert (info["argmax_x"], info["argmax_y"]) == (int(round(u)), int(round(v)))
    assert info["map_max"] == M.max() <= 1.0


def test_max_normalised_single_point_closed_form():
    """Z = the map maximum: one point's map is exp(-(r^2 - r_min^2) / (2 sigma^2)),
    r_min the distance from the point to its nearest pixel, so it peaks at 1."""
    th, ph = 0.07, -0.04
    p = O.Params(48, 36, window=4, smooth_len=2, mode=O.MODE_HEADING, normalize="max")
    st = run(_const_velocity(2, (0, 0, 0.05), rot=rot_y(th) @ rot_x(ph)), p,
             K=(40.0, 40.0, 23.5, 17.5), depth=np.full((2, 36, 48), 0.5))
    info, pts, M, G = st.frame(1)
    s = 3
    u, v, sig = pts.u[s], pts.v[s], pts.sigma[s]
    xn, yn = int(round(u)), int(round(v))
    r2min = (xn - u) ** 2 + (yn - v) ** 2
    assert r2min > 0.01          # off-pixel: the count-normalised peak is below 1
    for x, y in ((10, 20), (xn, yn), (xn + 3, yn - 2)):
        want = math.exp(-(((x - u) ** 2 + (y - v) ** 2) - r2min) / (2 * sig ** 2))
        assert abs(M[y, x] - want) <= 1e-14
    assert M.max() == 1.0 and M[yn, xn] == 1.0
    assert info["map_max"] == 1.0 and (info["argmax_x"], info["argmax_y"]) == (xn, yn)
    # depth 0.5 < d0 = 1: motion-guided depth equals the normalised map
    np.testing.assert_array_equal(G, M)


@pytest.mark.parametrize("u_out,normalised", [(-15.0, True), (-27.0, False)])
def test_max_normalisation_floor(u_out, normalised):
    """One point left of the image (yaw puts it at u = cx - fx tan(theta)):
    15 px out its map still peaks at exp(-15^2 / (2 sigma^2)) >= 2^-20 and is
    rescaled to 1; 27 px out the peak is below 2^-20 and the count map stays."""
    fx, cx = 40.0, 23.5
    th = math.atan((cx - u_out) / fx)
    maps = {}
    for norm in ("count", "max"):
        p = O.Params(48, 36, window=4, smooth_len=2, mode=O.MODE_HEADING, normalize=norm)
        st = run(_const_velocity(2, (0, 0, 0.05), rot=rot_y(th)), p, K=(fx, fx, cx, 17.5),
                 depth=np.full((2, 36, 48), 2.0))
        maps[norm] = st.frame(1)
    (ic, pc, Mc, _), (im, _, Mm, _) = maps["count"], maps["max"]
    assert ic["n_valid"] == 1 and abs(pc.u[3] - u_out) < 1e-9
    # nearest pixel: column 0, and the lowest row closest to v (v = cy = 17.5)
    dys = np.abs(np.arange(36) - pc.v[3])
    y0 = int(np.argmin(dys))
    peak = math.exp(-(u_out ** 2 + dys[y0] ** 2) / (2 * (0.1 * fx) ** 2))
    assert abs(Mc.max() - peak) <= 1e-12 * peak
    assert (ic["argmax_x"], ic["argmax_y"]) == (0, y0) == (0, 17)
    if normalised:
        assert Mc.max() >= O.NORM_FLOOR and Mm.max() == 1.0 and im["map_max"] == 1.0
    else:
        assert Mc.max() < O.NORM_FLOOR
        np.testing.assert_array_equal(Mm, Mc)
        assert im["map_max"] == ic["map_max"] == Mc.max()


def test_max_normalised_is_a_rescaled_count_map():
    """The two normalisations differ by one positive factor per frame; empty
    frames stay all zero under both."""
    from synth import small_stream
    w = small_stream()
    maps = {}
    for norm in ("count", "max"):
        p = O.Params(96, 72, window=8, smooth_len=15, mode=O.MODE_ACCEL, normalize=norm)
        st = run(w.poses[:24], p, K=w.K() * np.array([0.3, 0.3, 0.3, 0.3]),
                 depth=np.full((24, 72, 96), 3.0))
        maps[norm] = [st.frame(n) for n in (0, 1, 20, 23)]
    for (ic, _, Mc, Gc), (im, _, Mm, Gm) in zip(maps["count"], maps["max"]):
        assert ic["n_valid"] == im["n_valid"]
        if ic["n_valid"] == 0:
            assert not Mc.any() and not Mm.any() and im["map_max"] == 0.0
            continue
        c = Mc.max()
        if c < O.NORM_FLOOR:
            np.testing.assert_array_equal(Mm, Mc)
            continue
        assert 0.0 < c <= 1.0 and Mm.max() == 1.0
        np.testing.assert_allclose(Mm * c, Mc, rtol=1e-15, atol=0)
        np.testing.assert_allclose(Gm * c, Gc, rtol=1e-15, atol=0)
        assert (im["argmax_x"], im["argmax_y"]) == (ic["argmax_x"], ic["argmax_y"])
    assert any(i["n_valid"] > 0 for i, *_ in maps["max"])
    assert any(i["n_valid"] == 0 for i, *_ in maps["max"])


def test_brute_force_tiny_two_points():
    """4x3 map from two hand-placed points with sigma = 1 (values by hand)."""
    pts = O.FramePoints(0, 0, np.array([0.0, 3.0]), np.array([0.0, 2.0]),
                        np.array([1.0, 1.0]), np.array([1.0, 1.0]),
                        np.array([True, True]), np.zeros((2, 3)))
    M = O.focus_map(pts, 4, 3)
    e = math.exp
    assert M.shape == (3, 4)
    assert abs(M[0, 0] - (1 + e(-6.5)) / 2) < 1e-16
    assert abs(M[2, 3] - (1 + e(-6.5)) / 2) < 1e-16
    assert abs(M[1, 1] - (e(-1.0) + e(-2.5)) / 2) < 1e-16
    assert abs(M[0, 3] - (e(-4.5) + e(-2.0)) / 2) < 1e-16
    # sampled evaluation agrees with the full map
    xs, ys = np.array([0, 3, 1, 3]), np.array([0, 2, 1, 0])
    np.testing.assert_array_equal(O.focus_map(pts, 4, 3, xs, ys), M[ys, xs])


def test_map_range_and_guided_depth():
    from synth import small_stream
    w = small_stream()
    p = O.Params(320, 240, window=8, smooth_len=15, mode=O.MODE_HEADING)
    st = run(w.poses[:30], p, K=w.K(), depth=w.depth_stack(0, 30))
    for n in (16, 29):
        info, pts, M, G = st.frame(n)
        assert info["n_valid"] > 0
        assert M.min() >= 0.0 and M.max() <= 1.0 and M.max() > 0.1
        assert np.all(G >= 0.0) and np.all(G <= M)
        D = st.depth[n]
        bad = ~(np.isfinite(D) & (D > 0))
        assert bad.any() and np.all(G[bad] == 0.0)


def test_guided_depth_closed_forms():
    M = np.full((2, 3), 0.5)
    D = np.array([[4.0, 1.0, 0.5], [0.0, np.nan, np.inf]])
    G = O.guided_depth(M, D, 1.0)
    np.testing.assert_array_equal(G, [[0.125, 0.5, 0.5], [0.0, 0.0, 0.0]])
    np.testing.assert_array_equal(O.guided_depth(M, np.full((2, 3), -1.0), 1.0), 0.0)


# ------------------------------------------------------------- invariants --
def _noisy_walk(n=40, seed=3):
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    for k in range(n):
        t = k / 30.0
        cs.append(np.array([0.3 * math.sin(1.3 * t), -0.05 * t * t, 1.4 * t + 0.2 * t * t])
                  + rng.normal(0, 0.002, 3))
        rs.append(rot_y(0.15 * math.sin(3 * t)) @ rot_x(0.05 * math.sin(12 * t)))
    return trajectory(cs, rs)


@pytest.mark.parametrize("mode", [O.MODE_ACCEL, O.MODE_HEADING])
@pytest.mark.parametrize("k", [-3, 5])
def test_translation_scale_invariance_is_bit_exact(mode, k):
    poses = _noisy_walk()
    scaled = poses.copy()
    scaled[:, :, 3] *= 2.0 ** k
    p = O.Params(96, 72, window=8, smooth_len=7, mode=mode)
    a = run(poses, p, K=(80.0, 80.0, 48.0, 36.0))
    b = run(scaled, p, K=(80.0, 80.0, 48.0, 36.0))
    for n in range(10, 40, 7):
        pa, pb = a.points(n), b.points(n)
        assert pa.n_valid > 0
        assert pa.valid_mask == pb.valid_mask
        assert np.array_equal(pa.u, pb.u) and np.array_equal(pa.v, pb.v)
        assert np.array_equal(pa.sigma, pb.sigma)
        assert np.array_equal(O.focus_map(pa, 96, 72), O.focus_map(pb, 96, 72))


def test_world_frame_invariance():
    """T_t -> T_t G for a rigid G (any yaw/pitch/roll and offset) changes nothing."""
    poses = _noisy_walk()
    G = np.eye(4)
    G[:3, :3] = rot_y(1.1) @ rot_x(-0.4) @ rot_y(0.3)
    G[:3, 3] = [12.0, -3.0, 40.0]
    moved = np.stack([(O.to4x4(T) @ G)[:3] for T in poses])
    p = O.Params(96, 72, window=8, smooth_len=7, mode=O.MODE_ACCEL)
    a = run(poses, p, K=(80.0, 80.0, 48.0, 36.0))
    b = run(moved, p, K=(80.0, 80.0, 48.0, 36.0))
    for n in range(10, 40, 5):
        pa, pb = a.points(n), b.points(n)
        assert pa.valid_mask == pb.valid_mask
        np.testing.assert_allclose(pa.u, pb.u, atol=1e-6)
        np.testing.assert_allclose(pa.v, pb.v, atol=1e-6)
        np.testing.assert_allclose(pa.sigma, pb.sigma, rtol=1e-9)


def test_mirror_symmetric_trajectory_gives_mirrored_map():
    """Reflect the world in x (S = diag(-1,1,1)), principal point on the axis."""
    poses = _noisy_walk()
    S = np.diag([-1.0, 1.0, 1.0])
    mirrored = np.stack([np.concatenate([S @ T[:, :3] @ S, (S @ T[:, 3])[:, None]], 1)
                         for T in poses])
    width, height = 96, 72
    K = (80.0, 80.0, (width - 1) / 2.0, 36.0)
    p = O.Params(width, height, window=8, smooth_len=7, mode=O.MODE_HEADING)
    a = run(poses, p, K=K)
    b = run(mirrored, p, K=K)
    for n in (20, 39):
        Ma = O.focus_map(a.points(n), width, height)
        Mb = O.focus_map(b.points(n), width, height)
        assert Ma.max() > 1e-3
        np.testing.assert_allclose(Mb, Ma[:, ::-1], rtol=1e-9, atol=1e-300)


# -------------------------------------------------- qualitative (Sec. 2.4) --
def test_accelerating_right_turn_moves_focus_right():
    cs, rs = [], []
    psi, speed, pos = 0.0, 0.04, np.zeros(3)
    for k in range(40):
        cs.append(pos.copy())
        rs.append(np.eye(3))
        psi += 0.01
        speed += 0.001
        pos = pos + speed * np.array([math.sin(psi), 0.0, math.cos(psi)])
    p = O.Params(320, 240, window=4, smooth_len=5, mode=O.MODE_ACCEL)
    pts = run(trajectory(cs, rs), p).points(39)
    assert pts.n_valid == 4 and np.all(pts.u > 160.0)


def test_ascending_moves_focus_up():
    cs = [np.array([0.0, -0.0005 * k * k, 0.05 * k + 0.0005 * k * k]) for k in range(30)]
    for mode in (O.MODE_ACCEL, O.MODE_HEADING):
        p = O.Params(320, 240, window=4, smooth_len=5, mode=mode)
        pts = run(trajectory(cs), p).points(29)
        assert pts.n_valid == 4 and np.all(pts.v < 120.0)


def test_head_yaw_offset_keeps_focus_on_body_heading():
    """Head yawed 15 deg left of a straight body path: the focus stays on the path."""
    th = math.radians(-15.0)
    p = O.Params(320, 240, window=8, smooth_len=7, mode=O.MODE_HEADING)
    st = run(_const_velocity(30, (0, 0, 0.05), rot=rot_y(th)), p)
    pts = st.points(29)
    # the body heading (+z) projects to u = cx - fx tan(theta), right of centre
    np.testing.assert_allclose(pts.u, 160.0 - 260.0 * math.tan(th), atol=1e-9)
    assert np.all(pts.u > 160.0)


# ------------------------------------------------ further structural pins --
def test_all_points_projected_into_current_frame():
    """Fig. 4: every motion vector is rotated by R_n of the current frame n.

    A camera whose yaw changes every frame while it moves along +z: in HEADING
    mode every point of frame n lands on cx - fx tan(theta_n), not on the
    yaw of its own frame i.
    """
    thetas = [0.02 * k for k in range(20)]
    cs = [np.array([0.0, 0.0, 0.05 * k]) for k in range(20)]
    p = O.Params(320, 240, window=6, smooth_len=2, mode=O.MODE_HEADING)
    st = run(trajectory(cs, [rot_y(t) for t in thetas]), p)
    for n in (10, 19):
        np.testing.assert_allclose(st.points(n).u, 160.0 - 260.0 * math.tan(thetas[n]),
                                   atol=1e-9)


def test_magnitude_scaling_and_clamp():
    """s_i = clamp(|d_i| / mean|d|, 0.25, 4) and sigma_i = 0.1 fx s_i."""
    speeds = [0.01, 0.02, 0.03, 0.10]            # m/frame of the 4 newest steps
    zs = [0.0]
    for v in [0.05] * 6 + speeds:
        zs.append(zs[-1] + v)
    p = O.Params(320, 240, window=4, smooth_len=2, mode=O.MODE_HEADING)
    st = run(trajectory([np.array([0.0, 0.0, z]) for z in zs]), p)
    pts = st.points(len(zs) - 1)
    np.testing.assert_allclose(pts.s, [0.25, 0.5, 0.75, 2.5], rtol=1e-12)
    np.testing.assert_allclose(pts.sigma, 0.1 * 260.0 * pts.s, rtol=1e-15)
    speeds = [0.01] * 7 + [1.0]
    zs = [0.0]
    for v in [0.05] * 3 + speeds:
        zs.append(zs[-1] + v)
    p = O.Params(320, 240, window=8, smooth_len=2, mode=O.MODE_HEADING)
    pts = run(trajectory([np.array([0.0, 0.0, z]) for z in zs]), p).points(len(zs) - 1)
    np.testing.assert_allclose(pts.s, [0.25] * 7 + [4.0], rtol=0)


@pytest.mark.parametrize("ratio,valid", [(0.0, False), (5e-4, False), (2e-3, True)])
def test_lateral_acceleration_threshold(ratio, valid):
    """|d_z| must exceed 1e-3 |d|: a purely sideways acceleration is no point."""
    a = 0.004
    cs = [np.array([0.5 * a * k * k, 0.0, 0.05 * k + 0.5 * ratio * a * k * k]) for k in range(12)]
    p = O.Params(320, 240, window=2, smooth_len=3, mode=O.MODE_ACCEL)
    pts = run(trajectory(cs), p).points(11)
    assert bool(pts.valid.all()) is valid and bool(pts.valid.any()) is valid


def test_argmax_ties_go_to_lowest_index():
    pts = O.FramePoints(0, 0, np.array([0.0, 3.0]), np.array([0.0, 2.0]),
                        np.array([1.0, 1.0]), np.array([1.0, 1.0]),
                        np.array([True, True]), np.zeros((2, 3)))
    M = O.focus_map(pts, 4, 3)
    assert M[0, 0] == M[2, 3] == M.max()
    assert O.map_argmax(M, 2) == (0, 0, M[0, 0])


def test_focus_pixel_rounds_half_to_even_and_clips():
    def fp(u, v, ok=True):
        pts = O.FramePoints(0, 0, np.array([0.0, u]), np.array([0.0, v]), np.ones(2), np.ones(2),
                            np.array([False, ok]), np.zeros((2, 3)))
        return O.focus_pixel(pts, 320, 240)
    assert fp(150.5, 10.5)[3:] == (150, 10)
    assert fp(151.5, 11.5)[3:] == (152, 12)
    assert fp(-0.4, 239.4)[3:] == (0, 239)
    assert fp(-0.6, 5.0)[3:] == (-1, -1)
    assert fp(319.6, 5.0)[3:] == (-1, -1)
    assert fp(10.0, 10.0, ok=False) == (0, 0.0, 0.0, -1, -1)
