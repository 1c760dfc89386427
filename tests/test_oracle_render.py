"""Pins of the FP64 render oracle against facts that do not come from the oracle.

Each test targets a plausible mistake: a wrong rotation convention, a
transposed Jacobian, a dropped term in the EWA covariance, an off-by-one in
the pixel-centre convention, a wrong stop rule, a wrong gradient.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from oracle.raster import Options, _t
from paper_2505_18992_gb300 import scenes


def _one(mean, scale, quat, opac, color, W=33, H=25, f=40.0, T=None, **kw):
    T = np.eye(4)[None] if T is None else T
    return oracle.render(np.array([mean], np.float64), np.array([scale], np.float64),
                         np.array([quat], np.float64), np.array([opac], np.float64),
                         np.array([color], np.float64), T, f, f, W / 2.0, H / 2.0, W, H, **kw)


def test_quat_rotation_matches_scipy():
    rng = np.random.default_rng(0)
    q = rng.normal(size=(50, 4))
    R = oracle.quat_to_rotmat(_t(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy is (x,y,z,w)
    assert np.abs(R - ref).max() < 1e-13


def test_single_isotropic_gaussian_closed_form():
    # an isotropic Gaussian on the optical axis: Sigma' = ((f s / z)^2 + 0.3) I
    W, H, f, z, s, o = 33, 25, 40.0, 2.0, 0.05, 0.8
    col = (0.2, 0.5, 0.9)
    out = _one((0, 0, z), (s, s, s), (1, 0, 0, 0), o, col, W, H, f)
    var = (f * s / z) ** 2 + 0.3
    xs = np.arange(W) + 0.5 - W / 2.0
    ys = np.arange(H) + 0.5 - H / 2.0
    g = o * np.exp(-(xs[None, :] ** 2 + ys[:, None] ** 2) / (2 * var))
    a = np.where(g >= 1 / 255, g, 0.0)
    assert np.abs(out["alpha"][0] - a).max() < 1e-14
    for ch in range(3):
        assert np.abs(out["rgb"][0, ch] - a * col[ch]).max() < 1e-14
    assert np.abs(out["depth"][0] - a * z).max() < 1e-14
    assert np.array_equal(out["n_contrib"][0], (g >= 1 / 255).astype(np.int64))
    # peak lands on the pixel whose centre is closest to (cx, cy)
    j, i = np.unravel_index(np.argmax(out["alpha"][0]), (H, W))
    assert (i, j) == (W // 2, H // 2)


def test_ewa_covariance_against_numerical_jacobian():
    # Sigma' - eps I must equal J_num Sigma_c J_num^T, J_num = finite-difference
    # Jacobian of the pinhole projection, Sigma_c built with scipy rotations.
    rng = np.random.default_rng(1)
    f, cx, cy = 500.0, 320.0, 240.0
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec(rng.normal(size=3) * 0.3).as_matrix()
    T[:3, 3] = rng.normal(size=3) * 0.2 + np.array([0, 0, 0.5])
    means = rng.normal(size=(20, 3)) * 0.5 + np.array([0, 0, 3.0])
    scales = np.exp(rng.uniform(-5, -2, size=(20, 3)))
    quats = rng.normal(size=(20, 4))
    t = _t
    pr = oracle.project(t(means), t(scales), t(quats), t(T), f, f, cx, cy, Options())

    def pi(p):
        return np.array([f * p[0] / p[2] + cx, f * p[1] / p[2] + cy])

    for i in range(20):
        p = T[:3, :3] @ means[i] + T[:3, 3]
        h = 1e-6
        Jn = np.stack([(pi(p + h * e) - pi(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
        Rq = Rotation.from_quat(quats[i, [1, 2, 3, 0]]).as_matrix()
        Sc = T[:3, :3] @ Rq @ np.diag(scales[i] ** 2) @ Rq.T @ T[:3, :3].T
        ref = Jn @ Sc @ Jn.T + 0.3 * np.eye(2)
        A, B, C = pr["cov"][i].numpy()
        got = np.array([[A, B], [B, C]])
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
        assert abs(pr["u"][i].item() - pi(p)[0]) < 1e-9
        conic = np.linalg.inv(ref)
        a, b, c = pr["conic"][i].numpy()
        assert np.allclose([a, b, c], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-5)


def test_extent_is_the_bounding_box_of_the_alpha_min_ellipse():
    rng = np.random.default_rng(2)
    sc = scenes.random_gaussians(30, 200, 150, 150.0, seed=4, scale_range=(0.02, 0.2))
    t = _t
    pr = oracle.project(t(sc.means), t(sc.scales), t(sc.quats), t(sc.camera.T_cw[0]),
                        150.0, 150.0, 100.0, 75.0, Options())
    ext = oracle.extent(pr, sc.opacities, 200, 150, Options())
    for i in np.nonzero(ext["live"])[0]:
        A, B, C = pr["cov"][i].numpy()
        k = 2 * math.log(sc.opacities[i] * 255.0)
        # boundary of {d : d^T Sigma'^-1 d = k} sampled through an eigendecomposition
        lam, E = np.linalg.eigh(np.array([[A, B], [B, C]]))
        th = np.linspace(0, 2 * math.pi, 20001)
        pts = E @ (np.sqrt(k * lam)[:, None] * np.stack([np.cos(th), np.sin(th)]))
        assert abs(pts[0].max() - ext["rx"][i]) < 1e-6 * ext["rx"][i] + 1e-9
        assert abs(pts[1].max() - ext["ry"][i]) < 1e-6 * ext["ry"][i] + 1e-9
    del rng


def test_tile_counts_by_enumerating_pixels():
    sc = scenes.random_gaussians(60, 150, 90, 120.0, seed=5, scale_range=(0.01, 0.3))
    opts = Options(tile_w=16, tile_h=8)
    t = _t
    pr = oracle.project(t(sc.means), t(sc.scales), t(sc.quats), t(sc.camera.T_cw[0]),
                        120.0, 120.0, 75.0, 45.0, opts)
    ext = oracle.extent(pr, sc.opacities, 150, 90, opts)
    u, v = pr["u"].numpy(), pr["v"].numpy()
    for i in range(60):
        if not ext["live"][i]:
            assert ext["count"][i] == 0
            continue
        xs = [x for x in range(150) if abs(x + 0.5 - u[i]) <= ext["rx"][i]]
        ys = [y for y in range(90) if abs(y + 0.5 - v[i]) <= ext["ry"][i]]
        tiles = {(x // 16, y // 8) for x in xs for y in ys}
        assert ext["count"][i] == len(tiles)


def test_rect_min_quadratic_separable_closed_form_and_sampling():
    rng = np.random.default_rng(11)
    for _ in range(100):
        # b = 0: the minimum is a dx^2 + c dy^2, dx and dy the distances of 0 to the intervals
        a, c = rng.uniform(0.1, 3.0, 2)
        x0, x1 = np.sort(rng.uniform(-3, 3, 2))
        y0, y1 = np.sort(rng.uniform(-3, 3, 2))
        dx, dy = max(x0, -x1, 0.0), max(y0, -y1, 0.0)
        assert oracle.rect_min_quadratic(a, 0.0, c, x0, x1, y0, y1) == pytest.approx(
            a * dx * dx + c * dy * dy, rel=1e-14, abs=1e-15)
        # general positive-definite form: dense sampling bounds the minimum from above,
        # and from below within the largest change of q over one grid step
        L = rng.normal(size=(2, 2))
        M = L @ L.T + 0.05 * np.eye(2)
        got = oracle.rect_min_quadratic(M[0, 0], M[0, 1], M[1, 1], x0, x1, y0, y1)
        X, Y = np.meshgrid(np.linspace(x0, x1, 401), np.linspace(y0, y1, 401))
        qs = (M[0, 0] * X * X + 2 * M[0, 1] * X * Y + M[1, 1] * Y * Y).min()
        step = max(x1 - x0, y1 - y0) / 400.0
        grad = 2.0 * np.abs(M).sum() * 3.0
        assert got <= qs + 1e-12
        assert qs - got <= grad * step


def _proj_dict(u, v, cov, z=1.0):
    A, B, C = (np.asarray(t, np.float64) for t in cov)
    det = A * C - B * B
    return {"u": _t(u), "v": _t(v), "z": _t(np.full(np.shape(u), z)),
            "cov": _t(np.stack([A, B, C], -1)), "conic": _t(np.stack([C / det, -B / det, A / det], -1))}


def test_tile_cover_hand_worked_circle():
    # sigma = 2 px, o = 0.5: r = 2 sqrt(2 ln(127.5)) = 6.228 px around (21.5, 11.5) on
    # 16x8 tiles.  The bounding box spans tile columns 0-1 and rows 0-2 (6 tiles); the
    # nearest pixel-centre column segments of the corner tiles (0, 0) and (0, 2) are
    # 7.2 and 7.8 px from the centre, those of the other four 0, 4, 5 and 6 px away.
    pr = _proj_dict([21.5], [11.5], ([4.0], [0.0], [4.0]))
    opts = Options(tile_w=16, tile_h=8)
    cov = oracle.tile_cover(pr, np.array([0.5]), 64, 32, opts)
    assert cov["count"][0] == 4 and not cov["flags"][0]
    ext = oracle.extent(pr, np.array([0.5]), 64, 32, opts)
    assert ext["count"][0] == 6


def test_tile_cover_against_pixels_and_dense_sampling():
    sc = scenes.random_gaussians(80, 150, 90, 120.0, seed=9, scale_range=(0.01, 0.4))
    opts = Options(tile_w=16, tile_h=8)
    pr = oracle.project(_t(sc.means), _t(sc.scales), _t(sc.quats), _t(sc.camera.T_cw[0]),
                        120.0, 120.0, 75.0, 45.0, opts)
    ext = oracle.extent(pr, sc.opacities, 150, 90, opts)
    cov = oracle.tile_cover(pr, sc.opacities, 150, 90, opts)
    u, v = pr["u"].numpy(), pr["v"].numpy()
    con = pr["conic"].numpy()
    tighter = 0
    for i in range(80):
        if not ext["live"][i]:
            assert cov["count"][i] == 0
            continue
        a, b, c = con[i]
        k = 2 * math.log(sc.opacities[i] / opts.alpha_min)
        qf = lambda X, Y: a * X * X + 2 * b * X * Y + c * Y * Y  # noqa: E731
        # tiles holding a pixel centre with alpha >= alpha_min are all listed
        X, Y = np.meshgrid(np.arange(150) + 0.5 - u[i], np.arange(90) + 0.5 - v[i])
        ys, xs = np.nonzero(qf(X, Y) <= k)
        lattice = {(x // 16, y // 8) for x, y in zip(xs, ys)}
        assert cov["count"][i] >= len(lattice)
        # dense samples of each tile's (widened) pixel-centre columns: a sampled hit is
        # a hit, and a tile without one is a hit only when its sampled minimum is
        # within one sampling step of k
        mx = 1e-5 * ext["rx"][i] + 2e-3
        my = 1e-5 * ext["ry"][i] + 2e-3
        sampled, near = 0, 0
        for ty in range(12):
            ya, yb = ty * 8 + 0.5 - v[i] - my, min(ty * 8 + 8, 90) - 0.5 - v[i] + my
            for tx in range(10):
                cols = np.arange(tx * 16, min(tx * 16 + 16, 150)) + 0.5 - u[i]
                Xs = (cols[:, None, None] + np.linspace(-mx, mx, 5)[None, :, None]).reshape(-1, 1)
                Ys = np.linspace(ya, yb, 401)[None, :]
                qmin = qf(Xs, Ys).min()
                step = max(mx / 2, (yb - ya) / 400)
                reach = np.abs(Xs).max() + max(abs(ya), abs(yb))
                bound = 2 * (abs(a) + 2 * abs(b) + abs(c)) * reach * step
                sampled += qmin <= k
                near += k < qmin <= k + bound
        assert sampled <= cov["count"][i] <= sampled + near
        tighter += cov["count"][i] < ext["count"][i]
    assert tighter > 0  # the ellipse test drops bounding-box tiles


def test_two_gaussians_hand_worked_and_depth_order():
    # Two isotropic Gaussians centred on the same pixel centre.  At that pixel
    # alpha_i = o_i, so C = o1 c1 + (1 - o1) o2 c2 with the nearer one first.
    W = H = 9
    f = 10.0
    means = np.array([[0.05, 0.05, 2.0], [0.05, 0.05, 3.0]])  # u = v = 4.75 ... shift below
    # put the mean exactly on the centre of pixel (4,4): u = f x / z + 4.5 = 4.5
    means[:, :2] = 0.0
    scales = np.full((2, 3), 0.05)
    quats = np.tile([1.0, 0, 0, 0], (2, 1))
    opac = np.array([0.6, 0.5])
    cols = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    out = oracle.render(means, scales, quats, opac, cols, np.eye(4)[None], f, f, 4.5, 4.5, W, H)
    c = out["rgb"][0, :, 4, 4]
    assert np.allclose(c, [0.6, 0.4 * 0.5, 0.0], atol=1e-15)
    assert abs(out["depth"][0, 4, 4] - (0.6 * 2.0 + 0.4 * 0.5 * 3.0)) < 1e-14
    assert abs(out["t_final"][0, 4, 4] - 0.4 * 0.5) < 1e-15
    # swap depths: the green one is now in front
    means[:, 2] = [3.0, 2.0]
    out = oracle.render(means, scales, quats, opac, cols, np.eye(4)[None], f, f, 4.5, 4.5, W, H)
    assert np.allclose(out["rgb"][0, :, 4, 4], [0.5 * 0.6, 0.5, 0.0], atol=1e-15)


def test_equal_depths_are_ordered_by_index():
    # Two isotropic Gaussians at the identical mean (equal z): the lower index
    # composites first, C = o0 c0 + (1 - o0) o1 c1 at the shared pixel centre.
    # The pixel is flagged as a possible depth tie unless exact ties are accepted.
    from oracle.raster import Margins
    W = H = 9
    f = 10.0
    means = np.array([[0.0, 0.0, 2.5], [0.0, 0.0, 2.5]])
    scales = np.array([[0.05] * 3, [0.08] * 3])
    quats = np.tile([1.0, 0, 0, 0], (2, 1))
    opac = np.array([0.6, 0.5])
    cols = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    args = (np.eye(4)[None], f, f, 4.5, 4.5, W, H)
    out = oracle.render(means, scales, quats, opac, cols, *args)
    assert np.allclose(out["rgb"][0, :, 4, 4], [0.6, 0.4 * 0.5, 0.0], atol=1e-15)
    assert out["flags"][0, 4, 4]
    out = oracle.render(means, scales, quats, opac, cols, *args, margins=Margins(exact_ties=True))
    assert not out["flags"][0, 4, 4]
    # the same two Gaussians listed the other way round: green first
    out = oracle.render(means[::-1].copy(), scales[::-1].copy(), quats, opac[::-1].copy(), cols[::-1].copy(), *args)
    assert np.allclose(out["rgb"][0, :, 4, 4], [0.5 * 0.6, 0.5, 0.0], atol=1e-15)
    # a depth 1e-9 apart is still flagged with exact ties accepted
    means[1, 2] += 1e-9
    out = oracle.render(means, scales, quats, opac, cols, *args, margins=Margins(exact_ties=True))
    assert out["flags"][0, 4, 4]


def test_stop_rule_clamp_and_skip():
    W = H = 5
    f = 10.0
    n = 20
    means = np.zeros((n, 3))
    means[:, 2] = 2.0 + 0.01 * np.arange(n)
    scales = np.full((n, 3), 0.05)
    quats = np.tile([1.0, 0, 0, 0], (n, 1))
    cols = np.ones((n, 3))
    T = np.eye(4)[None]
    # alpha = 0.5 at the centre pixel: T after k contributors is 0.5^k; the 14th
    # would take T below 1e-4 (0.5^14 = 6.1e-5), so 13 contribute.
    out = oracle.render(means, scales, quats, np.full(n, 0.5), cols, T, f, f, 2.5, 2.5, W, H)
    assert out["n_contrib"][0, 2, 2] == 13
    assert abs(out["t_final"][0, 2, 2] - 0.5 ** 13) < 1e-18
    assert abs(out["alpha"][0, 2, 2] - (1 - 0.5 ** 13)) < 1e-15
    # opacity 1 is clamped to 0.99 at the centre
    out = oracle.render(means[:1], scales[:1], quats[:1], np.ones(1), cols[:1], T, f, f, 2.5, 2.5, W, H)
    assert abs(out["alpha"][0, 2, 2] - 0.99) < 1e-15
    # opacity just below 1/255 never contributes
    out = oracle.render(means[:1], scales[:1], quats[:1], np.full(1, 0.999 / 255), cols[:1], T,
                        f, f, 2.5, 2.5, W, H)
    assert out["n_contrib"].sum() == 0 and out["alpha"].max() == 0.0


def test_near_plane():
    kw = dict(W=5, H=5, f=10.0)
    assert _one((0, 0, 0.19), (0.01,) * 3, (1, 0, 0, 0), 0.9, (1, 1, 1), **kw)["alpha"].max() == 0
    assert _one((0, 0, 0.21), (0.01,) * 3, (1, 0, 0, 0), 0.9, (1, 1, 1), **kw)["alpha"].max() > 0.5


def test_invariants_on_planes_scene():
    sc = scenes.tiny_planes(n=3000, width=96, height=72, f=90.0)
    out = oracle.render_scene(sc)
    T = out["t_final"]
    assert T.min() >= 1e-4 and T.max() <= 1.0
    assert np.allclose(out["alpha"], 1 - T, atol=0)
    # sum of weights = 1 - T: with all colours 1 and bg 0 the colour equals alpha
    out1 = oracle.render(sc.means, sc.scales, sc.quats, sc.opacities, np.ones_like(sc.colors),
                         sc.camera.T_cw, sc.camera.fx, sc.camera.fy, sc.camera.cx, sc.camera.cy,
                         sc.camera.width, sc.camera.height)
    for ch in range(3):
        assert np.abs(out1["rgb"][0, ch] - out1["alpha"][0]).max() < 1e-12
    # depth is a convex-ish combination: D <= A * max z, D >= A * min z of the scene
    z = out["proj"][0]["z"]
    assert np.all(out["depth"] <= out["alpha"] * z.max() + 1e-12)
    # background enters as T * bg
    out_bg = oracle.render_scene(sc, opts=Options(bg=(0.25, 0.5, 1.0)))
    for ch, b in enumerate((0.25, 0.5, 1.0)):
        assert np.abs(out_bg["rgb"][0, ch] - out["rgb"][0, ch] - b * T[0]).max() < 1e-12


def test_brute_force_equals_candidate_filter():
    sc = scenes.random_gaussians(40, 48, 40, 50.0, seed=7, scale_range=(0.05, 0.4))
    a = oracle.render_scene(sc)
    b = oracle.render_scene(sc, brute=True, block_w=7)
    # equal up to summation order (zero-weight terms change torch's reduction tree)
    for k in ("rgb", "depth", "t_final"):
        assert np.abs(a[k] - b[k]).max() < 1e-14, k
    assert np.array_equal(a["n_contrib"], b["n_contrib"])
    assert a["n_contrib"].max() >= 5


def _fd_scene(n, seed, W=32, H=24, f=30.0, views=1):
    sc = scenes.random_gaussians(n, W, H, f, seed=seed, scale_range=(0.08, 0.35), n_views=views)
    sc.quats = sc.quats.astype(np.float64)
    return sc


def _loss(sc, g, means=None, scales=None, quats=None, opac=None, cols=None, T=None):
    cam = sc.camera
    out = oracle.render(sc.means if means is None else means, sc.scales if scales is None else scales,
                        sc.quats if quats is None else quats, sc.opacities if opac is None else opac,
                        sc.colors if cols is None else cols, cam.T_cw if T is None else T,
                        cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    L = (out["rgb"] * g[0]).sum() + (out["depth"] * g[1]).sum() + (out["alpha"] * g[2]).sum()
    return L, out["n_contrib"]


@pytest.mark.parametrize("seed", [11, 12])
def test_gradients_central_differences_every_parameter(seed):
    sc = _fd_scene(4, seed)
    cam = sc.camera
    g = scenes.upstream_grads(seed + 1, 1, cam.height, cam.width)
    out = oracle.render_scene(sc, grads=g)
    assert out["n_contrib"].max() >= 2
    base = [np.asarray(a, np.float64) for a in sc.arrays()]
    names = ("d_means", "d_scales", "d_quats", "d_opacities", "d_colors")
    h = 1e-6
    checked = 0
    for gi, name in enumerate(names):
        arr = base[gi]
        for idx in np.ndindex(arr.shape):
            args = [a.copy() for a in base]
            args[gi][idx] += h
            Lp, ncp = _loss(sc, g, *args)
            args[gi][idx] -= 2 * h
            Lm, ncm = _loss(sc, g, *args)
            if not (np.array_equal(ncp, out["n_contrib"]) and np.array_equal(ncm, out["n_contrib"])):
                continue  # the step crossed a decision; derivative undefined there
            fd = (Lp - Lm) / (2 * h)
            an = out[name][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)
            checked += 1
    assert checked >= 50


def _se3_exp(xi):
    H = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    H[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    H[:3, 3] = rho
    return scipy.linalg.expm(H)


def test_pose_gradient_through_the_exponential_map():
    sc = _fd_scene(6, 21, views=2)
    cam = sc.camera
    g = scenes.upstream_grads(22, 2, cam.height, cam.width)
    out = oracle.render_scene(sc, grads=g)
    h = 1e-6
    for v in range(2):
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Tp = cam.T_cw.copy()
            Tp[v] = _se3_exp(e) @ cam.T_cw[v]
            Lp, _ = _loss(sc, g, T=Tp)
            Tm = cam.T_cw.copy()
            Tm[v] = _se3_exp(-e) @ cam.T_cw[v]
            Lm, _ = _loss(sc, g, T=Tm)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - out["d_pose"][v, k]) <= 1e-6 * max(1.0, abs(fd)), (v, k)


def test_pose_gradient_rigid_motion_identity():
    # moving the camera by xi equals moving every Gaussian by the inverse motion:
    # d/d rho = R_cw sum_i dL/dmu_i, d/d phi = R_cw sum_i [(mu_i - c) x dL/dmu_i + dq/domega^T dL/dq_i]
    sc = scenes.tiny_planes(n=2000, width=64, height=48, f=60.0)
    sc.quats = sc.quats * np.float32(1.7)  # non-unit quaternions are normalised inside
    cam = sc.camera
    T = cam.T_cw[0].copy()
    T[:3, :3] = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    T[:3, 3] = -T[:3, :3] @ np.array([0.2, -0.1, -3.0])
    sc.camera.T_cw = T[None]
    g = scenes.upstream_grads(3, 1, cam.height, cam.width)
    out = oracle.render_scene(sc, grads=g)
    R = T[:3, :3]
    c = -R.T @ T[:3, 3]
    dmu = out["d_means"]
    dq = out["d_quats"]
    rho_ref = R @ dmu.sum(0)
    q = sc.quats.astype(np.float64)
    om = np.zeros(3)
    for k in range(3):
        w = np.eye(3)[k]
        # first-order change of q under q <- (1, w/2) (x) q
        dq_w = 0.5 * np.concatenate([-(q[:, 1:] @ w)[:, None],
                                     q[:, :1] * w[None] + np.cross(w[None], q[:, 1:])], 1)
        om[k] = (dq * dq_w).sum() + (dmu * np.cross(w[None], sc.means - c[None])).sum()
    phi_ref = R @ om
    ref = np.concatenate([rho_ref, phi_ref])
    assert np.abs(out["d_pose"][0] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_clamped_alpha_has_no_opacity_gradient():
    W = H = 5
    g_rgb = np.zeros((1, 3, H, W))
    g_rgb[0, :, 2, 2] = 1.0  # only the centre pixel, where o exp(0) = 1 is clamped to 0.99
    g = (g_rgb, np.zeros((1, H, W)), np.zeros((1, H, W)))
    out = _one((0, 0, 2.0), (0.01, 0.01, 0.01), (1, 0, 0, 0), 1.0, (1, 1, 1), W=W, H=H, f=10.0, grads=g)
    assert abs(out["alpha"][0, 2, 2] - 0.99) < 1e-15
    assert out["d_opacities"][0] == 0.0
    assert np.all(out["d_means"] == 0.0)
    # unclamped (o = 0.5) the same pixel does move the opacity gradient
    out = _one((0, 0, 2.0), (0.01, 0.01, 0.01), (1, 0, 0, 0), 0.5, (1, 1, 1), W=W, H=H, f=10.0, grads=g)
    assert abs(out["d_opacities"][0] - 3.0) < 1e-12  # dC/do = 1 per channel at the centre
