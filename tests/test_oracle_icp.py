"""Pins of the FP64 voxel-ICP oracle (Sec. III-B, Eq. 10-12)."""
import numpy as np

import importlib

from oracle.pose import se3_exp

I = importlib.import_module("oracle.icp")  # the module (the package exports icp() as voxel_icp)


def _planes(rng, n=(3000, 2000, 2000)):
    a, b, c = n
    return np.concatenate([np.c_[rng.uniform(-5, 5, a), rng.uniform(-5, 5, a), np.zeros(a)],
                           np.c_[rng.uniform(-5, 5, b), np.full(b, 3.0), rng.uniform(0, 3, b)],
                           np.c_[np.full(c, -4.0), rng.uniform(-5, 5, c), rng.uniform(0, 3, c)]])


def _tr(c):
    T = np.eye(4)
    T[:3, 3] = c
    return T


def test_downsampling_keeps_the_first_point_of_each_voxel():
    rng = np.random.default_rng(0)
    p = rng.uniform(-2, 2, size=(400, 3)).astype(np.float32)
    idx = I.voxel_downsample(p, 0.5)
    seen = {}
    for i, q in enumerate(p):  # brute force in index order
        seen.setdefault(tuple(int(np.floor(x / np.float32(0.5))) for x in q), i)
    assert sorted(seen.values()) == list(idx)
    assert len(I.voxel_downsample(np.zeros((0, 3), np.float32), 0.5)) == 0


def test_double_downsampling_is_two_first_point_passes():
    rng = np.random.default_rng(3)
    p = rng.uniform(-3, 3, size=(2000, 3)).astype(np.float32)
    idx = I.double_downsample(p, 0.25, 0.75)
    first = {}
    for i, q in enumerate(p):
        first.setdefault(tuple(np.floor(q / np.float32(0.25)).astype(int)), i)
    stage1 = sorted(first.values())
    second = {}
    for i in stage1:
        second.setdefault(tuple(np.floor(p[i] / np.float32(0.75)).astype(int)), i)
    assert sorted(second.values()) == list(idx)
    # every kept point is an original point and voxels of edge v2 hold at most one
    keys = I.voxel_keys(p[idx], 0.75)
    assert len(np.unique(keys, axis=0)) == len(idx)


def test_weight_is_the_derivative_of_rho_over_e():
    sigma = 0.3
    for e in (0.01, 0.1, 0.5, 2.0):
        h = 1e-7
        d = (I.gm_rho(e + h, sigma) - I.gm_rho(e - h, sigma)) / (2 * h)
        assert abs(d / e - I.gm_weight(e, sigma)) < 1e-7 * max(1.0, I.gm_weight(e, sigma))
    assert I.gm_weight(0.0, sigma) == 3.0 / sigma  # rho ~ e^2 / (2 sigma / 3) near 0
    assert abs(I.gm_rho(1e6, sigma) - 0.5) < 1e-12  # bounded influence


def _check_normal_equations(c):
    rng = np.random.default_rng(1)
    s = rng.normal(size=(30, 3)) + np.array([20.0, -5.0, 3.0])
    m = s + rng.normal(scale=0.05, size=s.shape)
    sigma = 0.2
    H, b, _ = I.normal_equations(s, m, sigma, c=c)
    w = np.array([I.gm_weight(np.linalg.norm(a - q), sigma) for a, q in zip(s, m)])
    cc = np.zeros(3) if c is None else np.asarray(c)

    def cost(xi):  # fixed weights, s' = c + Exp(xi) (s - c)
        T = _tr(cc) @ se3_exp(xi) @ _tr(-cc)
        t = s @ T[:3, :3].T + T[:3, 3]
        return 0.5 * (w * ((t - m) ** 2).sum(1)).sum()

    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        assert abs((cost(e) - cost(-e)) / (2 * h) - b[k]) < 1e-6 * max(1.0, abs(b[k]))
    assert np.allclose(H, H.T) and np.all(np.linalg.eigvalsh(H) > 0)
    # the Hessian of the linearised cost: H xi + b is its gradient, so
    # check the gradient of 1/2 sum w |r + J xi|^2 at a random xi
    xi = rng.normal(scale=1e-3, size=6)

    def lin_cost(x):
        tot = 0.0
        for si, mi, wi in zip(s, m, w):
            J = np.hstack([np.eye(3), -I.skew(si - cc)])
            r = si - mi + J @ x
            tot += 0.5 * wi * r @ r
        return tot

    g = np.array([(lin_cost(xi + h * np.eye(6)[k]) - lin_cost(xi - h * np.eye(6)[k])) / (2 * h) for k in range(6)])
    assert np.allclose(g, H @ xi + b, rtol=1e-6, atol=1e-6)


def test_normal_equations_are_the_gauss_newton_system():
    _check_normal_equations(None)


def test_normal_equations_about_a_centre():
    _check_normal_equations([18.0, -4.0, 2.0])


def test_centred_step_equals_the_plain_step():
    # Tr(c) Exp(xi_c) Tr(-c) == Exp(xi_0) for the steps solved about c and about 0
    rng = np.random.default_rng(4)
    s = _planes(rng, (300, 200, 200)) + np.array([30.0, 40.0, 0.0])
    m = s + rng.normal(scale=0.03, size=s.shape)
    c = np.array([29.0, 41.0, 1.0])
    x0 = I.solve_step(*I.normal_equations(s, m, 0.3)[:2])
    xc = I.solve_step(*I.normal_equations(s, m, 0.3, c=c)[:2])
    assert np.allclose(_tr(c) @ se3_exp(xc) @ _tr(-c), se3_exp(x0), atol=1e-9)


def test_searches_match_brute_force():
    rng = np.random.default_rng(5)
    mp = rng.uniform(-2, 2, size=(3000, 3)).astype(np.float32)
    mp[100] = mp[7]  # an exact duplicate: the tie goes to the lower index
    q = np.concatenate([rng.uniform(-2.2, 2.2, size=(300, 3)), mp[[7, 8, 9]].astype(np.float64)])
    tau = 0.15
    from scipy.spatial import cKDTree
    got64 = I.nearest(q, cKDTree(mp.astype(np.float64)), tau)
    got32 = I.nearest_f32(q, mp, tau)
    m64 = mp.astype(np.float64)
    for i, x in enumerate(q):
        d64 = np.sqrt(((m64 - x) ** 2).sum(1))
        j = int(np.argmin(d64))
        assert got64[i] == (j if d64[j] < tau else -1)
        x32 = x.astype(np.float32)
        d = mp - x32
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        ok = np.nonzero(d2 < np.float32(tau) * np.float32(tau))[0]
        assert got32[i] == (ok[np.argmin(d2[ok])] if len(ok) else -1)
    assert got32[-3] == 7 and got64[-3] == 7


def _scene(seed, outliers=0):
    rng = np.random.default_rng(seed)
    pts = _planes(rng).astype(np.float32)
    T_true = se3_exp(np.array([0.3, -0.2, 0.1, 0.02, -0.03, 0.05]))
    scan = ((pts - T_true[:3, 3]) @ T_true[:3, :3]).astype(np.float32)  # T_true maps scan onto map
    if outliers:
        scan = np.concatenate([scan, rng.uniform(-6, 6, size=(outliers, 3)).astype(np.float32)])
        scan = scan[rng.permutation(len(scan))]
    T0 = se3_exp(np.array([0.05, 0.04, -0.03, 0.01, 0.01, -0.01])) @ T_true
    return pts, scan, T_true, T0


def test_recovers_a_known_rigid_motion():
    pts, scan, T_true, T0 = _scene(2)
    out = I.icp(scan, pts, T0, v1=0.1, v2=0.3, tau=0.5, sigma=0.3, iterations=60, eps=1e-9)
    assert out["stop"] == I.CONVERGED
    assert np.abs(out["T"] - T_true).max() < 1e-5
    assert out["correspondences"] == len(out["src_idx"])
    assert out["counts"][0] <= out["counts"][-1]


def test_robust_to_outliers():
    pts, scan, T_true, T0 = _scene(6, outliers=1500)
    out = I.icp(scan, pts, T0, v1=0.1, v2=0.3, tau=0.5, sigma=0.3, iterations=60, eps=1e-9)
    assert out["stop"] == I.CONVERGED
    assert np.abs(out["T"][:3, 3] - T_true[:3, 3]).max() < 1e-3
    assert np.abs(out["T"][:3, :3] - T_true[:3, :3]).max() < 1e-3


def test_stops_on_too_few_correspondences():
    pts, scan, _, T0 = _scene(2)
    out = I.icp(scan, pts + 100.0, T0, v1=0.1, v2=0.3, tau=0.5, sigma=0.3)
    assert out["stop"] == I.TOO_FEW and out["iterations"] == 1
    assert np.array_equal(out["T"], T0)
