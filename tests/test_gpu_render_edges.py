"""Edge cases of the rasterizer's decisions, on the GPU through the C ABI, against the FP64 oracle.

Each scene puts many pixels right on one of the method's special cases:
  * exactly equal depths (the order rule: equal camera z goes by Gaussian index);
  * near-degenerate Gaussians: needles and flat discs seen edge-on, whose 2D
    covariance has a condition number of 1e4 to beyond 1e6;
  * Gaussians within 1e-4 m of the near plane, on either side;
  * the transmittance stop rule (a stack of alpha = 0.5 layers, 13 contribute)
    and the 0.99 clamp, both at a pixel centre.
Tolerances are those of every other parity test: images within 1e-5, contributor
counts bit-exact, gradients within 1e-3 (tests/helpers.py).
"""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from oracle.raster import Margins, Options
from paper_2505_18992_gb300 import scenes
from tests.helpers import (assert_grad_close, assert_images_close, assert_pose_close, masked_upstream,
                           tile_count_mask)
from tests.test_gpu_render import GRAD_KEYS, _gpu_backward, _gpu_forward

pytestmark = pytest.mark.gpu


def _quat_wxyz(R):
    """float32 (w, x, y, z) of rotation matrices R [n,3,3] (columns = the Gaussian's axes)."""
    q = Rotation.from_matrix(R).as_quat()  # (x, y, z, w)
    return np.ascontiguousarray(q[:, [3, 0, 1, 2]]).astype(np.float32)


def _scene(name, means, scales, quats, opac, cols, W, H, f, Ts, cx=None, cy=None):
    cam = scenes.Camera(W, H, f, f, W / 2.0 if cx is None else cx, H / 2.0 if cy is None else cy,
                        np.asarray(Ts, np.float64).reshape(-1, 4, 4))
    f32 = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    return scenes.GaussianScene(name, f32(means), f32(scales), f32(quats), f32(opac), f32(cols), cam)


def _with_background(rng, parts, n_bg, W, H, f, depth=(1.5, 4.0)):
    bg = scenes.random_gaussians(n_bg, W, H, f, seed=int(rng.integers(1 << 30)), depth=depth,
                                 scale_range=(0.01, 0.06))
    keys = ("means", "scales", "quats", "opacities", "colors")
    out = [np.concatenate([p[i] for p in parts] + [getattr(bg, k)], 0) for i, k in enumerate(keys)]
    return out


def _parity(sc, margins=None, tile_counts=True):
    """Forward and backward of sc on the GPU (16x16 tiles) against the oracle.

    Returns the GPU forward, the oracle's forward and the GPU projection
    (tile counts etc., as numpy)."""
    ref0 = oracle.render_scene(sc, margins=margins)
    r, g, T, out = _gpu_forward(sc, tile_w=16, tile_h=16)
    rep = assert_images_close(out, ref0, ref0["flags"], what=sc.name)
    assert rep["flagged_frac"] < 0.05, rep
    p = {k: v.cpu().numpy() for k, v in r.project(*g, T).items()}
    if tile_counts and sc.camera.n_views == 1:
        cam = sc.camera
        cover = oracle.tile_cover(ref0["proj"][0], sc.opacities, cam.width, cam.height, Options())
        mask = tile_count_mask(ref0["extent"][0], sc.opacities) | cover["flags"]
        assert np.array_equal(p["tile_count"][0][~mask], cover["count"][~mask])
    g_up = scenes.upstream_grads(41, sc.camera.n_views, sc.camera.height, sc.camera.width)
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, grads=gm, margins=margins)
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])
    return out, ref0, p


# ---------------------------------------------------------------------------
# exactly equal depths
# ---------------------------------------------------------------------------

def _tie_scene(seed=3, groups=8, per=4, W=128, H=96, f=110.0, n_views=2):
    rng = np.random.default_rng(seed)
    z = rng.uniform(1.5, 3.0, groups)
    xy = rng.uniform(-0.6, 0.6, (groups, 2)) * z[:, None] * np.array([W / (2 * f), H / (2 * f)])
    centre = np.concatenate([xy, z[:, None]], 1)
    n = groups * per
    means = np.repeat(centre, per, 0)                      # identical means within a group
    scales = np.exp(rng.uniform(np.log(0.02), np.log(0.08), (n, 3)))
    quats = rng.normal(size=(n, 4))
    opac = rng.uniform(0.3, 0.9, n)
    cols = rng.uniform(0, 1, (n, 3))
    parts = [(means, scales, quats, opac, cols)]
    allv = _with_background(rng, parts, 150, W, H, f)
    Ts = [np.eye(4)] + [scenes.perturb_pose(np.eye(4), rng, 0.1, 4.0) for _ in range(n_views - 1)]
    return _scene("ties", *allv, W, H, f, Ts), n, per


def test_equal_depths_go_by_index():
    sc, n_tied, per = _tie_scene()
    # the test can only fail a wrong order if the order shows: list every tie
    # group the other way round and the oracle's image changes
    perm = np.arange(sc.n)
    perm[:n_tied] = perm[:n_tied].reshape(-1, per)[:, ::-1].ravel()
    rev = scenes.GaussianScene("ties reversed", *(np.ascontiguousarray(a[perm]) for a in sc.arrays()), sc.camera)
    exact = Margins(exact_ties=True)
    a = oracle.render_scene(sc, margins=exact)
    b = oracle.render_scene(rev, margins=exact)
    assert np.abs(a["rgb"] - b["rgb"]).max() > 1e-2
    tie_px = np.abs(a["rgb"] - b["rgb"]).max(1) > 1e-4
    assert tie_px.sum() > 200
    out, ref0, _ = _parity(sc, margins=exact, tile_counts=False)
    assert not ref0["flags"][tie_px].any()          # the tie pixels take part in the comparison
    assert np.abs(out["rgb"] - b["rgb"]).max() > 1e-2  # and the GPU did not take the reversed order


# ---------------------------------------------------------------------------
# near-degenerate 2D covariances
# ---------------------------------------------------------------------------

def _needle_scene(seed=5, n_needles=24, n_discs=16, W=160, H=120, f=150.0):
    rng = np.random.default_rng(seed)
    n = n_needles + n_discs
    z = rng.uniform(1.5, 4.0, n)
    z[:4] = 1.6
    xy = rng.uniform(-0.7, 0.7, (n, 2)) * z[:, None] * np.array([W / (2 * f), H / (2 * f)])
    means = np.concatenate([xy, z[:, None]], 1)
    ray = means / np.linalg.norm(means, axis=1, keepdims=True)
    v = rng.normal(size=(n, 3))
    perp = v - (v * ray).sum(1, keepdims=True) * ray
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    length = np.exp(rng.uniform(np.log(0.15), np.log(3.0), n))
    length[:4] = [7.0, 8.0, 9.0, 10.0]  # 2D condition numbers beyond 1e6 (at z = 1.6)
    thin = np.exp(rng.uniform(np.log(1e-4), np.log(1e-3), n))  # scale ratio 1e3 - 1e4
    R = np.zeros((n, 3, 3))
    scales = np.zeros((n, 3))
    # needles: the long axis across the ray (tilted towards it by up to 15 degrees)
    tilt = np.radians(rng.uniform(-15, 15, n))[:, None]
    a = np.cos(tilt) * perp + np.sin(tilt) * ray
    b = np.cross(a, ray)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    c = np.cross(a, b)
    nd = slice(0, n_needles)
    R[nd] = np.stack([a, b, c], 2)[nd]
    scales[nd] = np.stack([length, length * thin, length * thin * rng.uniform(0.5, 2.0, n)], 1)[nd]
    # discs seen edge-on: the normal across the ray, so the disc's plane holds the ray
    dk = slice(n_needles, n)
    normal = perp
    e1 = np.cross(normal, ray)
    R[dk] = np.stack([ray, e1, normal], 2)[dk]
    scales[dk] = np.stack([length, length * rng.uniform(0.5, 1.0, n), length * thin], 1)[dk]
    quats = _quat_wxyz(R)
    opac = rng.uniform(0.3, 0.95, n)
    cols = rng.uniform(0, 1, (n, 3))
    allv = _with_background(rng, [(means, scales, quats, opac, cols)], 80, W, H, f, depth=(4.0, 6.0))
    return _scene("needles", *allv, W, H, f, [np.eye(4)]), n


def _conditioning(proj):
    A, B, C = proj["cov"][:, 0], proj["cov"][:, 1], proj["cov"][:, 2]
    h = np.sqrt(0.25 * (A - C) ** 2 + B * B)
    return (0.5 * (A + C) + h) / (0.5 * (A + C) - h)


def test_near_degenerate_covariances():
    sc, n_special = _needle_scene()
    ref0 = oracle.render_scene(sc)
    kappa = _conditioning(ref0["proj"][0])[:n_special]
    on_screen = ref0["extent"][0]["nonempty"][:n_special]
    assert (kappa[on_screen] >= 1e4).sum() >= 12
    assert (kappa[on_screen] >= 1e6).sum() >= 2
    _parity(sc)


# ---------------------------------------------------------------------------
# the near plane
# ---------------------------------------------------------------------------

def test_near_plane_within_1e4():
    W, H, f = 128, 96, 120.0
    rng = np.random.default_rng(9)
    offs = np.array([-1e-4, -1e-5, 1e-5, 1e-4])
    n = 48
    z = 0.2 + np.tile(offs, n // len(offs))
    xy = rng.uniform(-0.8, 0.8, (n, 2)) * z[:, None] * np.array([W / (2 * f), H / (2 * f)])
    cam_pts = np.concatenate([xy, z[:, None]], 1)
    T1 = scenes.perturb_pose(np.eye(4), rng, 0.2, 10.0)
    scales = np.exp(rng.uniform(np.log(0.001), np.log(0.004), (n, 3)))
    quats = rng.normal(size=(n, 4))
    opac = rng.uniform(0.5, 0.95, n)
    cols = rng.uniform(0, 1, (n, 3))
    for T in (np.eye(4), T1):
        # camera-space points at z = 0.2 +- 1e-4 .. 1e-5, placed in the world through T^-1
        Ti = np.linalg.inv(T)
        means = (cam_pts @ Ti[:3, :3].T + Ti[:3, 3]).astype(np.float32)
        zc = means.astype(np.float64) @ T[2, :3] + T[2, 3]
        assert np.all(np.abs(zc - z) < 2e-7)  # float32 means keep each point on its side
        allv = _with_background(rng, [(means, scales, quats, opac, cols)], 60, W, H, f)
        if T is T1:  # the background in front of the moved camera
            allv[0][n:] = (allv[0][n:].astype(np.float64) @ Ti[:3, :3].T + Ti[:3, 3]).astype(np.float32)
        sc = _scene("near plane", *allv, W, H, f, [T])
        out, ref0, p = _parity(sc)
        pr = ref0["proj"][0]
        u, v = pr["u"][:n], pr["v"][:n]
        inside = (u > 1) & (u < W - 1) & (v > 1) & (v < H - 1)
        ui, vi = np.floor(u).astype(int), np.floor(v).astype(int)
        front = (zc > 0.2) & inside
        behind = (zc <= 0.2) & inside
        assert front.sum() >= 8 and behind.sum() >= 8
        # the GPU's own decisions: a visible centre pixel blends, a culled one is left alone
        assert np.all(out["n_contrib"][0, vi[front], ui[front]] > 0)
        assert np.all(p["tile_count"][0][:n][zc <= 0.2] == 0)
        assert np.all(p["tile_count"][0][:n][front] > 0)


# ---------------------------------------------------------------------------
# the stop rule and the clamp at a pixel centre
# ---------------------------------------------------------------------------

def test_stop_rule_and_clamp_at_pixel_centres():
    W, H, f = 160, 120, 160.0
    cx, cy = 80.5, 60.5  # pixel (80, 60) has its centre on the optical axis
    k = 20
    z = 1.0 + 0.125 * np.arange(k)  # exact in binary
    # stack A: on the axis, alpha = 0.5 at pixel (80, 60): 0.5^13 >= 1e-4 > 0.5^14, so 13 blend
    ma = np.stack([np.zeros(k), np.zeros(k), z], 1)
    # stack B: u = 80.5 + 160 x / z = 100.5 and v = 40.5 at pixel (100, 40); the front layer
    # has opacity 0.999, clamped to 0.99, then 0.01 * 0.5^6 >= 1e-4 > 0.01 * 0.5^7: 7 blend
    mb = np.stack([z / 8.0, -z / 8.0, z], 1)
    means = np.concatenate([ma, mb], 0)
    scales = np.full((2 * k, 3), 0.02)
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (2 * k, 1))
    opac = np.full(2 * k, 0.5)
    opac[k] = 0.999
    rng = np.random.default_rng(13)
    cols = rng.uniform(0, 1, (2 * k, 3))
    allv = _with_background(rng, [(means, scales, quats, opac, cols)], 120, W, H, f, depth=(4.0, 6.0))
    sc = _scene("stop and clamp", *allv, W, H, f, [np.eye(4)], cx=cx, cy=cy)
    out, ref0, _ = _parity(sc)
    assert ref0["n_contrib"][0, 60, 80] == 13 and out["n_contrib"][0, 60, 80] == 13
    assert ref0["n_contrib"][0, 40, 100] == 7 and out["n_contrib"][0, 40, 100] == 7
    assert not ref0["flags"][0, 60, 80] and not ref0["flags"][0, 40, 100]
    assert out["t_final"][0, 60, 80] == np.float32(0.5) ** 13       # exact in float32
    one_minus = np.float32(1.0) - np.float32(0.99)
    assert out["t_final"][0, 40, 100] == one_minus * np.float32(0.5) ** 6


# ---------------------------------------------------------------------------
# tile lists of thousands of entries
# ---------------------------------------------------------------------------

def _long_list_scene(seed=21, n=5000, groups=10, per=4, W=96, H=72, f=100.0):
    """n Gaussians of about 5 px sigma, centred within 6 px of the corner shared
    by four 16x16 tiles, so each is listed in all four and every list runs past
    4,096 entries (many sort tiles of the tile-id sort, and compositing batches).
    Depth falls with the index, so the depth order reverses the index order.
    In front of them, `groups` groups of `per` Gaussians with identical means
    (bit-identical camera z), faint enough that the crowd behind still shows."""
    rng = np.random.default_rng(seed)
    cx, cy = 48.0, 32.0  # pixel (48, 32) is the corner of tiles (2..3, 1..2)
    z = np.linspace(4.0, 1.5, n) + rng.uniform(-1e-4, 1e-4, n)  # 5e-4 apart: no near-ties
    du, dv = rng.uniform(-6, 6, n), rng.uniform(-6, 6, n)
    means = np.stack([du * z / f, dv * z / f, z], 1)
    scales = np.exp(rng.uniform(np.log(0.04), np.log(0.06), (n, 3))) * z[:, None]
    opac = rng.uniform(0.3, 0.8, n)
    zt = rng.uniform(1.2, 1.45, groups)
    dt = rng.uniform(-6, 6, (groups, 2))
    tmeans = np.repeat(np.stack([dt[:, 0] * zt / f, dt[:, 1] * zt / f, zt], 1), per, 0)
    tscales = np.exp(rng.uniform(np.log(0.03), np.log(0.05), (groups * per, 3))) * np.repeat(zt, per)[:, None]
    topac = rng.uniform(0.05, 0.1, groups * per)
    m = n + groups * per
    parts = [(np.concatenate([means, tmeans]), np.concatenate([scales, tscales]), rng.normal(size=(m, 4)),
              np.concatenate([opac, topac]), rng.uniform(0, 1, (m, 3)))]
    allv = _with_background(rng, parts, 100, W, H, f, depth=(4.5, 6.0))
    return _scene("long lists", *allv, W, H, f, [np.eye(4)], cx=cx, cy=cy), m


def test_long_tile_lists_keep_depth_order_with_ties_by_index():
    sc, m = _long_list_scene()
    exact = Margins(exact_ties=True)
    out, ref0, p = _parity(sc, margins=exact)
    counts = p["tile_count"][0]
    # every centre lies within 1.5 sigma of the four tiles' shared corner, so each
    # of the crowd is listed in all four: their lists run past 4,096 entries
    assert (counts[:m] >= 4).all()
    # the tie rule shows: with the crowd's index order reversed (the depth order
    # unchanged but for the tie groups) the oracle's image changes, and the GPU's
    # image is not that one
    perm = np.arange(sc.n)
    perm[:m] = perm[:m][::-1]
    rev = scenes.GaussianScene("long lists reversed", *(np.ascontiguousarray(a[perm]) for a in sc.arrays()),
                               sc.camera)
    b = oracle.render_scene(rev, margins=exact)
    assert np.abs(ref0["rgb"] - b["rgb"]).max() > 1e-2
    assert np.abs(out["rgb"] - b["rgb"]).max() > 1e-2
