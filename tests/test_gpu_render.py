"""GPU rasterizer (through the C ABI) against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle.raster import Options
from paper_2505_18992_gb300 import scenes
from paper_2505_18992_gb300 import vpgs as C
from paper_2505_18992_gb300.render import Renderer, render
from tests.helpers import (assert_grad_close, assert_images_close, assert_pose_close, dev,
                           intrinsics, masked_upstream, scene_tensors, tile_count_mask)

pytestmark = pytest.mark.gpu

GRAD_KEYS = ("means", "scales", "quats", "opacities", "colors")


def _np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def _gpu_forward(sc, **opts):
    r = Renderer(intrinsics(sc), n_views=sc.camera.n_views, **opts)
    g, T = scene_tensors(sc)
    out = r.forward(*g, T)
    torch.cuda.synchronize()
    return r, g, T, _np(out)


def _gpu_backward(r, g, T, out_np, grads_np, reuse=False):
    fwd = {"t_final": dev(out_np["t_final"]), "n_iter": dev(out_np["n_iter"], torch.int32)}
    gr = {k: torch.zeros_like(t) for k, t in zip(GRAD_KEYS, g)}
    dpose = torch.zeros((r.V, 6), dtype=torch.float64, device="cuda")
    r.backward(*g, T, fwd, dev(grads_np[0]), dev(grads_np[1]), dev(grads_np[2]), grads=gr, dpose=dpose,
               check=True, reuse=reuse)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in gr.items()}, dpose.cpu().numpy()


@pytest.fixture(scope="module")
def planes():
    return scenes.tiny_planes()


@pytest.fixture(scope="module")
def planes_ref(planes):
    g = scenes.upstream_grads(7, 1, planes.camera.height, planes.camera.width)
    ref0 = oracle.render_scene(planes)
    gm = masked_upstream(g, ref0["flags"])
    ref = oracle.render_scene(planes, grads=gm)
    return ref, gm


def test_tile_counts_and_projection(planes, planes_ref):
    ref, _ = planes_ref
    r = Renderer(intrinsics(planes), tile_w=16, tile_h=16)  # the oracle's extents use 16x16 tiles
    g, T = scene_tensors(planes)
    p = {k: v.cpu().numpy() for k, v in r.project(*g, T).items()}
    ext = ref["extent"][0]
    cover = oracle.tile_cover(ref["proj"][0], planes.opacities, planes.camera.width, planes.camera.height,
                              Options(tile_w=16, tile_h=16))
    mask = tile_count_mask(ext, planes.opacities) | cover["flags"]
    cnt = p["tile_count"][0]
    assert np.array_equal(cnt[~mask], cover["count"][~mask])
    assert mask.mean() < 0.05
    assert (cover["count"] < ext["count"]).sum() > 0  # the cover is tighter than the box
    live = cnt > 0
    assert np.array_equal(p["tile_rect"][0][live & ~mask], ext["tiles"][live & ~mask])
    uv = np.stack([ref["proj"][0]["u"], ref["proj"][0]["v"]], 1)
    assert np.abs(p["mean2d"][0][live] - uv[live]).max() < 1e-4
    zz = ref["proj"][0]["z"]
    assert np.abs(p["depth"][0][live] - zz[live]).max() <= 1e-6 * zz.max()
    con = ref["proj"][0]["conic"]
    rel = np.abs(p["conic"][0][live] - con[live]) / np.abs(con[live]).max(1, keepdims=True)
    assert rel.max() < 1e-4


def test_forward_parity(planes, planes_ref):
    ref, _ = planes_ref
    _, _, _, out = _gpu_forward(planes)
    rep = assert_images_close(out, ref, ref["flags"], what="tiny planes")
    assert rep["flagged_frac"] < 0.01
    assert out["n_contrib"].max() > 10


def test_backward_parity(planes, planes_ref):
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes)
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


@pytest.mark.parametrize("keys", [(), ("means",), ("means", "scales", "quats")])
def test_geometric_backward_without_colour_or_opacity(planes, planes_ref, keys):
    """Asking for no opacity or colour gradient (pose tracking) selects the
    compositing backward that sums only the geometric 2D slots: the pose and
    the geometric gradients still match the oracle, and a full backward after
    it still does (the slots it leaves alone stay zero between calls)."""
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes)
    fwd = {"t_final": dev(out["t_final"]), "n_iter": dev(out["n_iter"], torch.int32)}
    gr = {k: torch.zeros_like(t) for k, t in zip(GRAD_KEYS, g) if k in keys}
    dpose = torch.zeros((r.V, 6), dtype=torch.float64, device="cuda")
    r.backward(*g, T, fwd, dev(gm[0]), dev(gm[1]), dev(gm[2]), grads=gr or None, dpose=dpose, check=True)
    torch.cuda.synchronize()
    for k in keys:
        assert_grad_close(gr[k].cpu().numpy(), ref["d_" + k], k)
    assert_pose_close(dpose.cpu().numpy(), ref["d_pose"])
    grads, dpose2 = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose2, ref["d_pose"])


def test_geometric_backward_three_views_ragged():
    """The geometric-only compositing backward (pose and means only) on 3 views
    of a ragged 97x61 image matches the oracle."""
    sc = scenes.random_gaussians(300, 97, 61, 80.0, seed=21, scale_range=(0.02, 0.2), n_views=3)
    g_up = scenes.upstream_grads(3, 3, 61, 97)
    ref0 = oracle.render_scene(sc)
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, grads=gm)
    r, g, T, out = _gpu_forward(sc)
    fwd = {"t_final": dev(out["t_final"]), "n_iter": dev(out["n_iter"], torch.int32)}
    gr = {"means": torch.zeros_like(g[0])}
    dpose = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
    r.backward(*g, T, fwd, dev(gm[0]), dev(gm[1]), dev(gm[2]), grads=gr, dpose=dpose, check=True)
    torch.cuda.synchronize()
    assert_grad_close(gr["means"].cpu().numpy(), ref["d_means"], "means")
    assert_pose_close(dpose.cpu().numpy(), ref["d_pose"])


@pytest.mark.parametrize("tile", [(8, 16), (8, 8), (32, 8)])
def test_backward_parity_other_tile_shapes(planes, planes_ref, tile):
    """Other tile shapes (a one-warp 8x8 tile, two- and four-warp tiles) add
    their warps' sums of a Gaussian by global atomics: all match the oracle."""
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes, tile_w=tile[0], tile_h=tile[1])
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


@pytest.mark.parametrize("tile", [(16, 16), (8, 16), (32, 8), (8, 32), (16, 8), (8, 8)])
def test_tile_shape_does_not_change_the_image(planes, planes_ref, tile):
    ref, _ = planes_ref
    _, _, _, out = _gpu_forward(planes, tile_w=tile[0], tile_h=tile[1])
    assert_images_close(out, ref, ref["flags"], what=str(tile))


def test_persistent_launch_is_bit_identical(planes):
    _, _, _, a = _gpu_forward(planes)
    _, _, _, b = _gpu_forward(planes, persistent_ctas=4)
    for k in ("rgb", "depth", "alpha", "t_final", "n_contrib", "n_iter"):
        assert np.array_equal(a[k], b[k]), k


def test_persistent_backward_matches_the_oracle(planes, planes_ref):
    """Forward and backward with persistent CTAs pulling tiles from a work queue
    (the autotuner's other launch form) match the oracle."""
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes, persistent_ctas=4)
    assert_images_close(out, ref, ref["flags"], what="persistent")
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


def test_multiview_pose_gradients_and_ragged_image():
    sc = scenes.random_gaussians(300, 97, 61, 80.0, seed=21, scale_range=(0.02, 0.2), n_views=3)
    g_up = scenes.upstream_grads(3, 3, 61, 97)
    ref0 = oracle.render_scene(sc)
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, grads=gm)
    r, g, T, out = _gpu_forward(sc)
    assert_images_close(out, ref, ref["flags"], what="3 views")
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


def test_more_views_than_one_cull_round():
    """Ten views in one call: the pre-cull and the merged cull-and-projection
    take views in rounds of eight, so the second round holds two.  The images
    equal separate one-view renders bit for bit; gradients and poses match the
    oracle."""
    sc = scenes.random_gaussians(800, 96, 72, 90.0, seed=23, scale_range=(0.02, 0.15), n_views=10)
    r, g, T, out = _gpu_forward(sc)
    for v in (0, 7, 8, 9):
        o1 = _np(Renderer(intrinsics(sc), n_views=1).forward(*g, T[v:v + 1].contiguous()))
        for k in ("rgb", "depth", "alpha", "t_final", "n_contrib", "n_iter"):
            assert np.array_equal(out[k][v:v + 1], o1[k]), (v, k)
    g_up = scenes.upstream_grads(5, 10, 72, 96)
    ref0 = oracle.render_scene(sc)
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, grads=gm)
    assert_images_close(out, ref, ref["flags"], what="10 views")
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


@pytest.mark.parametrize("tile,height", [((8, 8), 123), ((16, 16), 290)])
def test_large_gaussians_spanning_many_tile_rows(tile, height):
    """Gaussians taller than 8 tile rows are emitted row-parallel (one warp per
    Gaussian): their tile counts, image and gradients still match the oracle."""
    sc = scenes.random_gaussians(40, 161, height, 90.0, seed=17, scale_range=(0.15, 0.6), depth=(1.2, 3.0))
    r, g, T, out = _gpu_forward(sc, tile_w=tile[0], tile_h=tile[1])
    p = {k: v.cpu().numpy() for k, v in r.project(*g, T).items()}
    cnt, rect = p["tile_count"][0], p["tile_rect"][0]  # rect: tx0, tx1, ty0, ty1
    assert ((rect[:, 3] - rect[:, 2] + 1)[cnt > 0] > 8).sum() >= 5  # the row-parallel path is taken
    ref0 = oracle.render_scene(sc)
    cover = oracle.tile_cover(ref0["proj"][0], sc.opacities, sc.camera.width, sc.camera.height,
                              Options(tile_w=tile[0], tile_h=tile[1]))
    mask = tile_count_mask(ref0["extent"][0], sc.opacities) | cover["flags"]
    assert np.array_equal(cnt[~mask], cover["count"][~mask])
    assert_images_close(out, ref0, ref0["flags"], what=f"large {tile}")
    g_up = scenes.upstream_grads(19, 1, height, 161)
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, grads=gm)
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


def test_many_tiles_render_every_tile_once():
    """43,200 tiles (3 views of 1280x720 in 8x8 tiles) are more than the
    launch-order kernel keeps in registers (32 per thread): every tile is still
    composited once, forward (full images against the oracle) and backward
    (against the same render in 16x16 tiles, 10,800 tiles)."""
    sc = scenes.random_gaussians(1500, 1280, 720, 700.0, seed=23, scale_range=(0.005, 0.03), n_views=3)
    ref = oracle.render_scene(sc)
    r8, g, T, out8 = _gpu_forward(sc, tile_w=8, tile_h=8, instances_per_gaussian=64)
    assert_images_close(out8, ref, ref["flags"], what="8x8, 43,200 tiles")
    r16, _, _, out16 = _gpu_forward(sc, tile_w=16, tile_h=16)
    gm = masked_upstream(scenes.upstream_grads(29, 3, 720, 1280), ref["flags"])
    a, pa = _gpu_backward(r8, g, T, out8, gm)
    b, pb = _gpu_backward(r16, g, T, out16, gm)
    for k in GRAD_KEYS:
        assert_grad_close(a[k], b[k], k)
    assert_pose_close(pa, pb)


def test_background_and_depth_only_upstream():
    sc = scenes.random_gaussians(200, 64, 48, 60.0, seed=5, scale_range=(0.02, 0.2))
    bg = (0.2, 0.4, 0.6)
    ref0 = oracle.render_scene(sc, opts=Options(bg=bg))
    g_up = scenes.upstream_grads(8, 1, 48, 64)
    g_up = (np.zeros_like(g_up[0]), g_up[1], np.zeros_like(g_up[2]))
    gm = masked_upstream(g_up, ref0["flags"])
    ref = oracle.render_scene(sc, opts=Options(bg=bg), grads=gm)
    r, g, T, out = _gpu_forward(sc, bg=bg)
    assert_images_close(out, ref, ref["flags"], what="bg")
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in ("means", "scales", "quats", "opacities"):
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert np.all(grads["colors"] == 0.0)


def test_empty_and_fully_culled_scenes():
    sc = scenes.random_gaussians(50, 40, 30, 40.0, seed=1)
    sc.means[:, 2] = -1.0  # behind the camera
    _, _, _, out = _gpu_forward(sc)
    assert out["alpha"].max() == 0.0 and out["n_contrib"].max() == 0
    assert np.all(out["t_final"] == 1.0)
    e = scenes.random_gaussians(1, 40, 30, 40.0, seed=1)
    r = Renderer(intrinsics(e))
    z = torch.zeros((0, 3), device="cuda")
    out = r.forward(z, z.clone(), torch.zeros((0, 4), device="cuda"), torch.zeros(0, device="cuda"),
                    z.clone(), dev(e.camera.T_cw, torch.float64))
    assert float(out["alpha"].abs().max()) == 0.0


def test_capacity_overflow_is_reported_then_grown(planes):
    r = Renderer(intrinsics(planes), instances_per_gaussian=0.01)
    g, T = scene_tensors(planes)
    r.reserve(planes.n, max_instances=100)
    out = r.forward(*g, T, check=False)
    st = r.stats()
    assert st.status == 2
    out = r.forward(*g, T, check=True)  # grows the workspace and renders
    assert r.stats().status == 0
    assert r.cap_m >= r.last_stats.n_instances
    del out


def test_lookback_wait_limit_reports_timeout():
    """A look-back wait limit of one poll makes the binning's scans and sorts give
    up on predecessors that have not published yet: the call records
    VPGS_ERR_TIMEOUT, writes nothing outside its workspace and images, and the
    next call with the default limit renders exactly as a fresh renderer does."""
    sc = scenes.random_gaussians(300_000, 640, 480, 500.0, seed=33, scale_range=(0.005, 0.02))
    g, T = scene_tensors(sc)
    r = Renderer(intrinsics(sc), spin_limit=1)
    r.reserve(sc.n)
    guard = 1 << 16
    ws = torch.full((r.ws_bytes + guard,), 0xA5, dtype=torch.uint8, device="cuda")
    r.ws = ws[:r.ws_bytes]  # same base address, so still 16-byte aligned
    bigs, out = {}, {}
    for k, t in r.alloc_images().items():
        big = torch.full((t.numel() + guard,), -7, dtype=t.dtype, device="cuda")
        bigs[k] = big
        out[k] = big[:t.numel()].view(t.shape)
    codes = []
    for _ in range(20):
        r.forward(*g, T, out=out, check=False)
        codes.append(int(r.stats().status))
        if codes[-1] == 4:
            break
    assert codes[-1] == 4 and set(codes) <= {0, 4}, codes
    assert bool((ws[r.ws_bytes:] == 0xA5).all())
    for k, big in bigs.items():
        assert bool((big[-guard:] == -7).all()), k
    r.opts.spin_limit = 0
    a = _np(r.forward(*g, T))
    assert r.stats().status == 0
    b = _np(Renderer(intrinsics(sc)).forward(*g, T))
    for k in ("rgb", "depth", "alpha", "t_final", "n_contrib", "n_iter"):
        assert np.array_equal(a[k], b[k]), k


def test_nonfinite_input_sets_status():
    sc = scenes.random_gaussians(20, 32, 24, 30.0, seed=2)
    sc.means[3, 0] = np.nan
    r = Renderer(intrinsics(sc))
    g, T = scene_tensors(sc)
    r.forward(*g, T, check=False)
    assert r.stats().status == 3


def test_invalid_arguments_are_rejected_on_the_host(planes):
    r = Renderer(intrinsics(planes))
    g, T = scene_tensors(planes)
    r.reserve(planes.n)
    gs = r._gauss(*g)
    bad = C.default_opts(tile_w=3)
    out = r.alloc_images()
    code = C.vpgs_render_fwd(r.ws.data_ptr(), r.ws_bytes, ctypes.byref(gs), ctypes.byref(r.cam),
                             T.data_ptr(), 1, ctypes.byref(bad), ctypes.byref(r._images(out)), None)
    assert code == 1
    code = C.vpgs_render_fwd(r.ws.data_ptr(), 1024, ctypes.byref(gs), ctypes.byref(r.cam),
                             T.data_ptr(), 1, ctypes.byref(r.opts), ctypes.byref(r._images(out)), None)
    assert code == 1


def test_autograd_function_matches_direct_calls(planes, planes_ref):
    ref, gm = planes_ref
    r = Renderer(intrinsics(planes))
    g, T = scene_tensors(planes)
    leaves = [t.clone().requires_grad_(True) for t in g]
    xi = torch.zeros((1, 6), dtype=torch.float64, device="cuda", requires_grad=True)
    rgb, depth, alpha = render(*leaves, T, r, xi=xi)
    L = (rgb * dev(gm[0])).sum() + (depth * dev(gm[1])).sum() + (alpha * dev(gm[2])).sum()
    L.backward()
    for k, leaf in zip(GRAD_KEYS, leaves):
        assert_grad_close(leaf.grad.cpu().numpy(), ref["d_" + k], k)
    assert_pose_close(xi.grad.cpu().numpy(), ref["d_pose"])


def test_autograd_render_checks_status_without_waiting(planes):
    """render() queues the status word instead of waiting for it: an instance
    overflow surfaces at renderer.check() (or a later render), not silently."""
    r = Renderer(intrinsics(planes))
    g, T = scene_tensors(planes)
    r.reserve(planes.n, max_instances=100)
    leaves = [t.clone().requires_grad_(True) for t in g]
    rgb, depth, alpha = render(*leaves, T, r)
    with pytest.raises(RuntimeError, match="capacity"):
        r.check()
    r.reserve(planes.n, max_instances=24 * planes.n)
    rgb, depth, alpha = render(*leaves, T, r)
    (rgb.sum() + depth.sum()).backward()
    r.check()
    assert not r._pending


def test_backward_reusing_the_forward_lists(planes, planes_ref):
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes)
    a, pa = _gpu_backward(r, g, T, out, gm, reuse=True)
    for k in GRAD_KEYS:
        assert_grad_close(a[k], ref["d_" + k], k)
    assert_pose_close(pa, ref["d_pose"])
    # a second reusing backward sees zeroed 2D gradient slots again.  Float atomics
    # sum in a schedule-dependent order on every run: a Gaussian's 2D sums gather
    # hundreds of per-(warp, pixel) terms, each up to the array scale, so two runs
    # agree to about sqrt(terms) FP32 roundings of that scale (1e-5 of it)
    b, pb = _gpu_backward(r, g, T, out, gm, reuse=True)
    for k in GRAD_KEYS:
        np.testing.assert_allclose(b[k], a[k], rtol=0, atol=1e-5 * np.abs(a[k]).max(), err_msg=k)
    np.testing.assert_allclose(pb, pa, rtol=1e-5, atol=1e-9 * np.abs(pa).max())


def test_reuse_after_another_forward_recomputes(planes, planes_ref):
    ref, gm = planes_ref
    r, g, T, out = _gpu_forward(planes)
    T2 = T.clone()
    T2[0, 0, 3] += 0.05
    r.forward(*g, T2)  # replaces the lists: the backward below must not take them
    a, pa = _gpu_backward(r, g, T, out, gm, reuse=True)
    for k in GRAD_KEYS:
        assert_grad_close(a[k], ref["d_" + k], k)
    assert_pose_close(pa, ref["d_pose"])


def test_autograd_backward_after_a_second_render(planes, planes_ref):
    ref, gm = planes_ref
    r = Renderer(intrinsics(planes))
    g, T = scene_tensors(planes)
    leaves = [t.clone().requires_grad_(True) for t in g]
    rgb, depth, alpha = render(*leaves, T, r)
    with torch.no_grad():
        render(*g, T + 0.0, r)  # another render on the same renderer before the backward
    L = (rgb * dev(gm[0])).sum() + (depth * dev(gm[1])).sum() + (alpha * dev(gm[2])).sum()
    L.backward()
    for k, leaf in zip(GRAD_KEYS, leaves):
        assert_grad_close(leaf.grad.cpu().numpy(), ref["d_" + k], k)


def test_full_size_room_sampled_rows():
    # the 1M-Gaussian 1200x680 room in the benchmark's launch configuration,
    # compared on sampled rows the oracle evaluates one by one
    sc = scenes.indoor_room()
    rows = [0, 171, 340, 521, 679]
    g_up = scenes.upstream_grads(11, 1, 680, 1200)
    ref0 = oracle.render_scene(sc, rows=rows)
    sel = np.zeros_like(ref0["flags"])
    sel[:, rows] = True
    ignore = ref0["flags"] | ~sel
    r, g, T, out = _gpu_forward(sc)
    shown = {k: (np.where(sel[:, None], v, 0) if k == "rgb" else np.where(sel, v, 0))
             for k, v in out.items()}
    assert_images_close(shown, ref0, ignore, what="room rows")
    # gradients from the sampled rows only
    gm = masked_upstream(g_up, ignore)
    ref = oracle.render_scene(sc, rows=rows, grads=gm)
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


def test_one_view_with_more_visible_pairs_than_one_sort_round():
    # 400,000 Gaussians, all in front of one 320x240 camera: the depth sort's
    # tiles (1,024 keys) and the instance-offset scan's tiles outnumber their
    # grids of 2 blocks per SM, so blocks take several tiles from the ticket
    sc = scenes.random_gaussians(400_000, 320, 240, 300.0, seed=41, scale_range=(0.002, 0.012))
    rows = [0, 120, 239]
    g_up = scenes.upstream_grads(12, 1, 240, 320)
    ref0 = oracle.render_scene(sc, rows=rows)
    sel = np.zeros_like(ref0["flags"])
    sel[:, rows] = True
    ignore = ref0["flags"] | ~sel
    r, g, T, out = _gpu_forward(sc)
    shown = {k: (np.where(sel[:, None], v, 0) if k == "rgb" else np.where(sel, v, 0))
             for k, v in out.items()}
    assert_images_close(shown, ref0, ignore, what="400k visible rows")
    gm = masked_upstream(g_up, ignore)
    ref = oracle.render_scene(sc, rows=rows, grads=gm)
    grads, dpose = _gpu_backward(r, g, T, out, gm)
    for k in GRAD_KEYS:
        assert_grad_close(grads[k], ref["d_" + k], k)
    assert_pose_close(dpose, ref["d_pose"])


def test_batched_views_equal_separate_views():
    sc = scenes.random_gaussians(3000, 160, 120, 140.0, seed=31, scale_range=(0.01, 0.1), n_views=4)
    r, g, T, out = _gpu_forward(sc)
    for v in range(4):
        r1 = Renderer(intrinsics(sc), n_views=1)
        o1 = _np(r1.forward(*g, T[v:v + 1].contiguous()))
        for k in ("rgb", "depth", "alpha", "t_final", "n_contrib", "n_iter"):
            assert np.array_equal(out[k][v:v + 1], o1[k]), (v, k)


def test_full_size_batched_keyframes_sampled_rows():
    # 2M Gaussians, 8 keyframes at 640x480 in one call, as timed by the benchmark
    sc = scenes.batched_keyframes()
    rows = [0, 239, 479]
    views = [0, 7]
    sub = scenes.GaussianScene("kf", sc.means, sc.scales, sc.quats, sc.opacities, sc.colors,
                               scenes.Camera(640, 480, sc.camera.fx, sc.camera.fy, sc.camera.cx, sc.camera.cy,
                                             sc.camera.T_cw[views]))
    ref = oracle.render_scene(sub, rows=rows)
    sel = np.zeros_like(ref["flags"])
    sel[:, rows] = True
    _, _, _, out = _gpu_forward(sc)
    shown = {k: (np.where(sel[:, None], v[views], 0) if k == "rgb" else np.where(sel, v[views], 0))
             for k, v in out.items()}
    assert_images_close(shown, ref, ref["flags"] | ~sel, what="keyframes")


@pytest.mark.parametrize("tile", [(8, 16), (16, 8)])
def test_tile_counts_other_shapes(planes, tile):
    from oracle.raster import Options, _t
    opts = Options(tile_w=tile[0], tile_h=tile[1])
    cam = planes.camera
    pr = oracle.project(_t(planes.means), _t(planes.scales), _t(planes.quats), _t(cam.T_cw[0]),
                        cam.fx, cam.fy, cam.cx, cam.cy, opts)
    ext = oracle.extent(pr, planes.opacities, cam.width, cam.height, opts)
    r = Renderer(intrinsics(planes), tile_w=tile[0], tile_h=tile[1])
    g, T = scene_tensors(planes)
    cnt = r.project(*g, T)["tile_count"][0].cpu().numpy()
    cover = oracle.tile_cover(pr, planes.opacities, cam.width, cam.height, opts)
    mask = tile_count_mask(ext, planes.opacities) | cover["flags"]
    assert np.array_equal(cnt[~mask], cover["count"][~mask])
