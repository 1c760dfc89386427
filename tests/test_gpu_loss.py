"""GPU mapping loss (Eq. 7-9) through the C ABI against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2505_18992_gb300 import vpgs as C
from paper_2505_18992_gb300.loss import MappingLoss, default_weights
from tests.helpers import assert_grad_close, dev

pytestmark = pytest.mark.gpu

TERMS = ("L_m", "L_c", "L_SSIM", "L_d", "L_vol")


def _case(V, H, W, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(V, 3, H, W))
    y = np.clip(x + rng.normal(scale=0.15, size=x.shape), 0, 1)
    d = rng.uniform(1, 4, size=(V, H, W))
    td = d + rng.normal(scale=0.1, size=d.shape)
    td[:, : H // 4] = 0.0  # no target depth in the top rows
    s = rng.uniform(0.005, 0.05, size=(n, 3))
    return [a.astype(np.float32).astype(np.float64) for a in (x, y, d, td, s)]


def _gpu(x, y, d, td, s, n_live=None, **w):
    V, _, H, W = x.shape
    L = MappingLoss(V, W, H, **w)
    gr = torch.empty((V, 3, H, W), device="cuda")
    gd = torch.empty((V, H, W), device="cuda")
    gs = torch.zeros((s.shape[0], 3), device="cuda")
    n_dev = None if n_live is None else torch.tensor([n_live], dtype=torch.int32, device="cuda")
    loss = L(dev(x), dev(y), dev(d), dev(td), dev(s), n_dev=n_dev, d_rgb=gr, d_depth=gd, d_scales=gs)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), gr.cpu().numpy(), gd.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("shape", [(2, 45, 70), (1, 32, 48), (3, 17, 5)])
def test_loss_and_gradients_match_the_oracle(shape):
    V, H, W = shape
    x, y, d, td, s = _case(V, H, W, 301, seed=H + W)
    ref = oracle.mapping_loss(x, y, d, td, s, lambda_d=0.7)
    loss, gr, gd, gs = _gpu(x, y, d, td, s, lambda_d=0.7)
    for i, k in enumerate(TERMS):
        assert abs(loss[i] - ref[k]) <= 2e-6 * max(1.0, abs(ref[k])), (k, loss[i], ref[k])
    assert_grad_close(gr, ref["d_rgb"], "rgb")
    assert_grad_close(gd, ref["d_depth"], "depth")
    assert_grad_close(gs, ref["d_scales"], "scales")


def test_device_count_limits_the_volume_term():
    x, y, d, td, s = _case(1, 20, 24, 50, seed=9)
    ref = oracle.mapping_loss(x, y, d, td, s[:31])
    loss, _, _, gs = _gpu(x, y, d, td, s, n_live=31)
    assert abs(loss[4] - ref["L_vol"]) <= 1e-6 * ref["L_vol"]
    assert np.abs(gs[31:]).max() == 0.0
    assert_grad_close(gs[:31], ref["d_scales"], "scales")


def test_identical_images_give_zero_colour_terms():
    x, _, d, td, s = _case(1, 40, 40, 10, seed=5)
    loss, gr, _, _ = _gpu(x, x, d, td, s)
    assert abs(loss[1]) == 0.0 and abs(loss[2]) < 1e-6
    assert np.abs(gr).max() < 1e-6


def test_full_size_frame():
    # one 1200x680 view, the size the mapping step renders
    x, y, d, td, s = _case(1, 680, 1200, 1000, seed=11)
    ref = oracle.mapping_loss(x, y, d, td, s)
    loss, gr, gd, gs = _gpu(x, y, d, td, s)
    for i, k in enumerate(TERMS):
        assert abs(loss[i] - ref[k]) <= 2e-6 * max(1.0, abs(ref[k])), k
    assert_grad_close(gr, ref["d_rgb"], "rgb")
    assert_grad_close(gd, ref["d_depth"], "depth")


def test_bad_arguments_are_rejected():
    w = default_weights()
    assert C.vpgs_mapping_loss_workspace_bytes(0, 10, 10) == 0
    assert C.vpgs_mapping_loss(None, 0, None, None, None, None, 1, 8, 8, None, 0, None, ctypes.byref(w),
                               None, None, None, None, None) == 1
    L = MappingLoss(1, 8, 8)
    t = torch.zeros((1, 3, 8, 8), device="cuda")
    bad = default_weights(lambda_ssim=1.5)
    code = C.vpgs_mapping_loss(L.ws.data_ptr(), L.ws.numel(), t.data_ptr(), t.data_ptr(), None, None, 1, 8, 8,
                               None, 0, None, ctypes.byref(bad), L.loss.data_ptr(), None, None, None, None)
    assert code == 1


def _tracking_gpu(x, y, d, td, lambda_d, with_depth=True):
    V, _, H, W = x.shape
    loss = torch.full((V,), -1.0, dtype=torch.float64, device="cuda")
    gr = torch.full((V, 3, H, W), 7.0, device="cuda")
    gd = torch.full((V, H, W), 7.0, device="cuda")
    xt, yt = dev(x), dev(y)  # held: the call takes raw addresses
    dt, tdt = (dev(d), dev(td)) if with_depth else (None, None)
    code = C.vpgs_tracking_loss(C.ptr(xt), C.ptr(yt), C.ptr(dt), C.ptr(tdt), V, W, H, lambda_d, C.ptr(loss),
                                C.ptr(gr), C.ptr(gd), None)
    assert code == 0
    torch.cuda.synchronize()
    return loss.cpu().numpy(), gr.cpu().numpy(), gd.cpu().numpy()


@pytest.mark.parametrize("shape", [(2, 45, 70), (3, 17, 5), (1, 680, 1200)])
def test_tracking_loss_matches_the_oracle(shape):
    """Per-view colour + depth L1 of coarse tracking: the gradients are sign x
    weight, so both sides agree bit for bit once the FP64 weights are rounded
    to float32 (the sign of a float32 difference is exact); the per-view loss
    is an FP32 / FP64 sum, 2e-6 relative."""
    V, H, W = shape
    x, y, d, td, _ = _case(V, H, W, 1, seed=H * W)
    y[0, 1, 0, :3] = x[0, 1, 0, :3]  # exact ties: zero gradient
    d[0, 2, :5] = td[0, 2, :5]
    ref = oracle.tracking_loss(x, y, d, td, lambda_d=0.5)
    loss, gr, gd = _tracking_gpu(x, y, d, td, 0.5)
    assert np.all(np.abs(loss - ref["L_t"]) <= 2e-6 * np.maximum(1.0, np.abs(ref["L_t"])))
    assert np.array_equal(gr, ref["d_rgb"].astype(np.float32))
    assert np.array_equal(gd, ref["d_depth"].astype(np.float32))
    assert gr[0, 1, 0, 0] == 0.0 and gd[0, 0, 0] == 0.0  # a tie, a pixel without a target depth


def test_tracking_loss_without_depth_and_bad_arguments():
    x, y, d, td, _ = _case(2, 19, 33, 1, seed=3)
    ref = oracle.tracking_loss(x, y)
    loss, gr, gd = _tracking_gpu(x, y, d, td, 1.0, with_depth=False)
    assert np.all(np.abs(loss - ref["L_t"]) <= 2e-6)
    assert np.array_equal(gr, ref["d_rgb"].astype(np.float32))
    assert np.all(gd == 7.0)  # untouched without depths
    t = torch.zeros((1, 3, 8, 8), device="cuda")
    assert C.vpgs_tracking_loss(None, t.data_ptr(), None, None, 1, 8, 8, 1.0, None, None, None, None) == 1
    assert C.vpgs_tracking_loss(t.data_ptr(), t.data_ptr(), t.data_ptr(), None, 1, 8, 8, 1.0, None, None, None,
                                None) == 1
    assert C.vpgs_tracking_loss(t.data_ptr(), t.data_ptr(), None, None, 0, 8, 8, 1.0, None, None, None, None) == 1
    assert C.vpgs_tracking_loss(t.data_ptr(), t.data_ptr(), None, None, 1, 8, 8, -1.0, None, None, None, None) == 1
