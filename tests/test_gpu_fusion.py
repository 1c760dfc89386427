"""GPU Eq. 14 distillation loss and Adam step through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_18992_gb300.fusion import Adam, DistillLoss
from tests.helpers import assert_grad_close, dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(4, 33, 47), (1, 480, 640)])
def test_distill_loss_matches_the_oracle(shape):
    m, H, W = shape
    rng = np.random.default_rng(H)
    a = rng.uniform(size=(m, 3, H, W)).astype(np.float32).astype(np.float64)
    b = np.clip(a + rng.normal(scale=0.1, size=a.shape), 0, 1).astype(np.float32).astype(np.float64)
    da = rng.uniform(1, 5, size=(m, H, W)).astype(np.float32).astype(np.float64)
    db = (da + rng.normal(scale=0.2, size=da.shape)).astype(np.float32).astype(np.float64)
    ref = oracle.distill_loss(a, b, da, db)
    L = DistillLoss(m, W, H)
    g = [torch.empty(a.shape, device="cuda"), torch.empty(a.shape, device="cuda"),
         torch.empty(da.shape, device="cuda"), torch.empty(da.shape, device="cuda")]
    loss = L(dev(a), dev(b), dev(da), dev(db), *g).cpu().numpy()
    for i, k in enumerate(("L", "L_c", "L_d")):
        assert abs(loss[i] - ref[k]) <= 1e-6 * ref[k], k
    for t, k in zip(g, ("d_rgb_a", "d_rgb_b", "d_depth_a", "d_depth_b")):
        assert_grad_close(t.cpu().numpy(), ref[k], k)


def test_distill_identical_renders_and_colour_only():
    rng = np.random.default_rng(3)
    a = rng.uniform(size=(2, 3, 20, 30))
    L = DistillLoss(2, 30, 20)
    assert float(L(dev(a), dev(a))[0]) == 0.0
    b = a + 0.25
    loss = L(dev(a), dev(b)).cpu().numpy()
    assert abs(loss[0] - 0.0625) < 1e-7 and loss[2] == 0.0


def test_adam_steps_match_the_oracle():
    rng = np.random.default_rng(4)
    n = 10_000
    p = rng.normal(size=n)
    m_ref, v_ref, p_ref = np.zeros(n), np.zeros(n), p.copy()
    pt = dev(p)
    gt = torch.zeros(n, device="cuda")
    opt = Adam(pt, gt, lr=0.01)
    for t in range(1, 4):
        g = rng.normal(size=n).astype(np.float32).astype(np.float64)
        gt.copy_(dev(g))
        opt.step()
        p_ref, m_ref, v_ref = oracle.adam_step(p_ref, g, m_ref, v_ref, t, lr=0.01)
    torch.cuda.synchronize()
    assert np.abs(pt.cpu().numpy() - p_ref).max() < 1e-5
    assert float(gt.abs().max()) == 0.0  # the gradient is consumed
