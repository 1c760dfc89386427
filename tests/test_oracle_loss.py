"""Pins of the FP64 mapping-loss oracle (Eq. 7-9) against facts that do not come from it."""
import math

import numpy as np
import pytest

import oracle
from oracle.loss import C1, C2


def test_window_is_a_normalised_symmetric_gaussian():
    w = oracle.gaussian_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    # ratio of neighbouring 1D taps follows exp(-(2i+1)/(2 sigma^2))
    g = w[5] / w[5].sum()
    assert abs(g[6] / g[5] - math.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


def test_identical_images_have_ssim_one_and_zero_loss():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(2, 3, 17, 23))
    out = oracle.mapping_loss(x, x)
    assert abs(out["ssim"] - 1.0) < 1e-12
    assert abs(out["L_m"]) < 1e-12 and np.abs(out["d_rgb"]).max() < 1e-9


def test_constant_images_closed_form_in_the_interior():
    # away from the zero padding, mu = the constants and all variances vanish
    a, b = 0.3, 0.7
    x = np.full((1, 1, 25, 25), a)
    y = np.full((1, 1, 25, 25), b)
    import torch
    m = oracle.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    assert abs(m[0, 0, 12, 12] - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12


def _brute_ssim(x, y):
    """Per-pixel windows written out with explicit zero padding."""
    w = oracle.gaussian_window()
    C, H, W = x.shape
    out = np.zeros_like(x)
    for c in range(C):
        xp = np.pad(x[c], 5)
        yp = np.pad(y[c], 5)
        for i in range(H):
            for j in range(W):
                wx, wy = xp[i:i + 11, j:j + 11], yp[i:i + 11, j:j + 11]
                mx, my = (w * wx).sum(), (w * wy).sum()
                sxx = (w * wx * wx).sum() - mx * mx
                syy = (w * wy * wy).sum() - my * my
                sxy = (w * wx * wy).sum() - mx * my
                out[c, i, j] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def test_ssim_map_against_brute_force_windows():
    import torch
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 9, 14))
    y = np.clip(x + rng.normal(scale=0.1, size=x.shape), 0, 1)
    m = oracle.ssim_map(torch.tensor(x[None]), torch.tensor(y[None])).numpy()[0]
    assert np.abs(m - _brute_ssim(x, y)).max() < 1e-12


def test_loss_terms_and_volume_closed_form():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(1, 3, 12, 10))
    y = rng.uniform(size=(1, 3, 12, 10))
    d = rng.uniform(1, 3, size=(1, 12, 10))
    td = rng.uniform(1, 3, size=(1, 12, 10))
    td[0, :3] = 0.0  # no target depth there
    s = rng.uniform(0.01, 0.1, size=(7, 3))
    out = oracle.mapping_loss(x, y, d, td, s, lambda_d=0.5)
    l1 = np.abs(x - y).mean()
    assert abs(out["L_c"] - l1) < 1e-14
    assert abs(out["L_SSIM"] - (0.8 * l1 + 0.2 * (1 - out["ssim"]))) < 1e-14
    assert abs(out["L_d"] - (np.abs(d - td) * (td > 0)).sum() / d.size) < 1e-14
    assert abs(out["L_vol"] - (s[:, 0] * s[:, 1] * s[:, 2]).sum()) < 1e-15
    assert abs(out["L_m"] - (out["L_c"] + out["L_SSIM"] + 0.5 * out["L_d"] + 0.001 * out["L_vol"])) < 1e-14
    # the volume gradient is the product of the other two scales
    assert np.abs(out["d_scales"] - 0.001 * np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], 1)).max() < 1e-16


@pytest.mark.parametrize("seed", [3, 4])
def test_gradients_central_differences(seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(2, 3, 8, 9))
    y = rng.uniform(size=(2, 3, 8, 9))
    d = rng.uniform(1, 3, size=(2, 8, 9))
    td = rng.uniform(1, 3, size=(2, 8, 9))
    s = rng.uniform(0.01, 0.1, size=(5, 3))
    out = oracle.mapping_loss(x, y, d, td, s)
    h = 1e-6
    for _ in range(6):
        idx = tuple(rng.integers(0, n) for n in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        num = (oracle.mapping_loss(xp, y, d, td, s, grads=False)["L_m"] -
               oracle.mapping_loss(xm, y, d, td, s, grads=False)["L_m"]) / (2 * h)
        assert abs(num - out["d_rgb"][idx]) < 1e-6 * max(1.0, abs(num))
    for _ in range(3):
        idx = tuple(rng.integers(0, n) for n in d.shape)
        dp, dm = d.copy(), d.copy()
        dp[idx] += h
        dm[idx] -= h
        num = (oracle.mapping_loss(x, y, dp, td, s, grads=False)["L_m"] -
               oracle.mapping_loss(x, y, dm, td, s, grads=False)["L_m"]) / (2 * h)
        assert abs(num - out["d_depth"][idx]) < 1e-6


def test_tracking_loss_hand_worked():
    # view 0: one colour channel differs at two pixels, one depth pixel has no target
    x = np.full((2, 3, 2, 2), 0.5)
    y = x.copy()
    y[0, 0] = [[0.25, 0.5], [1.0, 0.5]]
    d = np.full((2, 2, 2), 2.0)
    td = np.array([[[1.0, 0.0], [3.0, 2.0]], [[2.0, 2.0], [2.0, 2.0]]])
    out = oracle.tracking_loss(x, y, d, td, lambda_d=0.5)
    # colour: (0.25 + 0.5) / 12; depth: 0.5 * (1 + 1) / 4 (the pixel without a target is left out)
    assert np.allclose(out["L_t"], [0.75 / 12 + 0.25, 0.0], atol=1e-15)
    g = np.zeros_like(x)
    g[0, 0, 0, 0], g[0, 0, 1, 0] = 1 / 12, -1 / 12
    assert np.array_equal(out["d_rgb"], g)
    gd = np.zeros_like(d)
    gd[0, 0, 0], gd[0, 1, 0] = 0.125, -0.125
    assert np.array_equal(out["d_depth"], gd)
    # no depth: the colour term alone
    assert np.allclose(oracle.tracking_loss(x, y)["L_t"], [0.75 / 12, 0.0], atol=1e-15)


def test_tracking_loss_central_differences():
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(2, 3, 5, 7))
    y = rng.uniform(size=(2, 3, 5, 7))
    d = rng.uniform(1, 3, size=(2, 5, 7))
    td = rng.uniform(1, 3, size=(2, 5, 7))
    td[0, 1, 2] = 0.0
    out = oracle.tracking_loss(x, y, d, td, lambda_d=0.7)
    h = 1e-7
    total = lambda *a: oracle.tracking_loss(*a, lambda_d=0.7, grads=False)["L_t"].sum()  # noqa: E731
    for _ in range(6):
        idx = tuple(rng.integers(0, n) for n in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        num = (total(xp, y, d, td) - total(xm, y, d, td)) / (2 * h)
        assert abs(num - out["d_rgb"][idx]) < 1e-6
    for idx in [(0, 1, 2), (1, 4, 6), (0, 0, 0)]:
        dp, dm = d.copy(), d.copy()
        dp[idx] += h
        dm[idx] -= h
        num = (total(x, y, dp, td) - total(x, y, dm, td)) / (2 * h)
        assert abs(num - out["d_depth"][idx]) < 1e-6
