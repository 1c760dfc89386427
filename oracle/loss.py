"""FP64 CPU oracle of the mapping loss (Sec. III-A, Eq. 7-9).

TEST INFRASTRUCTURE.  Only the test-suite and the benchmark's CPU arms may
import this module; the product path never does.  It shares no code with the
CUDA path.

  L_m    = L_c + L_SSIM + lambda_d L_d + lambda_vol L_vol                 (Eq. 7)
  L_SSIM = (1 - lambda_SSIM) |I^ - I|_1 + lambda_SSIM (1 - SSIM(I^, I))   (Eq. 8)
  L_vol  = sum_i Prod(s_i)                                                (Eq. 9)

with lambda_SSIM = 0.2 and lambda_vol = 0.001 (Sec. IV).  Readings where the
paper is silent:
  * L_c and |.|_1 are mean absolute colour differences over all views,
    channels and pixels; L_d is the absolute depth difference summed over the
    pixels whose target depth is > 0 and divided by the number of pixels.
  * SSIM is the structural similarity of Wang et al. as 3D Gaussian Splatting
    evaluates it: an 11x11 Gaussian window with sigma 1.5 (normalised),
    zero-padded 'same' filtering per channel, C1 = 0.01^2, C2 = 0.03^2, and the
    mean of the SSIM map over views, channels and pixels.
  * lambda_d is an argument (1 by default).
Gradients are those of torch autograd through this code (|x| has derivative
sign(x), 0 at 0).

Coarse tracking (Sec. III-B) minimises the photometric and depth L1 errors of
the render at the current pose.  Reading: for each view v separately,
  L_t(v) = (1 / 3HW) sum_{c,p} |I^ - I| + lambda_d (1 / HW) sum_{p: D(p) > 0} |D^ - D|,
the same colour and depth terms as the mapping loss, normalised per view so
that a view's pose gradient does not depend on how many views share a call.

Pins (tests/test_oracle_loss.py): SSIM(x, x) = 1, a constant-image closed form,
brute-force windows on tiny images, the window's normalisation and symmetry,
the volume term in closed form, and central differences of every gradient;
for the tracking loss a hand-worked 2x2 example and central differences.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

F64 = torch.float64
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """Normalised 2D Gaussian window (outer product of the 1D one)."""
    x = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def ssim_map(x: torch.Tensor, y: torch.Tensor, size: int = 11, sigma: float = 1.5) -> torch.Tensor:
    """SSIM map of two image batches [B, C, H, W] (zero-padded, per channel)."""
    C = x.shape[1]
    w = torch.as_tensor(gaussian_window(size, sigma), dtype=F64)[None, None].repeat(C, 1, 1, 1)
    pad = size // 2

    def blur(t):
        return F.conv2d(t, w, padding=pad, groups=C)

    mu_x, mu_y = blur(x), blur(y)
    s_xx = blur(x * x) - mu_x * mu_x
    s_yy = blur(y * y) - mu_y * mu_y
    s_xy = blur(x * y) - mu_x * mu_y
    return ((2 * mu_x * mu_y + C1) * (2 * s_xy + C2)) / ((mu_x * mu_x + mu_y * mu_y + C1) * (s_xx + s_yy + C2))


def mapping_loss(rgb, target_rgb, depth=None, target_depth=None, scales=None, lambda_ssim=0.2,
                 lambda_d=1.0, lambda_vol=0.001, grads=True):
    """rgb, target_rgb [V,3,H,W]; depth, target_depth [V,H,W] (optional);
    scales [N,3] (optional).  Returns a dict with the loss terms
    (L_m, L_c, L_SSIM, L_d, L_vol, ssim) and, with grads, d_rgb, d_depth, d_scales."""
    x = torch.as_tensor(np.asarray(rgb), dtype=F64).clone().requires_grad_(grads)
    y = torch.as_tensor(np.asarray(target_rgb), dtype=F64)
    l1 = (x - y).abs().mean()
    ssim = ssim_map(x, y).mean()
    L_c = l1
    L_ssim = (1.0 - lambda_ssim) * l1 + lambda_ssim * (1.0 - ssim)
    L_d = torch.zeros((), dtype=F64)
    d = None
    if depth is not None:
        d = torch.as_tensor(np.asarray(depth), dtype=F64).clone().requires_grad_(grads)
        td = torch.as_tensor(np.asarray(target_depth), dtype=F64)
        L_d = ((d - td).abs() * (td > 0)).sum() / d.numel()
    L_vol = torch.zeros((), dtype=F64)
    s = None
    if scales is not None:
        s = torch.as_tensor(np.asarray(scales), dtype=F64).clone().requires_grad_(grads)
        L_vol = s.prod(dim=1).sum()
    L_m = L_c + L_ssim + lambda_d * L_d + lambda_vol * L_vol
    out = {key: float(val.detach()) for key, val in (("L_m", L_m), ("L_c", L_c), ("L_SSIM", L_ssim),
                                                         ("L_d", L_d), ("L_vol", L_vol), ("ssim", ssim))}
    if grads:
        L_m.backward()
        out["d_rgb"] = x.grad.numpy().copy()
        out["d_depth"] = d.grad.numpy().copy() if d is not None else None
        out["d_scales"] = s.grad.numpy().copy() if s is not None else None
    return out


def tracking_loss(rgb, target_rgb, depth=None, target_depth=None, lambda_d=1.0, grads=True):
    """rgb, target_rgb [V,3,H,W]; depth, target_depth [V,H,W] (optional).
    Returns a dict with the per-view losses "L_t" [V] and, with grads, d_rgb and
    d_depth (the gradient of sum_v L_t(v))."""
    x = torch.as_tensor(np.asarray(rgb), dtype=F64).clone().requires_grad_(grads)
    y = torch.as_tensor(np.asarray(target_rgb), dtype=F64)
    V, _, H, W = x.shape
    L = (x - y).abs().reshape(V, -1).sum(1) / (3 * H * W)
    d = None
    if depth is not None:
        d = torch.as_tensor(np.asarray(depth), dtype=F64).clone().requires_grad_(grads)
        td = torch.as_tensor(np.asarray(target_depth), dtype=F64)
        L = L + lambda_d * ((d - td).abs() * (td > 0)).reshape(V, -1).sum(1) / (H * W)
    out = {"L_t": L.detach().numpy().copy()}
    if grads:
        L.sum().backward()
        out["d_rgb"] = x.grad.numpy().copy()
        out["d_depth"] = d.grad.numpy().copy() if d is not None else None
    return out


__all__ = ["gaussian_window", "ssim_map", "mapping_loss", "tracking_loss", "C1", "C2"]
