"""FP64 CPU oracle of submap fusion by distillation (Sec. III-C, Eq. 14) and of
the Adam step the fusion loop takes on the submaps' parameters.

TEST INFRASTRUCTURE.  Only the test-suite and the benchmark's CPU arms may
import this module; the product path never does.  It shares no code with the
CUDA path.

  L = 1/m sum_{keyframes} ( (c_a - c_b)^2 + (d_a - d_b)^2 )            (Eq. 14)

c_a, c_b: the colour renders of the same keyframe from submaps a and b,
d_a, d_b: the depth renders.  Reading (the paper does not say how the squared
differences of an image are combined): the mean over channels and pixels for
the colour term and over pixels for the depth term, then the mean over the m
keyframes.  Adam is Kingma and Ba's, with bias correction.

Pins (tests/test_oracle_fusion.py): zero loss and gradients for identical
renders, a hand-worked 2-pixel case, the 1/m over keyframes (duplicated and
zero-difference keyframes), central differences of the gradients, and Adam's
first step (lr * g / (|g| + eps)) and a hand-worked second step.
"""
from __future__ import annotations

import numpy as np
import torch

F64 = torch.float64


def distill_loss(rgb_a, rgb_b, depth_a, depth_b, grads=True):
    """rgb_* [m,3,H,W], depth_* [m,H,W] -> dict L, L_c, L_d and the gradients."""
    a = torch.as_tensor(np.asarray(rgb_a), dtype=F64).clone().requires_grad_(grads)
    b = torch.as_tensor(np.asarray(rgb_b), dtype=F64).clone().requires_grad_(grads)
    da = torch.as_tensor(np.asarray(depth_a), dtype=F64).clone().requires_grad_(grads)
    db = torch.as_tensor(np.asarray(depth_b), dtype=F64).clone().requires_grad_(grads)
    m = a.shape[0]
    per_kf = ((a - b) ** 2).reshape(m, -1).mean(1) + ((da - db) ** 2).reshape(m, -1).mean(1)
    L = per_kf.mean()
    L_c = ((a - b) ** 2).reshape(m, -1).mean(1).mean()
    L_d = ((da - db) ** 2).reshape(m, -1).mean(1).mean()
    out = {"L": float(L.detach()), "L_c": float(L_c.detach()), "L_d": float(L_d.detach())}
    if grads:
        L.backward()
        out.update(d_rgb_a=a.grad.numpy().copy(), d_rgb_b=b.grad.numpy().copy(),
                   d_depth_a=da.grad.numpy().copy(), d_depth_b=db.grad.numpy().copy())
    return out


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns (p, m, v)."""
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


__all__ = ["distill_loss", "adam_step"]
