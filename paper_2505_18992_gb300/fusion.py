"""Submap fusion front end: Eq. 14 distillation loss and the Adam step (argument marshalling)."""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .render import current_stream_handle


class DistillLoss:
    """L = 1/m sum_kf (mean (c_a - c_b)^2 + mean (d_a - d_b)^2) over m keyframes."""

    def __init__(self, n_views: int, width: int, height: int, device="cuda"):
        self.V, self.W, self.H = int(n_views), int(width), int(height)
        n = C.vpgs_distill_workspace_bytes(self.V, self.W, self.H)
        if n == 0:
            raise ValueError("invalid image size")
        self.ws = torch.empty(n, dtype=torch.uint8, device=device)
        self.loss = torch.zeros(3, dtype=torch.float64, device=device)

    def __call__(self, rgb_a, rgb_b, depth_a=None, depth_b=None, d_rgb_a=None, d_rgb_b=None, d_depth_a=None,
                 d_depth_b=None):
        C.check(C.vpgs_distill_loss(self.ws.data_ptr(), self.ws.numel(), C.ptr(rgb_a), C.ptr(rgb_b),
                                    C.ptr(depth_a), C.ptr(depth_b), self.V, self.W, self.H, C.ptr(self.loss),
                                    C.ptr(d_rgb_a), C.ptr(d_rgb_b), C.ptr(d_depth_a), C.ptr(d_depth_b),
                                    current_stream_handle()), "vpgs_distill_loss")
        return self.loss


class Adam:
    """Adam over one float32 CUDA tensor whose gradient lives in `grad` (zeroed by each step)."""

    def __init__(self, param: torch.Tensor, grad: torch.Tensor, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.p, self.g = param, grad
        self.m = torch.zeros_like(param)
        self.v = torch.zeros_like(param)
        self.hyper = (ctypes.c_float * 4)(lr, betas[0], betas[1], eps)
        self.t = 0

    def step(self):
        self.t += 1
        C.check(C.vpgs_adam_step(self.p.data_ptr(), self.g.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                 self.p.numel(), self.hyper, self.t, current_stream_handle()), "vpgs_adam_step")
