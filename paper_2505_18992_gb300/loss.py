"""Mapping loss front end (Eq. 7-9): workspace management around vpgs_mapping_loss."""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .render import current_stream_handle


def default_weights(**kw) -> C.vpgs_loss_weights:
    w = C.vpgs_loss_weights()
    C.vpgs_loss_weights_default(ctypes.byref(w))
    for k, v in kw.items():
        setattr(w, k, v)
    return w


class MappingLoss:
    """L_m = L_c + L_SSIM + lambda_d L_d + lambda_vol L_vol and its gradient for
    V views of width x height (all tensors float32 CUDA, contiguous)."""

    def __init__(self, n_views: int, width: int, height: int, device="cuda", **weights):
        self.V, self.W, self.H = int(n_views), int(width), int(height)
        self.w = default_weights(**weights)
        n = C.vpgs_mapping_loss_workspace_bytes(self.V, self.W, self.H)
        if n == 0:
            raise ValueError("invalid loss image size")
        self.ws = torch.empty(n, dtype=torch.uint8, device=device)
        self.loss = torch.zeros(5, dtype=torch.float64, device=device)

    def __call__(self, rgb, target_rgb, depth=None, target_depth=None, scales=None, n_dev=None,
                 d_rgb=None, d_depth=None, d_scales=None):
        """Writes the loss terms into self.loss (L_m, L_c, L_SSIM, L_d, L_vol) and
        the gradients into the given buffers (d_scales accumulates); returns self.loss."""
        n = 0 if scales is None else scales.shape[0]
        C.check(C.vpgs_mapping_loss(self.ws.data_ptr(), self.ws.numel(), C.ptr(rgb), C.ptr(target_rgb),
                                    C.ptr(depth), C.ptr(target_depth), self.V, self.W, self.H, C.ptr(scales),
                                    n, C.ptr(n_dev), ctypes.byref(self.w), C.ptr(self.loss), C.ptr(d_rgb),
                                    C.ptr(d_depth), C.ptr(d_scales), current_stream_handle()),
                "vpgs_mapping_loss")
        return self.loss
