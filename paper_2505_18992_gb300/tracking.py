"""Coarse pose tracking by photometric + depth L1 (Sec. III-B), replayed from a CUDA graph.

One iteration: render the current pose, take the L1 gradients against the
frame (vpgs_tracking_loss: colour, and depth weighted by lambda_d where the
frame has a depth), back-propagate to the pose only (the compositing backward
then sums only the geometric 2D gradients), and step the pose on the device
(vpgs_pose_step, Adam).  The paper gives
neither the iteration count nor the step rule; 50 Adam iterations is the
tracking workload used here.  All buffers are preallocated, so `iters`
iterations can be captured once and replayed with a single host call.  The
backward of an iteration takes the forward's tile lists (same pose, same
workspace) unless reuse_binning=False.
"""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .render import Renderer, current_stream_handle


class Tracker:
    def __init__(self, renderer: Renderer, gaussians, T_cw: torch.Tensor, target_rgb: torch.Tensor,
                 target_depth: torch.Tensor, lr=(1e-3, 1e-3), lambda_d: float = 1.0, reuse_binning: bool = True):
        self.r = renderer
        self.g = [t.contiguous() for t in gaussians]
        self.T = T_cw  # [V,4,4] float64, updated in place
        self.target_rgb = target_rgb.contiguous()
        self.target_depth = None if target_depth is None else target_depth.contiguous()
        self.lr = (ctypes.c_double * 2)(*lr)
        self.lambda_d = lambda_d
        # within an iteration the forward and the backward see one pose and run back to
        # back on this renderer's workspace, so by default the backward takes the
        # forward's projection and tile lists (exactly what it would recompute);
        # reuse_binning=False recomputes them
        self.reuse = bool(reuse_binning)
        V = renderer.V
        dev = T_cw.device
        self.out = renderer.alloc_images()
        self.g_rgb = torch.empty_like(self.out["rgb"])
        self.g_depth = None if target_depth is None else torch.empty_like(self.out["depth"])
        self.dpose = torch.zeros((V, 6), dtype=torch.float64, device=dev)
        self.adam = torch.zeros((V, 13), dtype=torch.float64, device=dev)
        self.graph = None
        self.loss = torch.zeros(V, dtype=torch.float64, device=dev)  # L_t per view, last iteration

    def reset(self, T0: torch.Tensor):
        self.T.copy_(T0)
        self.adam.zero_()
        self.dpose.zero_()

    def prepare(self):
        """Sizes the workspace with a checked render (host sync); call before capture."""
        self.r.forward(*self.g, self.T, out=self.out, check=True)

    def iteration(self):
        r = self.r
        r.forward(*self.g, self.T, out=self.out, check=False)
        depth = None if self.target_depth is None else self.out["depth"]
        C.check(C.vpgs_tracking_loss(C.ptr(self.out["rgb"]), C.ptr(self.target_rgb), C.ptr(depth),
                                     C.ptr(self.target_depth), r.V, r.intr.width, r.intr.height, self.lambda_d,
                                     C.ptr(self.loss), C.ptr(self.g_rgb), C.ptr(self.g_depth),
                                     current_stream_handle()), "vpgs_tracking_loss")
        r.backward(*self.g, self.T, self.out, self.g_rgb, self.g_depth, None, grads=None,
                   dpose=self.dpose, reuse=self.reuse)
        C.check(C.vpgs_pose_step(self.T.data_ptr(), self.dpose.data_ptr(), self.adam.data_ptr(),
                                 r.V, self.lr, current_stream_handle()), "vpgs_pose_step")

    def run_eager(self, iters: int):
        for _ in range(iters):
            self.iteration()

    def capture(self, iters: int):
        """Records `iters` iterations into one CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.iteration()  # warm-up on the side stream before capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            for _ in range(iters):
                self.iteration()
        return self.graph

    def replay(self):
        self.graph.replay()
