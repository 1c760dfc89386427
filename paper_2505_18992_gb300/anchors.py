"""Submap expansion and anchor maintenance front end (Sec. III-A,
"Voxel-Based Submap Expansion and Activation").

Argument marshalling only: the statistics, pruning, growth and spawning run
in libvpgs.  Anchor and Gaussian positions are float32 CUDA tensors [n,3].
"""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .icp import VoxelMap
from .render import current_stream_handle


def _f32(t, what, cols=None):
    ok = t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    if cols is not None:
        ok = ok and t.dim() == 2 and t.shape[1] == cols
    if not ok:
        raise ValueError(f"{what} must be a contiguous float32 CUDA tensor" + (f" [n,{cols}]" if cols else ""))
    return t


class AnchorStats:
    """Per-anchor gradient and opacity statistics of a submap (device buffer)."""

    def __init__(self, n_anchors: int, device="cuda"):
        self.n = int(n_anchors)
        nbytes = C.vpgs_anchor_stats_bytes(self.n)
        if nbytes == 0:
            raise ValueError("invalid anchor count")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.reset()

    def reset(self):
        C.check(C.vpgs_anchor_stats_reset(self.buf.data_ptr(), self.buf.numel(), self.n, current_stream_handle()),
                "vpgs_anchor_stats_reset")

    def accumulate(self, k: int, src_index, grad_means, opacities, visible=None, n_dev=None):
        """Adds one step: the decoder's src_index [N] int32, dL/dmeans [N,3],
        opacities [N], visible [N] int32 (e.g. the tile counts) or None."""
        n = int(src_index.shape[0])
        C.check(C.vpgs_anchor_stats_accumulate(self.buf.data_ptr(), self.buf.numel(), self.n, int(k),
                                               C.ptr(src_index), C.ptr(n_dev), n, C.ptr(grad_means),
                                               C.ptr(opacities), C.ptr(visible), current_stream_handle()),
                "vpgs_anchor_stats_accumulate")

    def arrays(self) -> dict:
        """Views of the four arrays (g_sum, o_sum float32; g_cnt, visits int32)."""
        a4 = (4 * self.n + 15) // 16 * 16
        f = self.buf[:4 * a4]
        return {"g_sum": f[0:4 * self.n].view(torch.float32), "o_sum": f[a4:a4 + 4 * self.n].view(torch.float32),
                "g_cnt": f[2 * a4:2 * a4 + 4 * self.n].view(torch.int32),
                "visits": f[3 * a4:3 * a4 + 4 * self.n].view(torch.int32)}

    def status(self) -> int:
        v = ctypes.c_int32()
        C.check(C.vpgs_anchor_status(self.buf.data_ptr(), 0, self.n, ctypes.byref(v), current_stream_handle()),
                "vpgs_anchor_status")
        return v.value


class AnchorUpdate:
    """Pruning and growth of the anchors of one submap from its statistics."""

    def __init__(self, n_anchors: int, n_gaussians: int, tau_g: float, tau_o: float, grow_voxel: float,
                 device="cuda"):
        self.A, self.N = int(n_anchors), int(n_gaussians)
        nbytes = C.vpgs_anchor_update_workspace_bytes(self.A, self.N)
        if nbytes == 0:
            raise ValueError("invalid sizes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.opts = C.vpgs_anchor_update_opts(tau_g, tau_o, grow_voxel, 0)
        self.keep = torch.empty(max(self.A, 1), dtype=torch.int32, device=device)
        self.grown = torch.empty((max(self.N, 1), 3), dtype=torch.float32, device=device)
        self.counts = torch.zeros(2, dtype=torch.int32, device=device)

    def __call__(self, stats: AnchorStats, k: int, src_index, means, anchor_map: VoxelMap, n_dev=None):
        """Launches the update; returns (keep, grown, counts) device tensors (counts = [n_keep, n_grown])."""
        if anchor_map.n != self.A or ctypes.c_float(anchor_map.voxel).value != self.opts.grow_voxel:
            raise ValueError("the anchor map must hold the A anchors with voxel = grow_voxel")
        n = int(src_index.shape[0])
        if n > self.N:
            raise ValueError("more decoded Gaussians than the workspace holds")
        c = self.counts.data_ptr()
        C.check(C.vpgs_anchor_update(self.ws.data_ptr(), self.ws.numel(), stats.buf.data_ptr(), stats.buf.numel(),
                                     self.A, int(k), C.ptr(src_index), C.ptr(n_dev), n, C.ptr(means),
                                     anchor_map.buf.data_ptr(), anchor_map.buf.numel(), ctypes.byref(self.opts),
                                     self.keep.data_ptr(), c, self.grown.data_ptr(), c + 4, current_stream_handle()),
                "vpgs_anchor_update")
        return self.keep, self.grown, self.counts

    def results(self):
        """(kept anchor indices, grown anchor centres) trimmed on the host side (synchronises)."""
        nk, ng = (int(x) for x in self.counts.cpu())
        return self.keep[:nk], self.grown[:ng]

    def status(self) -> int:
        v = ctypes.c_int32()
        C.check(C.vpgs_anchor_status(self.ws.data_ptr(), 1, self.A, ctypes.byref(v), current_stream_handle()),
                "vpgs_anchor_status")
        return v.value


class Spawner:
    """New anchors of keyframes of one image size (alpha / depth spawning mask)."""

    def __init__(self, width: int, height: int, fx: float, fy: float, cx: float, cy: float, tau_alpha: float,
                 delta_depth: float, voxel: float, rho: float, max_samples: int, device="cuda"):
        self.cam = C.vpgs_camera(int(width), int(height), fx, fy, cx, cy)
        self.opts = C.vpgs_spawn_opts(tau_alpha, delta_depth, voxel, rho, int(max_samples), 0)
        nbytes = C.vpgs_spawn_workspace_bytes(int(width), int(height), int(max_samples))
        if nbytes == 0:
            raise ValueError("invalid sizes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.anchors = torch.empty((int(max_samples), 3), dtype=torch.float32, device=device)
        self.samples = torch.empty((int(max_samples), 3), dtype=torch.float32, device=device)
        self.counts = torch.zeros(2, dtype=torch.int32, device=device)

    def __call__(self, alpha, depth, depth_in, T_cw, gauss_map: VoxelMap, keep_samples: bool = False):
        """Launches the spawn; returns (anchors, samples or None, counts = [n_anchors, n_samples])."""
        for t, what in ((alpha, "alpha"), (depth, "depth"), (depth_in, "input depth")):
            _f32(t, what)
            if t.numel() != self.cam.width * self.cam.height:
                raise ValueError(f"{what} must hold H*W values")
        if not (T_cw.is_cuda and T_cw.dtype == torch.float64 and T_cw.numel() == 16 and T_cw.is_contiguous()):
            raise ValueError("T_cw must be a contiguous float64 CUDA tensor [4,4]")
        c = self.counts.data_ptr()
        C.check(C.vpgs_spawn_anchors(self.ws.data_ptr(), self.ws.numel(), alpha.data_ptr(), depth.data_ptr(),
                                     depth_in.data_ptr(), ctypes.byref(self.cam), T_cw.data_ptr(),
                                     gauss_map.buf.data_ptr(), gauss_map.buf.numel(), gauss_map.n, gauss_map.voxel,
                                     ctypes.byref(self.opts), self.anchors.data_ptr(), c,
                                     self.samples.data_ptr() if keep_samples else None, c + 4 if keep_samples else None,
                                     current_stream_handle()), "vpgs_spawn_anchors")
        return self.anchors, (self.samples if keep_samples else None), self.counts

    def results(self):
        na, ns = (int(x) for x in self.counts.cpu())
        return self.anchors[:na], self.samples[:ns]

    def status(self) -> int:
        v = ctypes.c_int32()
        C.check(C.vpgs_anchor_status(self.ws.data_ptr(), 2, 0, ctypes.byref(v), current_stream_handle()),
                "vpgs_anchor_status")
        return v.value
