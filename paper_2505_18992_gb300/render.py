"""Rasterizer front end: workspace management and the autograd Function.

`Renderer` owns the device workspace of a camera and passes tensors to the C
entry points; `RenderFn` puts the forward/backward pair behind
torch.autograd.  Only the final transmittance and the per-pixel list length
are kept from the forward: the backward recomputes the projection and the
per-tile sorted lists.  A renderer built with reuse_binning=True lets the
backward take them from the workspace instead, when no other render call
replaced them in between (more memory traffic saved, nothing recomputed).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import vpgs as C


def current_stream_handle(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclass
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def c(self) -> C.vpgs_camera:
        return C.vpgs_camera(self.width, self.height, self.fx, self.fy, self.cx, self.cy)


def _check_gauss(*ts):
    for t in ts:
        if t is None:
            continue
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("Gaussian tensors must be contiguous float32 CUDA tensors")


class Renderer:
    """Renders up to `n_views` views of one pinhole camera.

    `opts` are fields of vpgs_render_opts (tile_w, tile_h, alpha_min,
    alpha_max, t_min, dilation, near_z, bg, persistent_ctas).
    reuse_binning=True makes RenderFn's backward reuse the forward's tile lists.
    """

    def __init__(self, intr: Intrinsics, n_views: int = 1, device="cuda", instances_per_gaussian=24,
                 reuse_binning: bool = False, **opts):
        self.intr = intr
        self.cam = intr.c()
        self.opts = C.default_opts(**opts)
        self.V = int(n_views)
        self.device = torch.device(device)
        self.ws = None
        self.ws_bytes = 0
        self.cap_n = -1
        self.cap_m = 0
        self.inst_per_g = instances_per_gaussian
        self.last_stats = None
        self.generation = 0  # counts the calls that replace the workspace's tile lists
        self.reuse_binning = bool(reuse_binning)
        self._pending = []  # status words of unchecked renders: (event, pinned int32, what)
        self._slots = []

    # -- workspace -----------------------------------------------------------
    def reserve(self, n: int, max_instances: int | None = None):
        if max_instances is None:
            max_instances = max(self.cap_m, 1 << 16, int(self.inst_per_g * n * self.V))
        need = C.vpgs_render_workspace_bytes(int(n), self.V, ctypes.byref(self.cam),
                                             ctypes.byref(self.opts), int(max_instances))
        if need == 0:
            raise ValueError("invalid render configuration")
        if self.ws is None or need > self.ws_bytes or n > self.cap_n:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need
            self.generation += 1
        self.cap_n = max(self.cap_n, int(n))
        self.cap_m = max(self.cap_m, int(max_instances))

    def stats(self) -> C.vpgs_render_stats:
        st = C.vpgs_render_stats()
        C.check(C.vpgs_workspace_status(self.ws.data_ptr(), ctypes.byref(st),
                                        current_stream_handle()), "vpgs_workspace_status")
        self.last_stats = st
        return st

    # -- deferred status checks ------------------------------------------------
    def queue_status_check(self, what: str):
        """Queues an asynchronous copy of the workspace's status word (no host
        wait); a later `poll_status` or `check` raises if it was an error."""
        self.poll_status()
        if len(self._pending) >= 4:  # the GPU runs far behind: wait for the oldest
            self._pending[0][0].synchronize()
            self.poll_status()
        slot = self._slots.pop() if self._slots else torch.zeros(1, dtype=torch.int32, pin_memory=True)
        C.check(C.vpgs_workspace_status_copy(self.ws.data_ptr(), slot.data_ptr(), current_stream_handle()),
                "vpgs_workspace_status_copy")
        ev = torch.cuda.Event()
        ev.record()
        self._pending.append((ev, slot, what))

    def poll_status(self):
        """Raises for the first completed deferred check that found an error;
        leaves the ones still in flight alone (never waits)."""
        while self._pending and self._pending[0][0].query():
            ev, slot, what = self._pending.pop(0)
            code = int(slot[0])
            self._slots.append(slot)
            if code == 2:
                raise RuntimeError(f"{what}: tile-instance capacity exceeded (outputs undefined); "
                                   "call Renderer.reserve with a larger max_instances")
            C.check(code, what + " (device)")

    def check(self):
        """Waits for every deferred status check and raises if one found an error."""
        for ev, _, _ in self._pending:
            ev.synchronize()
        self.poll_status()

    # -- calls ---------------------------------------------------------------
    def _gauss(self, means, scales, quats, opacities, colors, n_dev=None) -> C.vpgs_gaussians:
        _check_gauss(means, scales, quats, opacities, colors)
        n = means.shape[0]
        return C.vpgs_gaussians(C.ptr(means), C.ptr(scales), C.ptr(quats), C.ptr(opacities),
                                C.ptr(colors), n, C.ptr(n_dev))

    def alloc_images(self):
        V, H, W = self.V, self.intr.height, self.intr.width
        kw = dict(device=self.device)
        return {"rgb": torch.empty((V, 3, H, W), dtype=torch.float32, **kw),
                "depth": torch.empty((V, H, W), dtype=torch.float32, **kw),
                "alpha": torch.empty((V, H, W), dtype=torch.float32, **kw),
                "t_final": torch.empty((V, H, W), dtype=torch.float32, **kw),
                "n_contrib": torch.empty((V, H, W), dtype=torch.int32, **kw),
                "n_iter": torch.empty((V, H, W), dtype=torch.int32, **kw)}

    @staticmethod
    def _images(out) -> C.vpgs_images:
        return C.vpgs_images(C.ptr(out.get("rgb")), C.ptr(out.get("depth")), C.ptr(out.get("alpha")),
                             C.ptr(out["t_final"]), C.ptr(out.get("n_contrib")), C.ptr(out["n_iter"]))

    def forward(self, means, scales, quats, opacities, colors, T_cw, n_dev=None, out=None,
                check=True):
        """Renders; returns a dict of images (rgb [V,3,H,W], depth, alpha, t_final,
        n_contrib, n_iter).  With check=True the call synchronises, reads the
        status word and grows the instance capacity if it overflowed."""
        if not (T_cw.is_cuda and T_cw.dtype == torch.float64 and T_cw.is_contiguous()):
            raise ValueError("T_cw must be a contiguous float64 CUDA tensor [V,4,4]")
        n = means.shape[0]
        if self.ws is None or n > self.cap_n:
            self.reserve(n)
        g = self._gauss(means, scales, quats, opacities, colors, n_dev)
        out = self.alloc_images() if out is None else out
        self.generation += 1
        for _ in range(4):
            code = C.vpgs_render_fwd(self.ws.data_ptr(), self.ws_bytes, ctypes.byref(g),
                                     ctypes.byref(self.cam), T_cw.data_ptr(), self.V,
                                     ctypes.byref(self.opts), ctypes.byref(self._images(out)),
                                     current_stream_handle())
            C.check(code, "vpgs_render_fwd")
            if not check:
                break
            st = self.stats()
            if st.status == 2:  # capacity: grow and redo
                self.reserve(n, int(st.n_instances * 1.25) + 1024)
                continue
            C.check(st.status, "vpgs_render_fwd (device)")
            break
        return out

    def project(self, means, scales, quats, opacities, colors, T_cw, n_dev=None):
        """Projection stage only: dict of tile_count [V,N] int32, tile_rect [V,N,4],
        mean2d [V,N,2], depth [V,N], conic [V,N,3] (culled entries hold zeros)."""
        n = means.shape[0]
        if self.ws is None or n > self.cap_n:
            self.reserve(n)
        g = self._gauss(means, scales, quats, opacities, colors, n_dev)
        self.generation += 1
        V, dev = self.V, self.device
        out = {"tile_count": torch.zeros((V, n), dtype=torch.int32, device=dev),
               "tile_rect": torch.zeros((V, n, 4), dtype=torch.int32, device=dev),
               "mean2d": torch.zeros((V, n, 2), dtype=torch.float32, device=dev),
               "depth": torch.zeros((V, n), dtype=torch.float32, device=dev),
               "conic": torch.zeros((V, n, 3), dtype=torch.float32, device=dev)}
        C.check(C.vpgs_render_project(self.ws.data_ptr(), self.ws_bytes, ctypes.byref(g),
                                      ctypes.byref(self.cam), T_cw.data_ptr(), self.V,
                                      ctypes.byref(self.opts), C.ptr(out["tile_count"]),
                                      C.ptr(out["tile_rect"]), C.ptr(out["mean2d"]),
                                      C.ptr(out["depth"]), C.ptr(out["conic"]),
                                      current_stream_handle()), "vpgs_render_project")
        return out

    def backward(self, means, scales, quats, opacities, colors, T_cw, fwd, g_rgb=None, g_depth=None,
                 g_alpha=None, grads=None, dpose=None, n_dev=None, check=False, reuse=False):
        """Accumulates gradients into `grads` (dict of float32 tensors shaped like
        the inputs; missing keys are not computed) and `dpose` [V,6] float64.

        reuse=True takes the projection and tile lists from the workspace (the
        preceding forward on this renderer had these very inputs, unchanged)."""
        g = self._gauss(means, scales, quats, opacities, colors, n_dev)
        opts = self.opts
        if reuse:
            opts = C.vpgs_render_opts.from_buffer_copy(self.opts)
            opts.flags |= C.RENDER_REUSE_BINNING
        grads = grads or {}
        gb = C.vpgs_gaussian_buffers(C.ptr(grads.get("means")), C.ptr(grads.get("scales")),
                                     C.ptr(grads.get("quats")), C.ptr(grads.get("opacities")),
                                     C.ptr(grads.get("colors")))
        code = C.vpgs_render_bwd(self.ws.data_ptr(), self.ws_bytes, ctypes.byref(g),
                                 ctypes.byref(self.cam), T_cw.data_ptr(), self.V,
                                 ctypes.byref(opts), ctypes.byref(self._images(fwd)),
                                 C.ptr(g_rgb), C.ptr(g_depth), C.ptr(g_alpha), ctypes.byref(gb),
                                 C.ptr(dpose), current_stream_handle())
        C.check(code, "vpgs_render_bwd")
        if check:
            C.check(self.stats().status, "vpgs_render_bwd (device)")


class RenderFn(torch.autograd.Function):
    """(means, scales, quats, opacities, colors, xi, T_cw, renderer) -> (rgb, depth, alpha).

    xi [V,6] float64 is a zero-valued handle for the camera-pose gradient: its
    .grad is dL/dxi for the left perturbation T_cw <- Exp(xi) T_cw at xi = 0.

    Neither pass waits for the GPU: each queues a copy of the workspace status
    word, and a device error (instance capacity, non-finite input) raises at a
    later render on the same renderer or at renderer.check().
    """

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, colors, xi, T_cw, renderer):
        # no host wait in an autograd step: the status word is checked later
        # (renderer.poll_status at the next render, renderer.check on request)
        out = renderer.forward(means, scales, quats, opacities, colors, T_cw, check=False)
        renderer.queue_status_check("render forward")
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.save_for_backward(means, scales, quats, opacities, colors, T_cw, out["t_final"],
                              out["n_iter"])
        ctx.mark_non_differentiable(out["t_final"])
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        means, scales, quats, opacities, colors, T_cw, t_final, n_iter = ctx.saved_tensors
        r = ctx.renderer
        need = ctx.needs_input_grad
        names = ("means", "scales", "quats", "opacities", "colors")
        srcs = (means, scales, quats, opacities, colors)
        grads = {k: torch.zeros_like(s) for k, s, nd in zip(names, srcs, need[:5]) if nd}
        dpose = torch.zeros((r.V, 6), dtype=torch.float64, device=means.device) if need[5] else None
        fwd = {"t_final": t_final, "n_iter": n_iter}
        cont = lambda t: None if t is None else t.contiguous()  # noqa: E731
        # recompute by default; with reuse_binning the lists are reusable unless another
        # call replaced them (saved tensors cannot change in place: autograd checks)
        reuse = r.reuse_binning and r.generation == ctx.generation
        r.backward(means, scales, quats, opacities, colors, T_cw, fwd, cont(g_rgb), cont(g_depth),
                   cont(g_alpha), grads=grads, dpose=dpose, reuse=reuse)
        r.queue_status_check("render backward")
        return (grads.get("means"), grads.get("scales"), grads.get("quats"),
                grads.get("opacities"), grads.get("colors"), dpose, None, None)


def render(means, scales, quats, opacities, colors, T_cw, renderer: Renderer, xi=None):
    """Differentiable render; returns (rgb [V,3,H,W], depth [V,H,W], alpha [V,H,W])."""
    if xi is None:
        xi = torch.zeros((renderer.V, 6), dtype=torch.float64, device=means.device)
    return RenderFn.apply(means, scales, quats, opacities, colors, xi, T_cw, renderer)
