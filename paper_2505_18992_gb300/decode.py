"""Anchor decoder front end: workspace, C calls and an autograd Function.

Decodes voxel anchors into neural Gaussians (Sec. III-A, Eq. 1-5) on the
GPU, FP32 or BF16 tensor cores, and back-propagates to the features,
offsets, scaling and MLP parameters.
"""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .render import current_stream_handle


def _cam(camera) -> C.vpgs_camera:
    return C.vpgs_camera(camera.width, camera.height, camera.fx, camera.fy, camera.cx, camera.cy)


class Decoder:
    def __init__(self, k: int = 10, bf16: bool = False, near_z: float = 0.2, guard: float = 0.15,
                 device="cuda"):
        self.k = int(k)
        self.bf16 = bool(bf16)
        self.opts = C.vpgs_decode_opts(near_z, guard)
        self.device = torch.device(device)
        self.ws = None
        self.ws_bytes = 0

    def _reserve(self, A: int):
        need = C.vpgs_decode_workspace_bytes(int(A), self.k)
        if need == 0:
            raise ValueError("invalid decoder configuration")
        if self.ws is None or need > self.ws_bytes:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need

    def _anchors(self, anchors, features, scaling, offsets) -> C.vpgs_anchors:
        for t in (anchors, scaling, offsets):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("anchors, scaling, offsets: contiguous float32 CUDA tensors")
        if features.dtype not in (torch.float32, torch.bfloat16) or not features.is_contiguous():
            raise ValueError("features: contiguous float32 or bfloat16 CUDA tensor [A,32]")
        return C.vpgs_anchors(C.ptr(anchors), C.ptr(scaling), C.ptr(offsets), C.ptr(features),
                              anchors.shape[0], self.k, 1 if features.dtype == torch.bfloat16 else 0)

    def alloc_outputs(self, n_anchors: int):
        """Output buffers for n_anchors anchors (A*k rows; only the first n_dev are written)."""
        cap = max(n_anchors * self.k, 1)
        dv = self.device
        return {"means": torch.empty((cap, 3), device=dv), "scales": torch.empty((cap, 3), device=dv),
                "quats": torch.empty((cap, 4), device=dv), "opacities": torch.empty((cap,), device=dv),
                "colors": torch.empty((cap, 3), device=dv),
                "n_dev": torch.empty((1,), dtype=torch.int32, device=dv),
                "src_index": torch.empty((cap,), dtype=torch.int32, device=dv)}

    def forward(self, anchors, features, scaling, offsets, params, camera, T_cw, out=None, sync=True):
        """Returns dict: means/scales/quats/opacities/colors (capacity A*k rows, the
        first n_dev written), n_dev (device int32 [1]), src_index, and with
        sync=True n (host int; reading it synchronises).  `out` reuses buffers
        from alloc_outputs."""
        A = anchors.shape[0]
        self._reserve(A)
        out = self.alloc_outputs(A) if out is None else out
        a = self._anchors(anchors, features, scaling, offsets)
        mlp = C.vpgs_mlp(C.ptr(params), 1 if self.bf16 else 0)
        buf = C.vpgs_gaussian_buffers(C.ptr(out["means"]), C.ptr(out["scales"]), C.ptr(out["quats"]),
                                      C.ptr(out["opacities"]), C.ptr(out["colors"]))
        C.check(C.vpgs_decode_anchors(self.ws.data_ptr(), self.ws_bytes, ctypes.byref(a), ctypes.byref(mlp),
                                      ctypes.byref(_cam(camera)), T_cw.data_ptr(), ctypes.byref(self.opts),
                                      ctypes.byref(buf), C.ptr(out["n_dev"]), C.ptr(out["src_index"]),
                                      current_stream_handle()), "vpgs_decode_anchors")
        if sync:
            out["n"] = int(out["n_dev"].item())
        return out

    def backward(self, anchors, features, scaling, offsets, params, camera, T_cw, fwd, grads, res=None):
        """grads: dict of dL/d{means,scales,quats,opacities,colors} shaped like fwd's
        outputs.  Returns dict of features, offsets, scaling and params gradients,
        accumulated (+=) into `res` when given, else into fresh zeroed tensors."""
        a = self._anchors(anchors, features, scaling, offsets)
        mlp = C.vpgs_mlp(C.ptr(params), 1 if self.bf16 else 0)
        cap = fwd["means"].shape[0]
        gl = C.vpgs_gaussians(C.ptr(grads["means"]), C.ptr(grads["scales"]), C.ptr(grads["quats"]),
                              C.ptr(grads["opacities"]), C.ptr(grads["colors"]), cap, C.ptr(fwd["n_dev"]))
        if res is None:
            res = {"features": torch.zeros(features.shape, dtype=torch.float32, device=self.device),
                   "offsets": torch.zeros_like(offsets), "scaling": torch.zeros_like(scaling),
                   "params": torch.zeros_like(params)}
        C.check(C.vpgs_decode_anchors_bwd(self.ws.data_ptr(), self.ws_bytes, ctypes.byref(a),
                                          ctypes.byref(mlp), ctypes.byref(_cam(camera)), T_cw.data_ptr(),
                                          ctypes.byref(self.opts), ctypes.byref(gl),
                                          C.ptr(fwd["src_index"]), C.ptr(res["features"]),
                                          C.ptr(res["offsets"]), C.ptr(res["scaling"]), C.ptr(res["params"]),
                                          current_stream_handle()), "vpgs_decode_anchors_bwd")
        return res
