"""FP64 CPU oracle of the anchor -> neural-Gaussian decoder (Sec. III-A, Eq. 1-5).

TEST INFRASTRUCTURE: see the package docstring; never used by the product.

Per anchor a with centre x^a, feature f^a (32), scaling l (3) and k offsets O:
  * cull       keep the anchor iff its camera depth exceeds near_z and its
               projected centre lies inside the image widened by `guard` of its
               size on every side (the paper only says the view is
               frustum-culled; this rule is the design reading C15)
  * Eq. 3      delta = |x^a - x^c|, d = (x^a - x^c) / delta, x^c the camera centre
  * Eq. 2      input [f^a, d, delta] (36) through three LINEAR-ReLU-LINEAR MLPs
               with hidden width 32 (Sec. IV): opacity (k), colour (3k) and
               covariance (7k; per Gaussian [scale 3, quaternion 4])
  * heads      opacity tanh, valid iff > 0 (Sec. III-A); colour sigmoid (Eq. 4);
               quaternion normalised ("follow 3D-GS"); scale sigmoid(F_s) * l (Eq. 5
               with s_v read as the anchor scaling l)
  * Eq. 1      mu^m = x^a + O^m * l (elementwise)
  * compaction valid Gaussians in (anchor, m) order; src_index = a * k + m

`bf16=True` emulates a BF16 tensor-core decode: the network input, both weight
matrices and the hidden activations are rounded to BF16 (round to nearest
even); biases stay FP32; every sum is exact FP64.  Gradients pass through the
rounding unchanged (straight-through), which is what a BF16-forward /
FP32-backward implementation computes.

Backward: reverse-mode autodiff of this code, to the features, offsets,
scaling and every MLP weight (flattened per MLP as W1, b1, W2, b2 in the order
opacity, colour, covariance).  The anchor centres and the camera are not
differentiated through the decoder.

Pins: tests/test_oracle_decode.py (exact hand-worked anchors, Eq. 3 on
Pythagorean triples, cull boundaries, BF16 rounding of hand-picked values,
finite differences of every gradient).
"""
from __future__ import annotations

import numpy as np
import torch

F64 = torch.float64
MLP_ORDER = ("opacity", "color", "cov")


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=F64)


def bf16_round(x: torch.Tensor) -> torch.Tensor:
    """Round-to-nearest-even to BF16 values, gradient passed straight through."""
    r = x.detach().to(torch.bfloat16).to(F64)
    return x + (r - x.detach())


def n_mlp_params(k: int, feat: int = 32, hidden: int = 32) -> int:
    din = feat + 4
    return sum(din * hidden + hidden + hidden * o + o for o in (k, 3 * k, 7 * k))


def _bf16_midpoint_distance(x: np.ndarray) -> np.ndarray:
    """Absolute distance of x to the nearest BF16 rounding midpoint."""
    x = np.asarray(x, np.float64)
    ax = np.abs(x)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
        ulp = np.exp2(e - 7)
        frac = ax / ulp - np.floor(ax / ulp)          # position inside the ulp
        d = np.abs(frac - 0.5) * ulp
    return np.where(ax > 0, d, np.inf)


FP32_EPS = 2.0 ** -24


def decode(anchors, features, scaling, offsets, mlp, T_cw, fx, fy, cx, cy, width, height,
           near_z=0.2, guard=0.15, bf16=False, grads=None, margin=1e-5, acc_ulps=8.0):
    """Decode anchors seen by one camera.

    Returns a dict with the compacted Gaussians (means, scales, quats,
    opacities, colors as float64 numpy arrays), src_index [N] (a*k + m), the
    kept-anchor mask [A], and a per-anchor `flags` mask marking anchors whose
    result depends on a decision taken within `margin` (relative) of its
    threshold (cull, ReLU, validity), or, with bf16, a value that an FP32
    evaluation within acc_ulps FP32 ulps of its sum of |terms| could round to
    the other BF16 neighbour.  With grads = dict of
    dL/d{means,scales,quats,opacities,colors} for the compacted Gaussians it
    also returns d_features [A,32], d_offsets [A,k,3], d_scaling [A,3] and
    d_w (flat MLP parameter gradient).
    """
    want = grads is not None
    A = anchors.shape[0]
    k = offsets.shape[1]
    T = np.asarray(T_cw, np.float64).reshape(4, 4)
    R, t = _t(T[:3, :3]), _t(T[:3, 3])
    xa = _t(anchors)
    f = _t(features).clone().requires_grad_(want)
    l = _t(scaling).clone().requires_grad_(want)
    O = _t(offsets).clone().requires_grad_(want)
    params = []
    for name in MLP_ORDER:
        params.append([_t(p).clone().requires_grad_(want) for p in mlp[name]])

    # frustum cull (decision, no gradient)
    with torch.no_grad():
        p = xa @ R.T + t
        z = p[:, 2]
        u = fx * p[:, 0] / z + cx
        v = fy * p[:, 1] / z + cy
        lo_u, hi_u = -guard * width, (1 + guard) * width
        lo_v, hi_v = -guard * height, (1 + guard) * height
        keep = (z > near_z) & (u >= lo_u) & (u <= hi_u) & (v >= lo_v) & (v <= hi_v)
        cull_near = ((z - near_z).abs() <= margin * near_z)
        for val, bound in ((u, lo_u), (u, hi_u), (v, lo_v), (v, hi_v)):
            cull_near |= (val - bound).abs() <= 10 * margin * (abs(bound) + 1.0)
    # Eq. 3: view distance and direction
    xc = -(R.T @ t)
    diff = xa - xc[None, :]
    delta = torch.linalg.norm(diff, dim=1, keepdim=True)
    d = diff / delta
    inp = torch.cat([f, d, delta], 1)                    # [A,36]
    if bf16:
        inp = bf16_round(inp)
    flags = cull_near.clone()
    outs = {}
    pre_all = []
    for name, (W1, b1, W2, b2) in zip(MLP_ORDER, params):
        W1e = bf16_round(W1) if bf16 else W1
        W2e = bf16_round(W2) if bf16 else W2
        pre = inp @ W1e.T + b1
        h = torch.relu(pre)
        if bf16:
            h = bf16_round(h)
        out = h @ W2e.T + b2
        outs[name] = out
        with torch.no_grad():
            scale = inp.abs() @ W1e.abs().T + b1.abs()
            flags |= ((pre.abs() <= margin * scale).any(1))
            oscale = h.abs() @ W2e.abs().T + b2.abs()
            if name == "opacity":
                flags |= ((out.abs() <= margin * oscale).any(1))
            pre_all.append((pre.detach().numpy(), scale.numpy()))
    if bf16:
        with torch.no_grad():
            # hidden units: FP32 accumulation error is bounded by a few ulps of the
            # sum of |terms|; flag values that close to a BF16 rounding midpoint
            for pa, sc in pre_all:
                near = (pa > 0) & (_bf16_midpoint_distance(pa) <= acc_ulps * FP32_EPS * sc)
                flags |= torch.as_tensor(near.any(1))
            # view inputs computed in FP32 (a few roundings) before the BF16 rounding
            vin = torch.cat([d, delta], 1).detach().numpy()
            dd = _bf16_midpoint_distance(vin) <= acc_ulps * FP32_EPS * np.abs(vin)
            flags |= torch.as_tensor(dd.any(1))
    # heads
    opac = torch.tanh(outs["opacity"])                    # [A,k]
    color = torch.sigmoid(outs["color"]).reshape(A, k, 3)
    cov = outs["cov"].reshape(A, k, 7)
    scales = torch.sigmoid(cov[..., :3]) * l[:, None, :]
    qraw = cov[..., 3:7]
    quats = qraw / torch.linalg.norm(qraw, dim=-1, keepdim=True)
    # Eq. 1
    means = xa[:, None, :] + O * l[:, None, :]
    with torch.no_grad():
        valid = (opac > 0) & keep[:, None]
        sel = torch.nonzero(valid.reshape(-1)).flatten()   # (anchor, m) order
    res = {
        "means": means.reshape(-1, 3)[sel], "scales": scales.reshape(-1, 3)[sel],
        "quats": quats.reshape(-1, 4)[sel], "opacities": opac.reshape(-1)[sel],
        "colors": color.reshape(-1, 3)[sel],
    }
    out = {key: val.detach().numpy().copy() for key, val in res.items()}
    out["src_index"] = sel.numpy().astype(np.int64)
    out["keep"] = keep.numpy()
    out["flags"] = flags.numpy()
    out["n"] = int(sel.numel())
    if want:
        L = sum((res[key] * _t(grads[key])).sum() for key in res)
        L.backward()
        out["d_features"] = f.grad.numpy().copy()
        out["d_offsets"] = O.grad.numpy().copy()
        out["d_scaling"] = l.grad.numpy().copy()
        flat = []
        for group in params:
            for prm in group:
                flat.append(prm.grad.numpy().reshape(-1))
        out["d_w"] = np.concatenate(flat)
    return out


def decode_scene(scene, **kw):
    cam = scene.camera
    return decode(scene.anchors, scene.features, scene.scaling, scene.offsets, scene.mlp,
                  cam.T_cw[0], cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, **kw)


def flatten_mlp(mlp) -> np.ndarray:
    """MLP parameters flattened in the order the gradients are reported."""
    return np.concatenate([np.asarray(p, np.float64).reshape(-1)
                           for name in MLP_ORDER for p in mlp[name]])


__all__ = ["decode", "decode_scene", "bf16_round", "n_mlp_params", "flatten_mlp", "MLP_ORDER"]
