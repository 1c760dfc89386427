"""Shared helpers of the GPU parity tests: device transfer, masks, tolerances.

Tolerances (stated once, used everywhere):
  * integer results (tile counts, contributor counts) are compared bit for bit
    away from decision margins;
  * FP32 colour, depth, alpha and final transmittance within 1e-5 absolute of
    the FP64 oracle on pixels whose decisions are not within a margin;
  * gradients: per tensor ||g - g_ref|| <= 1e-3 ||g_ref|| and per element
    |g - g_ref| <= 1e-3 |g_ref| + 1e-3 rms(g_ref); pose per component within
    1e-3 relative (plus 1e-3 of the largest component).
"""
from __future__ import annotations

import numpy as np
import torch

FWD_ATOL = 1e-5
GRAD_RTOL = 1e-3


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda").contiguous()


def scene_tensors(sc):
    g = [dev(a) for a in sc.arrays()]
    T = dev(sc.camera.T_cw, torch.float64)
    return g, T


def intrinsics(sc):
    from paper_2505_18992_gb300.render import Intrinsics
    c = sc.camera
    return Intrinsics(c.width, c.height, c.fx, c.fy, c.cx, c.cy)


def tile_count_mask(ext, opac, alpha_min=1.0 / 255.0):
    """Gaussians whose tile count may legitimately differ between FP32 and FP64:
    an exact rectangle edge close to a pixel-centre boundary (the GPU widens its
    rectangle by 1e-5 r + 2e-3 px), or an opacity at alpha_min."""
    edges = ext["edges"]
    r = np.maximum(ext["rx"], ext["ry"])[:, None]
    tol = 2.5e-3 + 2e-5 * r
    frac = np.abs(edges - np.round(edges))
    near_edge = np.any(frac <= tol, axis=1)
    near_amin = np.abs(np.asarray(opac, np.float64) - alpha_min) <= 1e-4 * alpha_min
    return (near_edge | near_amin) & ext["live"]


def assert_images_close(gpu, ref, flags, atol=FWD_ATOL, what=""):
    """gpu/ref: dicts with rgb [V,3,H,W], depth, alpha, t_final, n_contrib."""
    ok = ~flags
    report = {}
    for k in ("rgb", "depth", "alpha", "t_final"):
        g = gpu[k]
        r = ref[k]
        m = ok[:, None] if k == "rgb" else ok
        m = np.broadcast_to(m, r.shape)
        err = np.abs(g - r)[m]
        report[k] = float(err.max()) if err.size else 0.0
    nc_bad = int(((gpu["n_contrib"] != ref["n_contrib"]) & ok).sum())
    report["n_contrib_mismatch"] = nc_bad
    report["flagged_frac"] = float(flags.mean())
    for k in ("rgb", "depth", "alpha", "t_final"):
        assert report[k] <= atol, (what, k, report)
    assert nc_bad == 0, (what, report)
    return report


def grad_report(g, ref):
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    d = g - ref
    nref = np.linalg.norm(ref)
    rms = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    rel = np.linalg.norm(d) / nref if nref > 0 else np.linalg.norm(d)
    elem = np.abs(d) / (np.abs(ref) + rms + 1e-300)
    return {"rel_norm": float(rel), "max_elem": float(elem.max()) if elem.size else 0.0,
            "p99_elem": float(np.percentile(elem, 99)) if elem.size else 0.0}


def assert_grad_close(g, ref, name, rtol=GRAD_RTOL):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.abs(g - ref)
    rms = np.sqrt(np.mean(ref * ref))
    rep = grad_report(g, ref)
    assert rep["rel_norm"] <= rtol, (name, rep)
    bad = d > rtol * np.abs(ref) + rtol * rms
    assert not bad.any(), (name, rep, int(bad.sum()))
    return rep


def assert_pose_close(g, ref, rtol=GRAD_RTOL):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max(axis=-1, keepdims=True)
    bad = np.abs(g - ref) > rtol * np.abs(ref) + rtol * scale
    assert not bad.any(), (g, ref)


def masked_upstream(grads, flags):
    """Zero the upstream gradients at flagged pixels (both sides then ignore them)."""
    g_rgb, g_d, g_a = (np.array(x, copy=True) for x in grads)
    g_rgb[np.broadcast_to(flags[:, None], g_rgb.shape)] = 0.0
    g_d[flags] = 0.0
    g_a[flags] = 0.0
    return g_rgb, g_d, g_a
