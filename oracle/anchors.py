"""FP64 CPU oracle of submap expansion and anchor maintenance (Sec. III-A,
"Voxel-Based Submap Expansion and Activation").

TEST INFRASTRUCTURE.  Only the test-suite and the benchmark's CPU arms may
import this module; the product path never does.  It shares no code with the
CUDA path.

Spawning.  New anchors come from the pixels of a keyframe where the rendered
accumulated alpha is below a threshold or where the rendered depth departs
from the input depth; a budget of M_k of those pixels is back-projected with
the input depth (the posed point cloud), voxelised, and a voxel becomes an
anchor only if no Gaussian mean lies within a radius rho of it.

Statistics.  For each anchor (one voxel), the gradients of its neural
Gaussians are averaged; anchors whose average exceeds tau_g grow new anchors,
and the opacities of an anchor's neural Gaussians are accumulated so that
trivial anchors can be removed.

Readings where the paper is silent:
  * mask(p) = D_in(p) > 0 and (alpha(p) < tau_alpha or |D(p) - D_in(p)| >
    delta_d), decided in float32: only pixels with an input depth can be
    back-projected.
  * Sampling: of the C masked pixels in raster order, the pixel of rank r is
    kept iff floor((r+1) M / C) > floor(r M / C) (M evenly spaced ranks; all
    of them when C <= M); sample j is the one with floor((r+1) M / C) = j + 1.
    This deterministic spread stands in for random sampling.
  * Back-projection through the pixel centre (i + 1/2, j + 1/2) in FP64:
    x_c = (((i + 1/2) - cx) / fx * d, ((j + 1/2) - cy) / fy * d, d), the world
    point p = R^T (x_c - t) for T_cw = [R t], each coordinate summed as
    ((R_0k (x0 - t0) + R_1k (x1 - t1)) + R_2k (x2 - t2)); rounded to float32.
  * Voxelisation: the voxel of a coordinate is floor(x / v) in float32; the
    new anchor is the voxel centre (k + 1/2) v in float32; voxels are kept in
    the order of their first sample.
  * "No Gaussian mean within rho": no map point m with (dx^2 + dy^2) + dz^2 <
    rho^2 in float32, d = m - centre.
  * Statistics per anchor a: g_sum += |dL/dmu_i| over its decoded Gaussians i
    that are visible (rendered with a non-empty tile cover), g_cnt += 1 for
    each of them, o_sum += o_i over all its decoded Gaussians, visits += 1
    when it decoded any Gaussian.  The gradient is that of the 3D mean.
  * The statistics are float32 numbers (as the training keeps them) and both
    threshold tests below are decided in float32.
  * Growth: anchors with g_cnt > 0 and g_sum > tau_g g_cnt; candidates are
    the voxels (edge v_g) of those anchors' decoded Gaussian means that hold
    no existing anchor, as voxel centres, in the order of the first decoded
    Gaussian that reaches them.
  * Pruning: an anchor is removed when visits > 0 and o_sum < tau_o * visits.

Pins (tests/test_oracle_anchors.py): a hand-worked mask, the sampling rule's
count and spread, back-projection against a forward pinhole projection,
voxel centres, the radius rule against brute force, statistics against
per-anchor loops on a hand-made decode, growth and pruning on hand-made
statistics.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .icp import voxel_keys


def spawn_mask(alpha, depth, depth_in, tau_alpha, delta_d):
    """Boolean [H,W] mask of the pixels that may spawn anchors (decided in float32)."""
    a = np.asarray(alpha, np.float32)
    d = np.asarray(depth, np.float32)
    di = np.asarray(depth_in, np.float32)
    return (di > 0) & ((a < np.float32(tau_alpha)) | (np.abs(d - di) > np.float32(delta_d)))


def sample_ranks(count: int, budget: int) -> np.ndarray:
    """Ranks (ascending) of the kept masked pixels: r with floor((r+1)M/C) > floor(rM/C)."""
    if count <= budget:
        return np.arange(count, dtype=np.int64)
    r = np.arange(count, dtype=np.int64)
    return r[((r + 1) * budget) // count > (r * budget) // count]


def back_project(i, j, d, fx, fy, cx, cy, T_cw):
    """World points (float32 [n,3]) of pixels (i, j) (column, row) at depths d."""
    i = np.asarray(i, np.float64)
    j = np.asarray(j, np.float64)
    d = np.asarray(d, np.float32).astype(np.float64)
    x = np.stack([((i + 0.5) - np.float64(np.float32(cx))) / np.float64(np.float32(fx)) * d,
                  ((j + 0.5) - np.float64(np.float32(cy))) / np.float64(np.float32(fy)) * d, d], 1)
    T = np.asarray(T_cw, np.float64)
    e = x - T[:3, 3]
    p = np.stack([(T[0, k] * e[:, 0] + T[1, k] * e[:, 1]) + T[2, k] * e[:, 2] for k in range(3)], 1)
    return p.astype(np.float32)


def voxel_centres(keys, voxel) -> np.ndarray:
    """float32 centres (k + 1/2) v of integer voxel keys."""
    return ((np.asarray(keys, np.float64).astype(np.float32) + np.float32(0.5)) * np.float32(voxel)).astype(
        np.float32)


def first_voxels(points, voxel) -> tuple[np.ndarray, np.ndarray]:
    """(keys of the distinct voxels in order of first occurrence, index of that first point)."""
    if len(points) == 0:
        return np.zeros((0, 3), np.int64), np.zeros(0, np.int64)
    keys = voxel_keys(points, voxel)
    _, first = np.unique(keys, axis=0, return_index=True)
    first = np.sort(first)
    return keys[first], first


def any_within(centres, map_points, rho) -> np.ndarray:
    """True where some map point lies closer than rho (float32 decision)."""
    c32 = np.asarray(centres, np.float32)
    m32 = np.asarray(map_points, np.float32)
    out = np.zeros(len(c32), bool)
    if len(c32) == 0 or len(m32) == 0:
        return out
    rho2 = np.float32(rho) * np.float32(rho)
    tree = cKDTree(m32.astype(np.float64))
    cands = tree.query_ball_point(c32.astype(np.float64), r=float(rho) * 1.001 + 1e-6)
    for n, c in enumerate(cands):
        if c:
            d = m32[np.asarray(c)] - c32[n]
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            out[n] = bool((d2 < rho2).any())
    return out


def spawn(alpha, depth, depth_in, fx, fy, cx, cy, T_cw, tau_alpha, delta_d, budget, voxel, rho, map_points):
    """New anchor positions (float32 [n,3]) of one keyframe, and the samples they came from."""
    m = spawn_mask(alpha, depth, depth_in, tau_alpha, delta_d)
    rows, cols = np.nonzero(m)  # raster order
    keep = sample_ranks(len(rows), budget)
    rows, cols = rows[keep], cols[keep]
    pts = back_project(cols, rows, np.asarray(depth_in, np.float32)[rows, cols], fx, fy, cx, cy, T_cw)
    keys, _ = first_voxels(pts, voxel)
    centres = voxel_centres(keys, voxel)
    free = ~any_within(centres, map_points, rho)
    return centres[free], pts


def accumulate_stats(stats, src_index, k, grad_means, opacities, visible):
    """Adds one step's decode/render to stats = dict of g_sum, g_cnt, o_sum, visits (numpy, per anchor)."""
    src = np.asarray(src_index, np.int64)
    a = src // k
    g = np.linalg.norm(np.asarray(grad_means, np.float64), axis=1)
    vis = np.asarray(visible) != 0
    np.add.at(stats["g_sum"], a[vis], g[vis])
    np.add.at(stats["g_cnt"], a[vis], 1)
    np.add.at(stats["o_sum"], a, np.asarray(opacities, np.float64))
    stats["visits"][np.unique(a)] += 1
    return stats


def new_stats(n_anchors):
    return {"g_sum": np.zeros(n_anchors), "g_cnt": np.zeros(n_anchors, np.int64),
            "o_sum": np.zeros(n_anchors), "visits": np.zeros(n_anchors, np.int64)}


def prune(stats, tau_o) -> np.ndarray:
    """Indices (ascending) of the anchors kept."""
    v = np.asarray(stats["visits"])
    o = np.asarray(stats["o_sum"]).astype(np.float32)
    drop = (v > 0) & (o < np.float32(tau_o) * v.astype(np.float32))
    return np.nonzero(~drop)[0]


def grow(stats, src_index, k, means, tau_g, voxel, anchors) -> np.ndarray:
    """Voxel centres (float32 [n,3]) of the new anchors grown from high-gradient anchors."""
    cnt = np.asarray(stats["g_cnt"])
    g = np.asarray(stats["g_sum"]).astype(np.float32)
    hot = (cnt > 0) & (g > np.float32(tau_g) * cnt.astype(np.float32))
    a = np.asarray(src_index, np.int64) // k
    pts = np.asarray(means, np.float32)[hot[a]]
    keys, _ = first_voxels(pts, voxel)
    if len(keys) == 0:
        return np.zeros((0, 3), np.float32)
    occupied = {tuple(x) for x in voxel_keys(anchors, voxel)} if len(anchors) else set()
    free = np.array([tuple(x) not in occupied for x in keys], bool)
    return voxel_centres(keys[free], voxel)


__all__ = ["spawn_mask", "sample_ranks", "back_project", "voxel_centres", "first_voxels", "any_within", "spawn",
           "accumulate_stats", "new_stats", "prune", "grow"]
