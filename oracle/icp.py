"""FP64 CPU oracle of the voxel-based 3D Gaussian ICP of fine tracking
(Sec. III-B, Eq. 10-12).

TEST INFRASTRUCTURE.  Only the test-suite and the benchmark's CPU arms may
import this module; the product path never does.  It shares no code with the
CUDA path.

  S = { s = T p : p in P }                                  (Eq. 10, T the initial guess)
  dT = argmin sum_{(s, m) in C(tau)} rho(||T s - m||)       (Eq. 11)
  rho(e) = (e^2 / 2) / (sigma / 3 + e^2)                    (Eq. 12, Geman-McClure)

Readings where the paper is silent:
  * The voxel of a point is floor(p / v) per axis, decided in float32 (the
    points are float32; the division is the correctly rounded one).
  * Double downsampling: the scan is reduced to the lowest-index point of each
    voxel of edge v1, and the survivors to the lowest-index survivor of each
    voxel of edge v2; the kept points are original points, not voxel centres.
  * Correspondences: the nearest map point of each transformed source point
    (ties to the lower map index), kept when its distance is below tau.  The
    map points are the Gaussian means.  icp() searches exactly in FP64;
    nearest_f32() takes the same decision in float32 (the GPU's precision).
  * Minimisation by iteratively reweighted Gauss-Newton: weights
    w = rho'(e) / e = k / (k + e^2)^2 with k = sigma / 3; each step solves
    (sum w J^T J) xi = -(sum w J^T r), r = T s - m, J = [I, -[T s - c]x], and
    updates T <- Tr(c) Exp(xi) Tr(-c) T (left perturbation about a centre c,
    xi = (rho, phi)).  Every c gives the same iterates in exact arithmetic
    (Exp(Ad_X xi) = X Exp(xi) X^-1); icp() uses c = 0.  The loop stops when
    |xi| < eps (after applying that step), when fewer than 6 correspondences
    remain, when the system is not positive definite, or after a fixed number
    of iterations.  sigma and tau are arguments: the paper adapts sigma online
    and gives no rule.

Pins (tests/test_oracle_icp.py): brute-force downsampling, the weight against
a central difference of rho, the normal equations against central
differences of the weighted least-squares cost (at c = 0 and c != 0), the
float32 search against a brute-force scan, and exact recovery of a known rigid
motion from a perturbed start (also with outliers in the scan).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .pose import se3_exp

# stop codes of icp()
RAN_OUT, CONVERGED, TOO_FEW, DEGENERATE = 0, 1, 2, 3


def voxel_keys(points, voxel) -> np.ndarray:
    """Integer voxel of each point: floor(p / v) evaluated in float32."""
    q = np.asarray(points, np.float32) / np.float32(voxel)
    return np.floor(q).astype(np.int64)


def voxel_downsample(points, voxel) -> np.ndarray:
    """Indices (ascending) of the lowest-index point of every occupied voxel."""
    if len(points) == 0:
        return np.zeros(0, np.int64)
    _, first = np.unique(voxel_keys(points, voxel), axis=0, return_index=True)
    return np.sort(first)


def double_downsample(points, v1, v2) -> np.ndarray:
    """Original indices (ascending) kept by downsampling at v1 and then at v2."""
    i1 = voxel_downsample(points, v1)
    i2 = voxel_downsample(np.asarray(points)[i1], v2)
    return i1[i2]


def transform(T, p) -> np.ndarray:
    """T p in FP64, each coordinate as ((T_r0 x + T_r1 y) + T_r2 z) + T_r3."""
    p = np.asarray(p, np.float64)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return np.stack([((T[r, 0] * x + T[r, 1] * y) + T[r, 2] * z) + T[r, 3] for r in range(3)], axis=1)


def gm_rho(e, sigma):
    return 0.5 * e * e / (sigma / 3.0 + e * e)


def gm_weight(e, sigma):
    k = sigma / 3.0
    return k / (k + e * e) ** 2


def skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def nearest(s, tree, tau):
    """Exact FP64 nearest map index per point (-1: none closer than tau)."""
    if len(s) == 0:
        return np.zeros(0, np.int64)
    d, j = tree.query(s, k=1, distance_upper_bound=tau)
    return np.where(np.isfinite(d) & (d < tau), j, -1)


def nearest_f32(s, map_points, tau, tree=None):
    """The same search decided in float32: s rounded to float32, squared
    distance (dx^2 + dy^2) + dz^2 in float32, kept when below float32(tau)^2,
    ties to the lower map index."""
    m32 = np.asarray(map_points, np.float32)
    s32 = np.asarray(s, np.float64).astype(np.float32)
    tree = tree or cKDTree(np.asarray(map_points, np.float64))
    tau2 = np.float32(tau) * np.float32(tau)
    out = np.full(len(s32), -1, np.int64)
    cands = tree.query_ball_point(np.asarray(s, np.float64), r=float(tau) * 1.001 + 1e-6)
    for i, c in enumerate(cands):
        if not c:
            continue
        c = np.sort(np.asarray(c, np.int64))
        d = m32[c] - s32[i]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        ok = d2 < tau2
        if ok.any():
            c, d2 = c[ok], d2[ok]
            out[i] = c[np.argmin(d2)]  # argmin keeps the first (lowest index) of equal minima
    return out


def normal_equations(s, m, sigma, c=None, magnitude=False):
    """Weighted Gauss-Newton system about centre c for residuals r = s - m
    (s already transformed).  Returns H [6,6], b [6], sum rho; with
    magnitude=True also the sums of the absolute per-pair terms (|H|, |b|),
    the scale against which a rounding error in the sums is measured."""
    c = np.zeros(3) if c is None else np.asarray(c, np.float64)
    H = np.zeros((6, 6))
    b = np.zeros(6)
    Ha = np.zeros((6, 6))
    ba = np.zeros(6)
    cost = 0.0
    for si, mi in zip(np.asarray(s, np.float64), np.asarray(m, np.float64)):
        r = si - mi
        e = np.linalg.norm(r)
        w = gm_weight(e, sigma)
        J = np.hstack([np.eye(3), -skew(si - c)])
        H += w * J.T @ J
        b += w * J.T @ r
        Ha += np.abs(w * J.T @ J)
        ba += np.abs(w * J.T @ r)
        cost += gm_rho(e, sigma)
    return (H, b, cost, Ha, ba) if magnitude else (H, b, cost)


def solve_step(H, b):
    """xi = -H^-1 b by Cholesky; None when H is not positive definite."""
    try:
        L = np.linalg.cholesky(H)
    except np.linalg.LinAlgError:
        return None
    return -np.linalg.solve(L.T, np.linalg.solve(L, b))


def icp(scan, map_points, T0, v1, v2, tau, sigma, iterations=20, eps=1e-6):
    """Registers the scan (local frame) against the map from the initial guess
    T0.  Returns dict: T, iterations run, stop code, correspondences and cost
    of the last linearisation, |xi| of the last step, the kept source indices
    and the correspondence count of every iteration."""
    src_idx = double_downsample(scan, v1, v2)
    src = np.asarray(scan, np.float32)[src_idx]
    mp = np.asarray(map_points, np.float32).astype(np.float64)
    tree = cKDTree(mp) if len(mp) else None
    T = np.asarray(T0, np.float64).copy()
    out = {"iterations": 0, "stop": RAN_OUT, "correspondences": 0, "cost": 0.0, "xi_norm": 0.0,
           "src_idx": src_idx, "counts": []}
    for it in range(iterations):
        s = transform(T, src)
        j = nearest(s, tree, tau) if tree is not None else np.full(len(s), -1)
        ok = j >= 0
        out["iterations"] = it + 1
        out["correspondences"] = int(ok.sum())
        out["counts"].append(out["correspondences"])
        H, b, out["cost"] = normal_equations(s[ok], mp[j[ok]], sigma)
        if out["correspondences"] < 6:
            out["stop"] = TOO_FEW
            break
        xi = solve_step(H, b)
        if xi is None:
            out["stop"] = DEGENERATE
            break
        T = se3_exp(xi) @ T
        out["xi_norm"] = float(np.linalg.norm(xi))
        if out["xi_norm"] < eps:
            out["stop"] = CONVERGED
            break
    out["T"] = T
    return out


__all__ = ["voxel_keys", "voxel_downsample", "double_downsample", "transform", "gm_rho", "gm_weight",
           "nearest", "nearest_f32", "normal_equations", "solve_step", "icp",
           "RAN_OUT", "CONVERGED", "TOO_FEW", "DEGENERATE"]
