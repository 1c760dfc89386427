"""FP64 CPU oracle of the differentiable Gaussian rasterizer.

TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
benchmark's CPU-baseline / reference arms may import this module; the product
path never does.  It shares no code with the CUDA path.

What it computes (the paper renders with 3D Gaussian Splatting, Sec. I and
Sec. II, and states neither the projection nor the compositing rules, so every
rule below is a reading of it, stated here in full):

  * covariance   Sigma = R(q) diag(s)^2 R(q)^T, q=(w,x,y,z) normalised (Sec. III-A,
                 "follow 3D-GS" for the rotation head)
  * camera       p_c = R_cw mu + t_cw; u = fx x/z + cx, v = fy y/z + cy; pixel
                 (i,j) has its centre at (i+0.5, j+0.5)
  * EWA          Sigma' = J R_cw Sigma R_cw^T J^T + eps I, J the Jacobian of the
                 pinhole projection at p_c, eps = 0.3 px^2
  * near cull    z <= near_z contributes nothing
  * extent       the pixel rectangle where alpha >= alpha_min is possible:
                 half widths sqrt(2 ln(o/alpha_min) Sigma'_xx), same for y
  * alpha        alpha = min(alpha_max, o exp(-1/2 d^T Sigma'^-1 d)), d = pixel - (u,v)
  * order        ascending camera z, ties by Gaussian index
  * compositing  front to back: skip alpha < alpha_min; stop *before* the first
                 Gaussian with T (1-alpha) < t_min; C = sum alpha_i T_i c_i + T bg,
                 D = sum alpha_i T_i z_i, A = 1 - T
  * backward     the exact derivative of the forward above with its decisions
                 (skips, stop, clamp) held fixed, taken by reverse-mode autodiff
                 of this very code; the camera-pose gradient is with respect to a
                 left perturbation T_cw <- Exp(xi) T_cw at xi = 0, ordered
                 (rho_x, rho_y, rho_z, phi_x, phi_y, phi_z).

  * tile cover   (binning, not part of the image) a Gaussian is listed in a
                 tile when its alpha_min ellipse d^T Sigma'^-1 d <= 2 ln(o/alpha_min)
                 meets one of the tile's pixel-centre columns: the segment from
                 the first to the last pixel-centre row of the tile at the
                 column's centre x, widened by the extent margins 1e-5 r + 2e-3 px
                 (1e-5 rx + 2e-3 across, 1e-5 ry + 2e-3 along).

The oracle composites every pixel against every Gaussian in depth order; the
only shortcut is a candidate filter that drops Gaussians whose (widened)
extent rectangle misses the pixel block, which provably leaves every
alpha >= alpha_min pixel in (tests check `brute=True` gives the same result).

Pins (tests/test_oracle_render.py): single-Gaussian closed forms, rotation
against scipy, the projection Jacobian against finite differences of the
projection, compositing invariants, hand-worked two-Gaussian cases, brute
force, central finite differences of every gradient, and the rigid-motion
identity of the pose gradient.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

F64 = torch.float64


@dataclass
class Options:
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    dilation: float = 0.3
    near_z: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    tile_w: int = 16
    tile_h: int = 16


@dataclass
class Margins:
    """Relative distances to a decision threshold below which a pixel is flagged.

    A flagged pixel is one where FP32 and FP64 evaluations may legitimately take
    a different branch (skip / clamp / stop / depth order)."""
    alpha: float = 2e-5
    clamp: float = 2e-5
    t_stop: float = 2e-4
    depth_tie: float = 1e-6
    # Exactly equal depths are ordered by Gaussian index on both sides (the
    # reading of the order rule).  Only Gaussians with bit-identical camera z
    # on the device as well (identical means) may leave them unflagged.
    exact_ties: bool = False


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=F64)


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z)."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ]
    return torch.stack(rows, -1).reshape(q.shape[:-1] + (3, 3))


def hat(phi: torch.Tensor) -> torch.Tensor:
    """3x3 skew matrix [phi]_x."""
    z = torch.zeros((), dtype=phi.dtype)
    return torch.stack([
        torch.stack([z, -phi[2], phi[1]]),
        torch.stack([phi[2], z, -phi[0]]),
        torch.stack([-phi[1], phi[0], z]),
    ])


def perturbed_pose(T_cw: torch.Tensor, xi: torch.Tensor) -> torch.Tensor:
    """(I + xi^) T_cw: first-order left perturbation, exact derivative at xi = 0."""
    H = torch.zeros((4, 4), dtype=F64)
    H = H + torch.cat([torch.cat([hat(xi[3:]), xi[:3, None]], 1),
                       torch.zeros((1, 4), dtype=F64)], 0)
    return (torch.eye(4, dtype=F64) + H) @ T_cw


def project(means, scales, quats, T_cw, fx, fy, cx, cy, opts: Options):
    """Per-Gaussian camera-space mean, image mean, 2D covariance and its inverse."""
    R = T_cw[:3, :3]
    t = T_cw[:3, 3]
    p = means @ R.T + t
    x, y, z = p.unbind(-1)
    u = fx * x / z + cx
    v = fy * y / z + cy
    zero = torch.zeros_like(z)
    J = torch.stack([
        torch.stack([fx / z, zero, -fx * x / (z * z)], -1),
        torch.stack([zero, fy / z, -fy * y / (z * z)], -1),
    ], -2)                                            # [N,2,3]
    Rq = quat_to_rotmat(quats)                        # [N,3,3]
    Sigma = Rq @ torch.diag_embed(scales * scales) @ Rq.transpose(-1, -2)
    Sigma_c = R @ Sigma @ R.T
    cov = J @ Sigma_c @ J.transpose(-1, -2) + opts.dilation * torch.eye(2, dtype=F64)
    A, B, C = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    det = A * C - B * B
    conic = torch.stack([C / det, -B / det, A / det], -1)  # (a, b, c) of Sigma'^-1
    return {"p_c": p, "u": u, "v": v, "z": z, "cov": torch.stack([A, B, C], -1),
            "conic": conic}


def extent(proj, opac: np.ndarray, width: int, height: int, opts: Options):
    """Pixel and tile rectangles of every Gaussian (numpy, float64 / int64).

    Returns a dict with the four exact rectangle edges (before rounding), the
    clipped pixel range, the tile range and the tile count (0 when culled).
    """
    z = proj["z"].detach().numpy()
    u = proj["u"].detach().numpy()
    v = proj["v"].detach().numpy()
    cov = proj["cov"].detach().numpy()
    o = np.asarray(opac, np.float64)
    live = (z > opts.near_z) & (o >= opts.alpha_min)
    k = np.where(live, 2.0 * np.log(np.maximum(o, opts.alpha_min) / opts.alpha_min), 0.0)
    rx = np.sqrt(k * np.where(live, cov[:, 0], 0.0))
    ry = np.sqrt(k * np.where(live, cov[:, 2], 0.0))
    ex0, ex1 = u - rx - 0.5, u + rx - 0.5
    ey0, ey1 = v - ry - 0.5, v + ry - 0.5
    with np.errstate(invalid="ignore"):
        x0 = np.maximum(np.ceil(np.where(live, ex0, 0.0)), 0)
        x1 = np.minimum(np.floor(np.where(live, ex1, -1.0)), width - 1)
        y0 = np.maximum(np.ceil(np.where(live, ey0, 0.0)), 0)
        y1 = np.minimum(np.floor(np.where(live, ey1, -1.0)), height - 1)
    nonempty = live & (x0 <= x1) & (y0 <= y1)
    x0, x1, y0, y1 = (a.astype(np.int64) for a in (x0, x1, y0, y1))
    tx0, tx1 = x0 // opts.tile_w, x1 // opts.tile_w
    ty0, ty1 = y0 // opts.tile_h, y1 // opts.tile_h
    count = np.where(nonempty, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0)
    return {"live": live, "nonempty": nonempty, "rx": rx, "ry": ry,
            "edges": np.stack([ex0, ex1, ey0, ey1], 1),
            "pix": np.stack([x0, x1, y0, y1], 1),
            "tiles": np.stack([tx0, tx1, ty0, ty1], 1), "count": count}


def rect_min_quadratic(a, b, c, x0, x1, y0, y1):
    """Minimum of q(x, y) = a x^2 + 2 b x y + c y^2 over [x0, x1] x [y0, y1].

    q is convex (a > 0, ac > b^2) with its unconstrained minimum 0 at the
    origin.  When the origin lies outside the box, the minimum is on the box
    boundary; along each edge q is a one-dimensional convex quadratic whose
    minimiser (stationary point clamped to the edge) is taken in closed form.
    """
    a, b, c, x0, x1, y0, y1 = np.broadcast_arrays(*(np.asarray(t, np.float64)
                                                     for t in (a, b, c, x0, x1, y0, y1)))
    best = np.full(a.shape, np.inf)
    for xe in (x0, x1):                       # vertical edges: y free
        ys = np.clip(-b * xe / c, y0, y1)
        best = np.minimum(best, a * xe * xe + 2.0 * b * xe * ys + c * ys * ys)
    for ye in (y0, y1):                       # horizontal edges: x free
        xs = np.clip(-b * ye / a, x0, x1)
        best = np.minimum(best, a * xs * xs + 2.0 * b * xs * ye + c * ye * ye)
    inside = (x0 <= 0.0) & (x1 >= 0.0) & (y0 <= 0.0) & (y1 >= 0.0)
    return np.where(inside, 0.0, best)


def tile_cover(proj, opac: np.ndarray, width: int, height: int, opts: Options,
               tol_px: float = 1e-3, tol_rel: float = 1e-5):
    """Tiles each Gaussian is listed in (the tile-cover rule of the header).

    Every tile of the widened pixel rectangle is tested column by column: the
    Mahalanobis distance of a (widened) column segment is s = sqrt(min q),
    q = d^T Sigma'^-1 d, and the tile counts when some column has
    s <= sqrt(k), k = 2 ln(o/alpha_min).  Returns per Gaussian the count and a
    flag set when some column lies within tol_px pixels (Mahalanobis
    tol_px / sqrt(lambda_min(Sigma'))) or tol_rel relative of the threshold,
    where an FP32 evaluation may decide otherwise.
    """
    def arr(t):
        return t.detach().numpy() if torch.is_tensor(t) else np.asarray(t, np.float64)

    u, v, z, cov, con = (arr(proj[key]) for key in ("u", "v", "z", "cov", "conic"))
    o = np.asarray(opac, np.float64)
    n = len(u)
    count = np.zeros(n, np.int64)
    flag = np.zeros(n, bool)
    live = (z > opts.near_z) & (o >= opts.alpha_min)
    idx = np.nonzero(live)[0]
    if idx.size == 0:
        return {"count": count, "flags": flag}
    k = 2.0 * np.log(o[idx] / opts.alpha_min)
    A, B, C = cov[idx, 0], cov[idx, 1], cov[idx, 2]
    rx, ry = np.sqrt(k * A), np.sqrt(k * C)
    mx, my = 1e-5 * rx + 2e-3, 1e-5 * ry + 2e-3
    x0 = np.maximum(np.ceil(u[idx] - rx - mx - 0.5), 0).astype(np.int64)
    x1 = np.minimum(np.floor(u[idx] + rx + mx - 0.5), width - 1).astype(np.int64)
    y0 = np.maximum(np.ceil(v[idx] - ry - my - 0.5), 0).astype(np.int64)
    y1 = np.minimum(np.floor(v[idx] + ry + my - 0.5), height - 1).astype(np.int64)
    ok = (x0 <= x1) & (y0 <= y1)
    tw, th = opts.tile_w, opts.tile_h
    ntx = np.where(ok, x1 // tw - x0 // tw + 1, 0)
    nty = np.where(ok, y1 // th - y0 // th + 1, 0)
    per = ntx * nty
    g = np.repeat(np.arange(idx.size), per)              # one entry per (Gaussian, tile)
    local = np.arange(per.sum()) - np.repeat(np.cumsum(per) - per, per)
    tx = x0[g] // tw + local % ntx[g]
    ty = y0[g] // th + local // ntx[g]
    ncol = np.minimum(tx * tw + tw, width) - tx * tw      # pixel columns of the tile
    t = np.repeat(np.arange(g.size), ncol)                 # one entry per (Gaussian, tile, column)
    col = tx[t] * tw + np.arange(t.size) - np.repeat(np.cumsum(ncol) - ncol, ncol)
    gt = g[t]
    # the column's pixel-centre segment (rows clipped to the image), relative to (u, v), widened
    cx0 = col + 0.5 - u[idx][gt] - mx[gt]
    cx1 = col + 0.5 - u[idx][gt] + mx[gt]
    cy0 = ty[t] * th + 0.5 - v[idx][gt] - my[gt]
    cy1 = np.minimum(ty[t] * th + th, height) - 0.5 - v[idx][gt] + my[gt]
    q = rect_min_quadratic(con[idx, 0][gt], con[idx, 1][gt], con[idx, 2][gt], cx0, cx1, cy0, cy1)
    s, sk = np.sqrt(q), np.sqrt(k)[gt]
    lam_min = 0.5 * (A + C) - np.sqrt(0.25 * (A - C) ** 2 + B * B)
    tol = tol_rel * sk + tol_px / np.sqrt(lam_min[gt])
    tile_hit = np.bincount(t, weights=s <= sk, minlength=g.size) > 0
    tile_near = np.bincount(t, weights=np.abs(s - sk) <= tol, minlength=g.size) > 0
    count[idx] = np.bincount(g, weights=tile_hit, minlength=idx.size).astype(np.int64)
    flag[idx] = np.bincount(g, weights=tile_near, minlength=idx.size) > 0
    flag |= live & (np.abs(o - opts.alpha_min) <= 1e-4 * opts.alpha_min)
    return {"count": count, "flags": flag}


def _composite_block(px, py, cand, g2, opts: Options, margins: Margins, want_flags=True):
    """Front-to-back compositing of pixels (px[P], py[P]) over candidates `cand`.

    `cand` is already in compositing order.  g2 holds the 2D quantities
    (u, v, conic, o, z, rgb) as tensors.  Returns per-pixel colour [3,P], depth,
    final transmittance, contributor count and the margin flag.
    """
    P, n = px.shape[0], cand.shape[0]
    bg = torch.tensor(opts.bg, dtype=F64)
    if n == 0:
        T = torch.ones(P, dtype=F64)
        rgb = bg[:, None].expand(3, P) * T[None]
        return rgb, torch.zeros(P, dtype=F64), T, torch.zeros(P, dtype=torch.int64), \
            torch.zeros(P, dtype=torch.bool)
    u, v = g2["u"][cand], g2["v"][cand]
    a, b, c = g2["conic"][cand].unbind(-1)
    o, z, col = g2["o"][cand], g2["z"][cand], g2["rgb"][cand]
    dx = px[:, None] - u[None, :]                      # d = pixel - mean
    dy = py[:, None] - v[None, :]
    power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    raw = o * torch.exp(power)                          # [P,n]
    alpha = torch.clamp(raw, max=opts.alpha_max)
    with torch.no_grad():
        valid = alpha >= opts.alpha_min
    a_eff = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a_eff
    T_incl = torch.cumprod(one_minus, dim=1)            # T after each candidate
    T_ext = torch.cat([torch.ones(P, 1, dtype=F64), T_incl], 1)  # T before each, plus final
    with torch.no_grad():
        stop = valid & (T_incl < opts.t_min)
        has = stop.any(1)
        s = torch.where(has, stop.to(torch.int8).argmax(1), torch.full((P,), n))
        idx = torch.arange(n)[None, :]
        keep = valid & (idx < s[:, None])
    w = a_eff * T_ext[:, :n] * keep
    T_fin = T_ext.gather(1, s[:, None])[:, 0]
    rgb = (w[:, :, None] * col[None]).sum(1).T + bg[:, None] * T_fin[None]
    depth = (w * z[None]).sum(1)
    n_contrib = keep.sum(1)
    flags = torch.zeros(P, dtype=torch.bool)
    if want_flags:
        with torch.no_grad():
            seen = idx <= s[:, None]
            r = raw.detach()
            near_min = (r - opts.alpha_min).abs() <= margins.alpha * opts.alpha_min
            near_max = (r - opts.alpha_max).abs() <= margins.clamp * opts.alpha_max
            near_t = valid & ((T_incl.detach() - opts.t_min).abs() <= margins.t_stop * opts.t_min)
            flags = ((near_min | near_max | near_t) & seen).any(1)
            # depth ties among the Gaussians that decided the pixel: candidates
            # are in ascending z, so the previous decisive z is a running max
            sel = valid & seen
            zz = z.detach()[None, :].expand(P, n)
            zsel = torch.where(sel, zz, torch.full_like(zz, -math.inf))
            prev = torch.cat([torch.full((P, 1), -math.inf, dtype=F64),
                              torch.cummax(zsel, dim=1).values[:, :-1]], 1)
            gap = (zz - prev) <= margins.depth_tie * zz.abs()
            if margins.exact_ties:
                gap &= zz != prev
            flags |= (sel & gap).any(1)
    return rgb, depth, T_fin, n_contrib, flags


def _sorted_live(proj, ext):
    z = proj["z"].detach()
    order = torch.argsort(z, stable=True)              # ties keep index order
    live = torch.as_tensor(ext["live"])
    return order[live[order]]


def render(means, scales, quats, opacities, colors, T_cw, fx, fy, cx, cy, width, height,
           opts: Options = None, margins: Margins = None, grads=None, brute=False,
           rows=None, block_w=256):
    """Render every view; optionally back-propagate upstream gradients.

    Inputs are numpy arrays (means [N,3], scales [N,3], quats [N,4],
    opacities [N], colors [N,3]) and T_cw [V,4,4].  `grads` = (dL/dC [V,3,H,W],
    dL/dD [V,H,W], dL/dA [V,H,W]) or None.  `rows` restricts the work to a list
    of image rows (used for bounded CPU timing); outputs outside it stay zero.

    Returns a dict: rgb [V,3,H,W], depth, alpha, t_final [V,H,W], n_contrib
    [V,H,W] int64, flags [V,H,W] bool, per-view extents, and with `grads` the
    gradients d_means, d_scales, d_quats, d_opacities, d_colors and d_pose [V,6].
    """
    opts = opts or Options()
    margins = margins or Margins()
    Tv = np.asarray(T_cw, np.float64).reshape(-1, 4, 4)
    V = Tv.shape[0]
    want = grads is not None
    leaves = [_t(a).clone().requires_grad_(want) for a in (means, scales, quats, opacities, colors)]
    m3, s3, q4, o1, c3 = leaves
    out = {k: np.zeros((V, 3, height, width)) if k == "rgb" else np.zeros((V, height, width))
           for k in ("rgb", "depth", "alpha", "t_final")}
    out["n_contrib"] = np.zeros((V, height, width), np.int64)
    out["flags"] = np.zeros((V, height, width), bool)
    out["extent"] = []
    out["proj"] = []
    d_pose = np.zeros((V, 6))
    row_list = list(range(height)) if rows is None else list(rows)
    for vi in range(V):
        xi = torch.zeros(6, dtype=F64, requires_grad=want)
        Tp = perturbed_pose(_t(Tv[vi]), xi)
        proj = project(m3, s3, q4, Tp, fx, fy, cx, cy, opts)
        ext = extent(proj, opacities, width, height, opts)
        out["extent"].append(ext)
        out["proj"].append({k: t.detach().numpy().copy() for k, t in proj.items()})
        # 2D leaves: compositing graphs are built per pixel block on these
        g2 = {"u": proj["u"].detach().clone().requires_grad_(want),
              "v": proj["v"].detach().clone().requires_grad_(want),
              "conic": proj["conic"].detach().clone().requires_grad_(want),
              "o": o1.detach().clone().requires_grad_(want),
              "z": proj["z"].detach().clone().requires_grad_(want),
              "rgb": c3.detach().clone().requires_grad_(want)}
        order = _sorted_live(proj, ext)
        # candidate rectangles, widened so that every pixel at which an FP32
        # evaluation could still reach alpha_min is evaluated (and flagged)
        rx, ry = ext["rx"], ext["ry"]
        un, vn = proj["u"].detach().numpy(), proj["v"].detach().numpy()
        cx0 = un - rx * (1 + 1e-4) - 0.02 - 0.5
        cx1 = un + rx * (1 + 1e-4) + 0.02 - 0.5
        cy0 = vn - ry * (1 + 1e-4) - 0.02 - 0.5
        cy1 = vn + ry * (1 + 1e-4) + 0.02 - 0.5
        order_np = order.numpy()
        for j in row_list:
            if brute:
                row_c = order_np
            else:
                row_c = order_np[(cy0[order_np] <= j) & (cy1[order_np] >= j)]
            for x0 in range(0, width, block_w):
                x1 = min(width, x0 + block_w)
                if brute:
                    cand = row_c
                else:
                    cand = row_c[(cx0[row_c] <= x1 - 1) & (cx1[row_c] >= x0)]
                cand_t = torch.as_tensor(cand, dtype=torch.int64)
                px = torch.arange(x0, x1, dtype=F64) + 0.5
                py = torch.full((x1 - x0,), j + 0.5, dtype=F64)
                rgb, depth, T_fin, nc, fl = _composite_block(px, py, cand_t, g2, opts, margins)
                out["rgb"][vi, :, j, x0:x1] = rgb.detach().numpy()
                out["depth"][vi, j, x0:x1] = depth.detach().numpy()
                out["t_final"][vi, j, x0:x1] = T_fin.detach().numpy()
                out["alpha"][vi, j, x0:x1] = 1.0 - T_fin.detach().numpy()
                out["n_contrib"][vi, j, x0:x1] = nc.numpy()
                out["flags"][vi, j, x0:x1] = fl.numpy()
                if want and cand.size > 0:
                    g_rgb = _t(grads[0][vi, :, j, x0:x1])
                    g_d = _t(grads[1][vi, j, x0:x1])
                    g_a = _t(grads[2][vi, j, x0:x1])
                    alpha_px = 1.0 - T_fin
                    L = (rgb * g_rgb).sum() + (depth * g_d).sum() + (alpha_px * g_a).sum()
                    L.backward()
        if want:
            outs, gs = [], []
            for key, t in (("u", proj["u"]), ("v", proj["v"]), ("conic", proj["conic"]),
                           ("z", proj["z"])):
                if g2[key].grad is not None:
                    outs.append(t)
                    gs.append(g2[key].grad)
            outs.append(o1)
            gs.append(g2["o"].grad if g2["o"].grad is not None else torch.zeros_like(o1))
            outs.append(c3)
            gs.append(g2["rgb"].grad if g2["rgb"].grad is not None else torch.zeros_like(c3))
            torch.autograd.backward(outs, gs)
            d_pose[vi] = xi.grad.numpy() if xi.grad is not None else 0.0
    if want:
        names = ("d_means", "d_scales", "d_quats", "d_opacities", "d_colors")
        for name, leaf in zip(names, leaves):
            out[name] = leaf.grad.numpy().copy() if leaf.grad is not None else \
                np.zeros(leaf.shape)
        out["d_pose"] = d_pose
    return out


def render_scene(scene, **kw):
    """`render` on a scenes.GaussianScene-like object (arrays + camera)."""
    cam = scene.camera
    return render(scene.means, scene.scales, scene.quats, scene.opacities, scene.colors,
                  cam.T_cw, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, **kw)
