"""Seeded synthetic inputs for the rasterizer and the anchor decoder.

This module only *draws inputs*: Gaussian clouds on planes, walls, boxes and
street surfaces, anchor grids, MLP weights and camera poses.  It holds none of
the method's arithmetic (no projection, compositing or decoding) and is the one
module that both the CUDA path and the CPU oracle are fed from.  numpy only.

The workloads stand in for the paper's datasets (Replica/ScanNet rooms, KITTI
streets; Sec. IV "Datasets"), which are not available: shapes, sizes and value
distributions follow the scenes the paper evaluates on, values are random.

Conventions shared by every generator
  * Gaussians are structure-of-arrays, float32, C-contiguous:
      means [N,3], scales [N,3] (linear, metres), quats [N,4] (w,x,y,z, not
      normalised), opacities [N], colors [N,3].
  * A camera is a world->camera rigid transform T_cw (float64 [4,4]) plus
    pinhole intrinsics (fx, fy, cx, cy) and an image size (W, H).  The camera
    looks down +z, +x right, +y down.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Gaussians decoded per anchor (Sec. IV "Implementation Details": k = 10).
K_PER_ANCHOR = 10
FEAT_DIM = 32
HIDDEN = 32


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_cw: np.ndarray  # [V,4,4] float64

    @property
    def n_views(self) -> int:
        return int(self.T_cw.shape[0])

    @property
    def pixels(self) -> int:
        return self.n_views * self.width * self.height


@dataclass
class GaussianScene:
    name: str
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacities: np.ndarray
    colors: np.ndarray
    camera: Camera
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return (self.means, self.scales, self.quats, self.opacities, self.colors)


@dataclass
class AnchorScene:
    name: str
    anchors: np.ndarray   # [A,3] float32, voxel centres x^a
    features: np.ndarray  # [A,32] float32, f^a
    scaling: np.ndarray   # [A,3] float32, l
    offsets: np.ndarray   # [A,K,3] float32, O
    mlp: dict             # name -> (W1 [32,36], b1 [32], W2 [out,32], b2 [out]) float32
    camera: Camera
    k: int = K_PER_ANCHOR

    @property
    def n(self) -> int:
        return int(self.anchors.shape[0])


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at(eye, target, up) -> np.ndarray:
    """World->camera transform for a camera at `eye` looking at `target`.

    Camera axes: z forward, x right, y down (image rows grow downwards).
    """
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = -R @ eye
    return T


def perturb_pose(T_cw: np.ndarray, rng, trans_m: float, rot_deg: float) -> np.ndarray:
    """Left-multiply T_cw by a random rigid motion of the given magnitudes."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(rot_deg)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(ang) * Kx + (1 - math.cos(ang)) * (Kx @ Kx)
    d = rng.normal(size=3)
    d *= trans_m / np.linalg.norm(d)
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = d
    return P @ T_cw


# --------------------------------------------------------------------------
# attribute distributions shared by the explicit-Gaussian workloads
# --------------------------------------------------------------------------

def _attributes(rng, n: int):
    lo, hi = math.log(0.005), math.log(0.05)
    scales = np.exp(rng.uniform(lo, hi, size=(n, 3)))
    quats = rng.normal(size=(n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    opac = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    colors = rng.uniform(0.0, 1.0, size=(n, 3))
    return (scales.astype(np.float32), quats.astype(np.float32),
            opac.astype(np.float32), colors.astype(np.float32))


def _basis(normal):
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(n, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return n, e1, e2


def _rect_points(rng, origin, e1, e2, len1, len2, n):
    """n uniform points on the rectangle origin + [0,len1] e1 + [0,len2] e2."""
    a = rng.uniform(0, len1, size=(n, 1))
    b = rng.uniform(0, len2, size=(n, 1))
    return np.asarray(origin)[None, :] + a * e1[None, :] + b * e2[None, :]


def _split_by_area(n, areas):
    areas = np.asarray(areas, np.float64)
    counts = np.floor(n * areas / areas.sum()).astype(np.int64)
    counts[: n - counts.sum()] += 1
    return counts


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def tiny_planes(n: int = 10_000, width: int = 320, height: int = 240, f: float = 300.0,
                seed: int = 0) -> GaussianScene:
    """Small scene: n Gaussians on 3 random planes inside the 4 m cube [-2,2]^3.

    Camera 3 m in front of the cube centre looking +z.  At the default sizes this
    is the small parity workload (10,000 Gaussians, 320x240, fx=fy=300).
    """
    rng = np.random.default_rng(seed)
    counts = [n - 2 * (n // 3), n // 3, n // 3]
    pts = []
    for c in counts:
        p0 = rng.uniform(-1, 1, size=3)
        normal = rng.normal(size=3)
        nrm, e1, e2 = _basis(normal)
        got = []
        have = 0
        while have < c:
            a = rng.uniform(-3.5, 3.5, size=(4 * c + 16, 1))
            b = rng.uniform(-3.5, 3.5, size=(4 * c + 16, 1))
            q = p0[None] + a * e1[None] + b * e2[None]
            q = q[np.all(np.abs(q) <= 2.0, axis=1)]
            got.append(q)
            have += len(q)
        q = np.concatenate(got)[:c]
        q = q + rng.normal(0, 0.02, size=(c, 1)) * nrm[None]
        pts.append(q)
    means = np.concatenate(pts).astype(np.float32)
    scales, quats, opac, colors = _attributes(rng, n)
    T = look_at([0, 0, -3], [0, 0, 0], [0, -1, 0])
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, T[None])
    trng = np.random.default_rng(100 + seed)
    extra = {
        "target_rgb": trng.uniform(0, 1, size=(1, 3, height, width)).astype(np.float32),
        "target_depth": trng.uniform(1, 5, size=(1, height, width)).astype(np.float32),
    }
    return GaussianScene("tiny_planes", means, scales, quats, opac, colors, cam, extra)


def _room_points(rng, n, size=(6.0, 5.0, 3.0), n_boxes=20):
    X, Y, Z = size
    faces = []  # (origin, e1, e2, len1, len2, normal)
    ex, ey, ez = np.eye(3)
    faces += [((0, 0, 0), ex, ey, X, Y, ez), ((0, 0, Z), ex, ey, X, Y, -ez),
              ((0, 0, 0), ex, ez, X, Z, ey), ((0, Y, 0), ex, ez, X, Z, -ey),
              ((0, 0, 0), ey, ez, Y, Z, ex), ((X, 0, 0), ey, ez, Y, Z, -ex)]
    for _ in range(n_boxes):
        e = rng.uniform(0.3, 1.0, size=3)
        c = np.array([rng.uniform(0.5, X - 0.5), rng.uniform(0.5, Y - 0.5), 0.0])
        yaw = rng.uniform(0, 2 * math.pi)
        u = np.array([math.cos(yaw), math.sin(yaw), 0.0])
        v = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
        o = c - 0.5 * e[0] * u - 0.5 * e[1] * v
        faces += [(o + e[2] * ez, u, v, e[0], e[1], ez),
                  (o, u, ez, e[0], e[2], -v), (o + e[1] * v, u, ez, e[0], e[2], v),
                  (o, v, ez, e[1], e[2], -u), (o + e[0] * u, v, ez, e[1], e[2], u)]
    areas = [f[3] * f[4] for f in faces]
    counts = _split_by_area(n, areas)
    pts = []
    for (o, a, b, la, lb, nrm), c in zip(faces, counts):
        if c == 0:
            continue
        q = _rect_points(rng, np.asarray(o, np.float64), np.asarray(a), np.asarray(b), la, lb, int(c))
        q = q + rng.normal(0, 0.02, size=(int(c), 1)) * np.asarray(nrm)[None]
        pts.append(q)
    return np.concatenate(pts)


def indoor_room(n: int = 1_000_000, width: int = 1200, height: int = 680, f: float = 600.0,
                seed: int = 1) -> GaussianScene:
    """Room-like scene: n Gaussians on the 6 walls of a 6x5x3 m room plus 20 boxes.

    Camera at the room centre looking +x (1200x680, fx=fy=600 by default); the
    extra entry `T_track0` is the same pose perturbed by 2 cm / 1 degree, the
    start point of the pose-only tracking iterations.
    """
    rng = np.random.default_rng(seed)
    means = _room_points(rng, n).astype(np.float32)
    perm = rng.permutation(n)
    means = means[perm]
    scales, quats, opac, colors = _attributes(rng, n)
    T = look_at([3.0, 2.5, 1.5], [4.0, 2.5, 1.5], [0, 0, 1])
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, T[None])
    trng = np.random.default_rng(101)
    extra = {"T_track0": perturb_pose(T, trng, 0.02, 1.0)[None]}
    return GaussianScene("indoor_room", means, scales, quats, opac, colors, cam, extra)


def _kaiming_linear(rng, fan_in, fan_out):
    bound = 1.0 / math.sqrt(fan_in)
    W = rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(np.float32)
    b = rng.uniform(-bound, bound, size=(fan_out,)).astype(np.float32)
    return W, b


def decoder_mlps(rng, k: int = K_PER_ANCHOR) -> dict:
    """Three LINEAR->ReLU->LINEAR decoders (hidden 32) with torch-default init.

    Input width 36 = feature(32) + view direction(3) + view distance(1).
    Outputs: opacity k, colour 3k, covariance 7k (scale 3 + quaternion 4 per
    Gaussian).
    """
    din = FEAT_DIM + 4
    out = {}
    for name, dout in (("opacity", k), ("color", 3 * k), ("cov", 7 * k)):
        W1, b1 = _kaiming_linear(rng, din, HIDDEN)
        W2, b2 = _kaiming_linear(rng, HIDDEN, dout)
        out[name] = (W1, b1, W2, b2)
    return out


def street_anchors(n_anchors: int = 100_000, width: int = 1241, height: int = 376,
                   f: float = 718.0, length: float = 200.0, seed: int = 2,
                   voxel: float = 0.2, k: int = K_PER_ANCHOR,
                   cam_x: float = 2.0, x0: float = 0.0, mlp_seed=None) -> AnchorScene:
    """Voxel anchors over a street corridor [x0,x0+length]x[-10,10]x[0,8] m.

    Anchors sit at centres of 0.2 m voxels on the ground and on the two facades,
    sampled without replacement; 32-dim N(0,1) features, per-anchor scaling
    0.2*exp(U(-0.2,0.2)), offsets U(-1,1).  KITTI-like camera (1241x376,
    fx=fy=718) at 1.7 m height looking down the street.
    """
    rng = np.random.default_rng(seed)
    nx = int(round(length / voxel))
    ny = int(round(20.0 / voxel))
    nz = int(round(8.0 / voxel))
    n_ground, n_facade = nx * ny, nx * nz
    total = n_ground + 2 * n_facade
    n_anchors = min(n_anchors, total)
    pick = np.sort(rng.choice(total, size=n_anchors, replace=False))
    pts = np.empty((n_anchors, 3), np.float64)
    g = pick < n_ground
    ig = pick[g]
    pts[g] = np.stack([x0 + (ig // ny + 0.5) * voxel, -10.0 + (ig % ny + 0.5) * voxel,
                       np.full(ig.shape, 0.5 * voxel)], 1)
    fa = pick[~g] - n_ground
    side = fa // n_facade
    r = fa % n_facade
    ysgn = np.where(side == 0, -1.0, 1.0)
    pts[~g] = np.stack([x0 + (r // nz + 0.5) * voxel, ysgn * (10.0 - 0.5 * voxel),
                        (r % nz + 0.5) * voxel], 1)
    perm = rng.permutation(n_anchors)
    anchors = pts[perm].astype(np.float32)
    features = rng.normal(size=(n_anchors, FEAT_DIM)).astype(np.float32)
    scaling = (0.2 * np.exp(rng.uniform(-0.2, 0.2, size=(n_anchors, 3)))).astype(np.float32)
    offsets = rng.uniform(-1, 1, size=(n_anchors, k, 3)).astype(np.float32)
    mlp = decoder_mlps(rng if mlp_seed is None else np.random.default_rng(mlp_seed), k)
    T = look_at([cam_x, 0.0, 1.7], [cam_x + 1.0, 0.0, 1.7], [0, 0, 1])
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, T[None])
    return AnchorScene("street_anchors", anchors, features, scaling, offsets, mlp, cam, k)


def corridor_points(rng, n, x0=6.0, length=40.0):
    """n points on the ground and facades of a street section (explicit Gaussians)."""
    areas = [length * 20.0, length * 8.0, length * 8.0]
    counts = _split_by_area(n, areas)
    ex, ey, ez = np.eye(3)
    faces = [((x0, -10.0, 0.0), ex, ey, length, 20.0, ez),
             ((x0, -10.0, 0.0), ex, ez, length, 8.0, ey),
             ((x0, 10.0, 0.0), ex, ez, length, 8.0, -ey)]
    pts = []
    for (o, a, b, la, lb, nrm), c in zip(faces, counts):
        q = _rect_points(rng, np.asarray(o), a, b, la, lb, int(c))
        q = q + rng.normal(0, 0.02, size=(int(c), 1)) * nrm[None]
        pts.append(q)
    return np.concatenate(pts)


def batched_keyframes(n: int = 2_000_000, n_views: int = 8, width: int = 640, height: int = 480,
                      f: float = 525.0, radius: float = 2.0, seed: int = 3) -> GaussianScene:
    """Submap of n Gaussians (half room, half street section) seen by n_views keyframes.

    Keyframes sit on a horizontal arc around the room centre (angles evenly
    spaced in [-60, 60] degrees) and look at the arc centre.
    """
    rng = np.random.default_rng(seed)
    n_room = n // 2
    room = _room_points(rng, n_room)
    street = corridor_points(rng, n - n_room)
    means = np.concatenate([room, street]).astype(np.float32)
    means = means[rng.permutation(n)]
    scales, quats, opac, colors = _attributes(rng, n)
    c = np.array([3.0, 2.5, 1.5])
    Ts = []
    for ang in np.linspace(-60.0, 60.0, n_views):
        a = math.radians(ang)
        eye = c + radius * np.array([math.cos(a), math.sin(a), 0.0])
        Ts.append(look_at(eye, c, [0, 0, 1]))
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, np.stack(Ts))
    return GaussianScene("batched_keyframes", means, scales, quats, opac, colors, cam)


def random_gaussians(n: int, width: int, height: int, f: float, seed: int,
                     depth=(1.5, 4.0), spread: float = 1.0, scale_range=(0.005, 0.05),
                     n_views: int = 1) -> GaussianScene:
    """A handful of Gaussians in front of a camera at the origin (tiny test scenes)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(depth[0], depth[1], size=n)
    xy = rng.uniform(-spread, spread, size=(n, 2)) * z[:, None] * np.array(
        [width / (2 * f), height / (2 * f)])
    means = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    lo, hi = math.log(scale_range[0]), math.log(scale_range[1])
    scales = np.exp(rng.uniform(lo, hi, size=(n, 3))).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    opac = rng.uniform(0.05, 0.95, size=n).astype(np.float32)
    colors = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
    Ts = [np.eye(4)]
    for v in range(1, n_views):
        Ts.append(perturb_pose(np.eye(4), rng, 0.1, 5.0))
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, np.stack(Ts))
    return GaussianScene("random_gaussians", means, scales, quats, opac, colors, cam)


def upstream_grads(rng_seed: int, n_views: int, height: int, width: int):
    """Seeded upstream gradients dL/dC [V,3,H,W], dL/dD [V,H,W], dL/dA [V,H,W]."""
    rng = np.random.default_rng(rng_seed)
    g_rgb = rng.normal(size=(n_views, 3, height, width)).astype(np.float32)
    g_d = rng.normal(size=(n_views, height, width)).astype(np.float32)
    g_a = rng.normal(size=(n_views, height, width)).astype(np.float32)
    return g_rgb, g_d, g_a


@dataclass
class LidarScene:
    """A street map (Gaussian means, world frame) and one LiDAR scan of it."""
    name: str
    map_points: np.ndarray  # [M,3] float32, world
    scan: np.ndarray        # [P,3] float32, sensor frame
    T_true: np.ndarray      # [4,4] float64, sensor -> world
    T_init: np.ndarray      # [4,4] float64, the perturbed initial guess T_{i-1} T_pred


def _street_boxes(rng, x0, length):
    """Axis-aligned boxes (lo, hi) of a street: building blocks with set-backs
    and gaps behind y = +-10 m, poles at +-8.5 m and parked cars at +-6.3 m."""
    lo, hi = [], []
    for side in (-1.0, 1.0):
        x = x0 - 10.0
        while x < x0 + length + 10.0:
            run = rng.uniform(12.0, 30.0)
            gap = rng.uniform(1.0, 4.0) if rng.random() < 0.5 else 0.0
            near = 10.0 + rng.uniform(0.0, 2.5)
            h = rng.uniform(6.0, 15.0)
            y0, y1 = (near, near + 8.0) if side > 0 else (-near - 8.0, -near)
            lo.append((x, y0, 0.0))
            hi.append((x + run, y1, h))
            x += run + gap
        for px in np.arange(x0 + rng.uniform(0.0, 10.0), x0 + length, rng.uniform(15.0, 25.0)):
            lo.append((px - 0.15, side * 8.5 - 0.15, 0.0))
            hi.append((px + 0.15, side * 8.5 + 0.15, 6.0))
        for cx in np.sort(rng.uniform(x0, x0 + length, size=int(length // 12))):
            lo.append((cx - 2.25, side * 6.3 - 0.9, 0.0))
            hi.append((cx + 2.25, side * 6.3 + 0.9, 1.5))
    return np.asarray(lo, np.float64), np.asarray(hi, np.float64)


def _box_surface_points(rng, lo, hi, n):
    """n points uniform over the 4 sides and the top of each box (area-weighted)."""
    d = hi - lo
    faces = []  # (origin, e1, e2, normal) with e1, e2 spanning the face
    for b in range(len(lo)):
        x, y, z = lo[b]
        dx, dy, dz = d[b]
        faces += [((x, y, z), (dx, 0, 0), (0, 0, dz), (0, -1, 0)), ((x, y + dy, z), (dx, 0, 0), (0, 0, dz), (0, 1, 0)),
                  ((x, y, z), (0, dy, 0), (0, 0, dz), (-1, 0, 0)), ((x + dx, y, z), (0, dy, 0), (0, 0, dz), (1, 0, 0)),
                  ((x, y, z + dz), (dx, 0, 0), (0, dy, 0), (0, 0, 1))]
    o = np.asarray([f[0] for f in faces], np.float64)
    e1 = np.asarray([f[1] for f in faces], np.float64)
    e2 = np.asarray([f[2] for f in faces], np.float64)
    nrm = np.asarray([f[3] for f in faces], np.float64)
    area = np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1)
    which = rng.choice(len(faces), size=n, p=area / area.sum())
    u, v = rng.uniform(size=(2, n, 1))
    return o[which] + u * e1[which] + v * e2[which] + rng.normal(0, 0.02, size=(n, 1)) * nrm[which]


def _ray_cast(orig, dirs, lo, hi, max_range):
    """Nearest hit distance of rays from orig along unit dirs with the ground
    z = 0 and the boxes (slab test); inf where nothing is hit within range."""
    d = np.where(np.abs(dirs) < 1e-12, 1e-12, dirs)
    inv = 1.0 / d
    t = np.full(len(dirs), np.inf)
    down = dirs[:, 2] < 0
    t[down] = -orig[2] / dirs[down, 2]
    for b in range(len(lo)):
        t1 = (lo[b] - orig) * inv
        t2 = (hi[b] - orig) * inv
        tn = np.minimum(t1, t2).max(axis=1)
        tf = np.maximum(t1, t2).min(axis=1)
        hit = (tf >= tn) & (tn > 0)
        t = np.where(hit & (tn < t), tn, t)
    t[t > max_range] = np.inf
    return t


def street_lidar(n_map: int = 1_000_000, beams: int = 64, azimuths: int = 1800, length: float = 200.0,
                 x0: float = 0.0, max_range: float = 80.0, seed: int = 7) -> LidarScene:
    """A 64-beam LiDAR sweep (1800 azimuths, elevations -24.8..2 deg, 1 cm
    range noise, 80 m range) from 1.73 m above the middle of a street
    corridor [x0, x0+length] x [-20, 20] m, and a map of n_map Gaussian means
    (2 cm normal jitter) on the same ground, buildings, poles and cars.  The
    initial guess is off by N(0, 0.15 m) per axis and a 1 degree rotation
    (KITTI-like driving stands in for the paper's outdoor sequences)."""
    rng = np.random.default_rng(seed)
    lo, hi = _street_boxes(rng, x0, length)
    ground_area = (length + 20.0) * 40.0
    ext = hi - lo
    box_area = float(np.sum(2 * ext[:, 2] * (ext[:, 0] + ext[:, 1]) + ext[:, 0] * ext[:, 1]))
    n_ground = int(round(n_map * ground_area / (ground_area + box_area)))
    ground = np.c_[rng.uniform(x0 - 10.0, x0 + length + 10.0, n_ground), rng.uniform(-20.0, 20.0, n_ground),
                   rng.normal(0, 0.02, n_ground)]
    pts = np.concatenate([ground, _box_surface_points(rng, lo, hi, n_map - n_ground)])
    map_points = pts[rng.permutation(n_map)].astype(np.float32)
    yaw = math.radians(2.0)
    T_true = np.eye(4)
    T_true[:3, :3] = [[math.cos(yaw), -math.sin(yaw), 0.0], [math.sin(yaw), math.cos(yaw), 0.0], [0.0, 0.0, 1.0]]
    T_true[:3, 3] = (x0 + 0.5 * length, 0.5, 1.73)
    el = np.radians(np.linspace(-24.8, 2.0, beams))
    az = np.linspace(-math.pi, math.pi, azimuths, endpoint=False)
    E, A = np.meshgrid(el, az, indexing="ij")
    d_local = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    t = _ray_cast(T_true[:3, 3], d_local @ T_true[:3, :3].T, lo, hi, max_range)
    ok = np.isfinite(t)
    r = t[ok] + rng.normal(0, 0.01, int(ok.sum()))
    scan = (d_local[ok] * r[:, None]).astype(np.float32)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(1.0)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    dR = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    T_init = T_true.copy()
    T_init[:3, :3] = dR @ T_true[:3, :3]
    T_init[:3, 3] += rng.normal(0, 0.15, 3)
    return LidarScene("street_lidar", map_points, scan, T_true, T_init)


@dataclass
class SpawnFrame:
    """One keyframe for anchor spawning: rendered alpha/depth of the current
    map, the sensor's depth, the pose and the map's Gaussian means."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_cw: np.ndarray        # [4,4] float64
    alpha: np.ndarray       # [H,W] float32
    depth: np.ndarray       # [H,W] float32
    depth_in: np.ndarray    # [H,W] float32, 0 = no measurement
    gauss_means: np.ndarray  # [G,3] float32


def keyframe_spawn(width: int = 1200, height: int = 680, f: float = 600.0, n_gauss: int = 300_000,
                   seed: int = 11) -> SpawnFrame:
    """A keyframe inside the 6x5x3 m room (camera at the centre looking +x):
    the input depth is the ray-cast room (1 mm noise, 2 % missing); the map
    misses the region behind image columns 700-999, rows 150-499 (rendered
    alpha U(0, 0.3) there, 1 elsewhere) and an object moved by 0.3 m in
    columns 100-299, rows 400-599 (rendered depth off by 0.3 m); the map's
    Gaussian means are 1 cm-jittered surface points seen outside the hole."""
    rng = np.random.default_rng(seed)
    T = look_at([3.0, 2.5, 1.5], [4.0, 2.5, 1.5], [0, 0, 1])
    R, t = T[:3, :3], T[:3, 3]
    o = -R.T @ t  # camera centre
    cx, cy = width / 2.0, height / 2.0
    jj, ii = np.mgrid[0:height, 0:width]
    rc = np.stack([(ii + 0.5 - cx) / f, (jj + 0.5 - cy) / f, np.ones_like(ii, dtype=np.float64)], -1)
    dw = rc @ R  # world direction of each pixel ray (z_c = 1)
    hi = np.array([6.0, 5.0, 3.0])
    with np.errstate(divide="ignore", invalid="ignore"):
        tb = np.where(dw > 0, (hi - o) / dw, np.where(dw < 0, -o / dw, np.inf))
    z = tb.min(-1)  # depth along the optical axis
    depth_in = (z + rng.normal(0, 1e-3, z.shape)).astype(np.float32)
    depth_in[rng.uniform(size=z.shape) < 0.02] = 0.0
    hole = (ii >= 700) & (ii < 1000) & (jj >= 150) & (jj < 500)
    moved = (ii >= 100) & (ii < 300) & (jj >= 400) & (jj < 600)
    alpha = np.where(hole, rng.uniform(0, 0.3, z.shape), 1.0).astype(np.float32)
    depth = (z + rng.normal(0, 1e-3, z.shape) + np.where(moved, 0.3, 0.0)).astype(np.float32)
    seen = np.flatnonzero(~hole.ravel())
    pick = rng.choice(seen, size=n_gauss)
    pts = o + (z.ravel()[pick] + rng.normal(0, 0.01, n_gauss))[:, None] * dw.reshape(-1, 3)[pick]
    return SpawnFrame(width, height, f, f, cx, cy, T, alpha, depth, depth_in, pts.astype(np.float32))


@dataclass
class AnchorStep:
    """Decode-shaped inputs of one training step for the anchor statistics."""
    anchors: np.ndarray     # [A,3] float32
    k: int
    src_index: np.ndarray   # [N] int32, ascending (anchor, slot)
    means: np.ndarray       # [N,3] float32
    grads: np.ndarray       # [N,3] float32, dL/dmu
    opacities: np.ndarray   # [N] float32
    visible: np.ndarray     # [N] int32 (tile counts)


def anchor_step(n_anchors: int = 100_000, k: int = K_PER_ANCHOR, keep: float = 0.5, seed: int = 12) -> AnchorStep:
    """The street's anchors (0.2 m voxels) with half of their k slots decoded:
    means within 0.2 m of the anchor, gradient norms U(0, 2e-3) in random
    directions, opacities U(0, 1), tile counts 0-3."""
    rng = np.random.default_rng(seed)
    anchors = street_anchors(n_anchors=n_anchors, seed=seed).anchors
    A = len(anchors)
    src = np.sort(rng.choice(A * k, size=int(keep * A * k), replace=False)).astype(np.int32)
    n = len(src)
    means = (anchors[src // k] + rng.uniform(-0.2, 0.2, size=(n, 3))).astype(np.float32)
    grads = (rng.normal(size=(n, 3)) * rng.uniform(0, 2e-3, size=(n, 1))).astype(np.float32)
    opac = rng.uniform(0, 1, n).astype(np.float32)
    vis = rng.integers(0, 4, n).astype(np.int32)
    return AnchorStep(anchors, k, src, means, grads, opac, vis)
