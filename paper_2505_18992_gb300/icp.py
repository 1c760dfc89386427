"""Fine tracking front end: the voxel-hash ICP of Sec. III-B (Eq. 10-12).

Argument marshalling only: the map build, the double downsampling, the
correspondence search, the normal equations and the FP64 solve all run in
libvpgs.  Poses are local -> world, float64 [4,4] CUDA tensors.
"""
from __future__ import annotations

import ctypes

import torch

from . import vpgs as C
from .render import current_stream_handle

SYSTEM_SIZE = 29  # H upper triangle (21), b (6), sum rho, count
STOP_NAMES = {0: "iterations ran out", 1: "converged", 2: "too few correspondences", 3: "not positive definite"}


def _points(t: torch.Tensor, what: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 3 and t.is_contiguous()):
        raise ValueError(f"{what} must be a contiguous float32 CUDA tensor [n,3]")
    return t


def _pose(T: torch.Tensor) -> torch.Tensor:
    if not (T.is_cuda and T.dtype == torch.float64 and T.shape == (4, 4) and T.is_contiguous()):
        raise ValueError("poses are contiguous float64 CUDA tensors [4,4]")
    return T


class VoxelMap:
    """Voxel hash of the map points (the Gaussian means) with edge `voxel`."""

    def __init__(self, points: torch.Tensor, voxel: float):
        self.points = _points(points, "map points")
        self.n = int(points.shape[0])
        self.voxel = float(voxel)
        nbytes = C.vpgs_icp_map_bytes(self.n)
        if nbytes == 0:
            raise ValueError("too many map points")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=points.device)
        self.rebuild()

    def rebuild(self, points: torch.Tensor | None = None):
        """Rebuilds the hash (from new points of the same count, if given)."""
        if points is not None:
            if points.shape[0] != self.n:
                raise ValueError("rebuild keeps the point count")
            self.points = _points(points, "map points")
        C.check(C.vpgs_icp_build_map(self.buf.data_ptr(), self.buf.numel(), self.points.data_ptr(), self.n,
                                     self.voxel, current_stream_handle()), "vpgs_icp_build_map")

    def info(self) -> dict:
        inf = C.vpgs_icp_map_info()
        C.check(C.vpgs_icp_map_query(self.buf.data_ptr(), ctypes.byref(inf), current_stream_handle()),
                "vpgs_icp_map_query")
        return {"n_points": inf.n_points, "n_voxels": inf.n_voxels, "capacity": inf.capacity,
                "status": inf.status, "voxel": inf.voxel}


def icp_opts(map_voxel: float, voxel_1: float, voxel_2: float, tau: float, sigma: float, iterations: int = 20,
             eps: float = 1e-6) -> C.vpgs_icp_opts:
    return C.vpgs_icp_opts(map_voxel, voxel_1, voxel_2, tau, sigma, eps, int(iterations), 0)


class ICP:
    """Registration of scans of up to `max_scan_points` points against a VoxelMap."""

    def __init__(self, max_scan_points: int, voxel_1: float, voxel_2: float, tau: float, sigma: float,
                 iterations: int = 20, eps: float = 1e-6, device="cuda"):
        self.cap = int(max_scan_points)
        nbytes = C.vpgs_icp_workspace_bytes(self.cap)
        if nbytes == 0:
            raise ValueError("invalid scan capacity")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.report_buf = torch.zeros(ctypes.sizeof(C.vpgs_icp_report), dtype=torch.uint8, device=device)
        self.v1, self.v2, self.tau, self.sigma = float(voxel_1), float(voxel_2), float(tau), float(sigma)
        self.iterations, self.eps = int(iterations), float(eps)

    def register(self, vmap: VoxelMap, scan: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
        """Refines T (in place) so that T scan lands on the map; returns T."""
        _points(scan, "scan")
        _pose(T)
        if scan.shape[0] > self.cap:
            raise ValueError("scan larger than the workspace")
        opts = icp_opts(vmap.voxel, self.v1, self.v2, self.tau, self.sigma, self.iterations, self.eps)
        C.check(C.vpgs_icp_register(self.ws.data_ptr(), self.ws.numel(), vmap.buf.data_ptr(), vmap.buf.numel(),
                                    vmap.n, scan.data_ptr(), int(scan.shape[0]), ctypes.byref(opts), T.data_ptr(),
                                    self.report_buf.data_ptr(), current_stream_handle()), "vpgs_icp_register")
        return T

    def report(self) -> dict:
        """The last registration's report (synchronises)."""
        r = C.vpgs_icp_report.from_buffer_copy(bytes(self.report_buf.cpu().numpy()))
        return {"status": r.status, "iterations": r.iterations, "n_source": r.n_source, "n_corr": r.n_corr,
                "stop": r.stop, "cost": r.cost, "xi_norm": r.xi_norm}


def downsample(scan: torch.Tensor, voxel_1: float, voxel_2: float, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Original indices (ascending, int32) kept by the double downsampling."""
    _points(scan, "scan")
    n = int(scan.shape[0])
    if ws is None:
        ws = torch.empty(C.vpgs_icp_workspace_bytes(n), dtype=torch.uint8, device=scan.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=scan.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=scan.device)
    C.check(C.vpgs_icp_downsample(ws.data_ptr(), ws.numel(), scan.data_ptr(), n, voxel_1, voxel_2, idx.data_ptr(),
                                  cnt.data_ptr(), current_stream_handle()), "vpgs_icp_downsample")
    return idx[:int(cnt.item())]


def linearize(vmap: VoxelMap, src: torch.Tensor, T: torch.Tensor, centre: torch.Tensor, tau: float, sigma: float,
              want_corr: bool = True):
    """One linearisation of Eq. 11 at T: (system float64 [29], corr int32 [n] or None)."""
    _points(src, "source points")
    _pose(T)
    dev = src.device
    ws = torch.empty(C.vpgs_icp_workspace_bytes(0), dtype=torch.uint8, device=dev)
    system = torch.empty(SYSTEM_SIZE, dtype=torch.float64, device=dev)
    corr = torch.empty(max(int(src.shape[0]), 1), dtype=torch.int32, device=dev) if want_corr else None
    c = centre.to(device=dev, dtype=torch.float64).contiguous()
    C.check(C.vpgs_icp_linearize(ws.data_ptr(), ws.numel(), vmap.buf.data_ptr(), vmap.buf.numel(), vmap.n,
                                 vmap.voxel, src.data_ptr(), int(src.shape[0]), T.data_ptr(), c.data_ptr(), tau,
                                 sigma, system.data_ptr(), C.ptr(corr), current_stream_handle()),
            "vpgs_icp_linearize")
    return system, (corr[:int(src.shape[0])] if corr is not None else None)


def unpack_system(system):
    """(H [6,6], b [6], cost, count) from the 29 numbers of a linearisation."""
    import numpy as np

    s = np.asarray(system, np.float64)
    H = np.zeros((6, 6))
    k = 0
    for r in range(6):
        for c in range(r, 6):
            H[r, c] = H[c, r] = s[k]
            k += 1
    return H, s[21:27].copy(), float(s[27]), float(s[28])
