"""GPU parity of the voxel-hash ICP (Sec. III-B, Eq. 10-12) against the FP64 oracle.

Tolerances.  Integer work is bit-exact: voxel counts of the map, the indices
kept by the double downsampling, the correspondence of every source point
(both sides decide in float32 with correctly rounded operations).  The normal
equations are summed from FP32 per-pair terms (FP32 within a block, FP64
across blocks): every entry within 1e-5 of the sum of the absolute per-pair
terms (about 100 float32 roundings of headroom).  The registered pose: both
sides stop at |xi| < eps on the same cost, so the poses agree to what the
FP32 sums resolve, 1e-4 per entry (m, and unitless for the rotation).
"""
import importlib

import numpy as np
import pytest
import torch

from paper_2505_18992_gb300 import scenes
from paper_2505_18992_gb300.vpgs import VpgsError
from tests.helpers import dev

I = importlib.import_module("oracle.icp")
pytestmark = pytest.mark.gpu

MAP_VOXEL, V1, V2, TAU, SIGMA = 1.0, 0.5, 1.5, 1.0, 0.3
SYS_RTOL = 1e-5
POSE_ATOL = 1e-4


@pytest.fixture(scope="module")
def street():
    return scenes.street_lidar()


@pytest.fixture(scope="module")
def street_map(street):
    from paper_2505_18992_gb300.icp import VoxelMap
    return VoxelMap(dev(street.map_points), MAP_VOXEL)


def _check_system(system, corr, s, mp, sigma, c):
    from paper_2505_18992_gb300.icp import unpack_system
    ok = corr >= 0
    H, b, cost, Ha, ba = I.normal_equations(s[ok], mp[corr[ok]].astype(np.float64), sigma, c=c, magnitude=True)
    Hg, bg, costg, count = unpack_system(system)
    assert count == ok.sum()
    assert np.all(np.abs(Hg - H) <= SYS_RTOL * Ha + 1e-9)
    assert np.all(np.abs(bg - b) <= SYS_RTOL * ba + 1e-9)
    assert abs(costg - cost) <= SYS_RTOL * max(cost, 1.0)


def test_map_voxel_counts(street, street_map):
    info = street_map.info()
    keys = I.voxel_keys(street.map_points, MAP_VOXEL)
    assert info["status"] == 0 and info["n_points"] == len(street.map_points)
    assert info["n_voxels"] == len(np.unique(keys, axis=0))


@pytest.mark.parametrize("n", [0, 1, 1001])
def test_small_maps(n):
    from paper_2505_18992_gb300.icp import VoxelMap
    rng = np.random.default_rng(n)
    pts = rng.uniform(-3, 3, size=(n, 3)).astype(np.float32)
    m = VoxelMap(dev(pts.reshape(-1, 3)), 0.5)
    info = m.info()
    assert info["status"] == 0
    assert info["n_voxels"] == (len(np.unique(I.voxel_keys(pts, 0.5), axis=0)) if n else 0)


def test_map_flags_non_finite_points():
    from paper_2505_18992_gb300.icp import VoxelMap
    pts = np.random.default_rng(1).uniform(-3, 3, size=(500, 3)).astype(np.float32)
    pts[17, 1] = np.nan
    info = VoxelMap(dev(pts), 0.5).info()
    assert info["status"] == 3  # VPGS_ERR_NONFINITE
    assert info["n_voxels"] == len(np.unique(I.voxel_keys(np.delete(pts, 17, 0), 0.5), axis=0))


def test_downsampling_matches_the_oracle(street):
    from paper_2505_18992_gb300.icp import downsample
    got = downsample(dev(street.scan), V1, V2).cpu().numpy()
    assert np.array_equal(got, I.double_downsample(street.scan, V1, V2))
    rng = np.random.default_rng(2)
    for n in (0, 1, 777, 40_000):
        p = rng.uniform(-4, 4, size=(n, 3)).astype(np.float32)
        got = downsample(dev(p.reshape(-1, 3)), 0.2, 0.45).cpu().numpy()
        assert np.array_equal(got, I.double_downsample(p, 0.2, 0.45)), n


def test_linearisation_matches_the_oracle(street, street_map):
    from paper_2505_18992_gb300.icp import linearize
    src = street.scan[I.double_downsample(street.scan, V1, V2)]
    T = street.T_init
    c = T[:3, 3].copy()
    system, corr = linearize(street_map, dev(src), dev(T, torch.float64), torch.tensor(c), TAU, SIGMA)
    corr = corr.cpu().numpy()
    s = I.transform(T, src)
    want = I.nearest_f32(s, street.map_points, TAU)
    assert np.array_equal(corr, want)
    assert (corr >= 0).mean() > 0.8
    _check_system(system.cpu().numpy(), corr, s, street.map_points, SIGMA, c)


def test_linearisation_ties_and_tail():
    """Duplicate map points (ties go to the lower index), a point out of every
    voxel's reach, a ragged source count and tau < voxel."""
    from paper_2505_18992_gb300.icp import VoxelMap, linearize
    rng = np.random.default_rng(3)
    mp = rng.uniform(-2, 2, size=(5003, 3)).astype(np.float32)
    mp[4000:4100] = mp[10:110]  # exact duplicates with higher indices
    src = np.concatenate([mp[5:200] + rng.normal(0, 0.01, size=(195, 3)).astype(np.float32),
                          rng.uniform(-2.5, 2.5, size=(38, 3)).astype(np.float32),
                          np.array([[40.0, 0, 0]], np.float32)])
    vmap = VoxelMap(dev(mp), 0.25)
    T = np.eye(4)
    tau = 0.2
    system, corr = linearize(vmap, dev(src), dev(T, torch.float64), torch.zeros(3), tau, SIGMA)
    corr = corr.cpu().numpy()
    s = I.transform(T, src)
    assert np.array_equal(corr, I.nearest_f32(s, mp, tau))
    assert corr[-1] == -1
    _check_system(system.cpu().numpy(), corr, s, mp, SIGMA, np.zeros(3))


def _register(street_map, scan, T0, iterations=60, eps=1e-6):
    from paper_2505_18992_gb300.icp import ICP
    icp = ICP(len(scan), V1, V2, TAU, SIGMA, iterations=iterations, eps=eps)
    T = dev(T0, torch.float64)
    icp.register(street_map, dev(scan.reshape(-1, 3)), T)
    return T.cpu().numpy(), icp.report(), icp


def test_registration_matches_the_oracle(street, street_map):
    T, rep, _ = _register(street_map, street.scan, street.T_init)
    ref = I.icp(street.scan, street.map_points, street.T_init, V1, V2, TAU, SIGMA, iterations=60, eps=1e-6)
    assert rep["status"] == 0
    assert rep["n_source"] == len(ref["src_idx"])
    assert rep["stop"] == ref["stop"] == I.CONVERGED
    assert np.abs(T - ref["T"]).max() < POSE_ATOL
    assert np.abs(T[:3, 3] - street.T_true[:3, 3]).max() < 0.03
    assert abs(rep["n_corr"] - ref["correspondences"]) <= 2


def test_registration_with_outliers_and_a_ragged_scan(street, street_map):
    rng = np.random.default_rng(4)
    scan = np.concatenate([street.scan[:50_001],
                           rng.uniform(-30, 30, size=(3000, 3)).astype(np.float32)])
    T, rep, _ = _register(street_map, scan, street.T_init)
    ref = I.icp(scan, street.map_points, street.T_init, V1, V2, TAU, SIGMA, iterations=60, eps=1e-6)
    assert rep["n_source"] == len(ref["src_idx"])
    assert rep["stop"] == ref["stop"]
    assert np.abs(T - ref["T"]).max() < POSE_ATOL


def test_graph_replay_is_bit_identical(street, street_map):
    from paper_2505_18992_gb300.icp import ICP
    icp = ICP(len(street.scan), V1, V2, TAU, SIGMA, iterations=30, eps=1e-6)
    scan = dev(street.scan)
    T0 = dev(street.T_init, torch.float64)
    T_eager = T0.clone()
    icp.register(street_map, scan, T_eager)
    torch.cuda.synchronize()
    T_graph = T0.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        icp.register(street_map, scan, T_graph)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        icp.register(street_map, scan, T_graph)
    for _ in range(2):
        T_graph.copy_(T0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(T_graph, T_eager)


def test_degenerate_inputs(street, street_map):
    from paper_2505_18992_gb300.icp import ICP, VoxelMap
    # empty scan: fewer than 6 correspondences on the first iteration, pose unchanged
    T, rep, _ = _register(street_map, np.zeros((0, 3), np.float32), street.T_init)
    assert rep["stop"] == 2 and rep["iterations"] == 1 and np.array_equal(T, street.T_init)
    # empty map
    empty = VoxelMap(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), MAP_VOXEL)
    T, rep, _ = _register(empty, street.scan, street.T_init)
    assert rep["stop"] == 2 and rep["n_corr"] == 0 and np.array_equal(T, street.T_init)
    # a non-finite scan point is dropped and reported
    scan = street.scan[:20_000].copy()
    scan[123] = np.inf
    T, rep, _ = _register(street_map, scan, street.T_init)
    assert rep["status"] == 3
    assert rep["n_source"] == len(I.double_downsample(np.delete(scan, 123, 0), V1, V2))
    # host-side argument check: tau above the map voxel
    icp = ICP(10, V1, V2, TAU * 2, SIGMA)
    with pytest.raises(VpgsError):
        icp.register(street_map, dev(street.scan[:10]), dev(street.T_init, torch.float64))
