"""Pins of the FP64 oracle of submap expansion and anchor maintenance (Sec. III-A)."""
import importlib

import numpy as np

A = importlib.import_module("oracle.anchors")


def test_mask_hand_worked():
    alpha = np.array([[0.1, 0.9, 0.9], [0.9, 0.9, 0.2]])
    depth = np.array([[1.0, 1.0, 2.0], [1.0, 3.0, 1.0]])
    dep_in = np.array([[1.0, 1.05, 1.0], [0.0, 1.0, 0.0]])
    m = A.spawn_mask(alpha, depth, dep_in, tau_alpha=0.5, delta_d=0.1)
    # (0,0) low alpha; (0,1) depth within 0.1; (0,2) depth off by 1; (1,0) no input depth;
    # (1,1) depth off by 2; (1,2) low alpha but no input depth
    assert m.tolist() == [[True, False, True], [False, True, False]]


def test_sample_ranks():
    assert A.sample_ranks(10, 3).tolist() == [3, 6, 9]  # worked by hand
    assert A.sample_ranks(4, 10).tolist() == [0, 1, 2, 3]
    assert A.sample_ranks(0, 5).tolist() == []
    rng = np.random.default_rng(0)
    for _ in range(50):
        c = int(rng.integers(1, 5000))
        m = int(rng.integers(1, c + 1))
        r = A.sample_ranks(c, m)
        assert len(r) == m and r[-1] == c - 1
        gaps = np.diff(np.concatenate([[-1], r]))
        assert gaps.max() - gaps.min() <= 1  # evenly spread


def test_back_projection_inverts_the_pinhole():
    rng = np.random.default_rng(1)
    from oracle.pose import se3_exp
    T = se3_exp(rng.normal(scale=0.5, size=6))
    fx, fy, cx, cy = 500.0, 480.0, 320.0, 240.0
    i = rng.integers(0, 640, 200)
    j = rng.integers(0, 480, 200)
    d = rng.uniform(0.5, 20.0, 200).astype(np.float32)
    p = A.back_project(i, j, d, fx, fy, cx, cy, T).astype(np.float64)
    xc = p @ T[:3, :3].T + T[:3, 3]
    assert np.allclose(xc[:, 2], d, rtol=1e-6)
    assert np.allclose(fx * xc[:, 0] / xc[:, 2] + cx, i + 0.5, atol=1e-3)
    assert np.allclose(fy * xc[:, 1] / xc[:, 2] + cy, j + 0.5, atol=1e-3)


def test_voxel_centres_and_first_voxels():
    c = A.voxel_centres(np.array([[-1, 0, 2]]), 0.5)
    assert c.tolist() == [[-0.25, 0.25, 1.25]]
    pts = np.array([[0.1, 0.1, 0.1], [1.2, 0, 0], [0.2, 0.3, 0.4], [-0.1, 0, 0], [1.9, 0.5, 0.5]], np.float32)
    keys, first = A.first_voxels(pts, 1.0)
    assert keys.tolist() == [[0, 0, 0], [1, 0, 0], [-1, 0, 0]] and first.tolist() == [0, 1, 3]


def test_radius_rule_against_brute_force():
    rng = np.random.default_rng(2)
    mp = rng.uniform(-2, 2, size=(2000, 3)).astype(np.float32)
    c = rng.uniform(-2.2, 2.2, size=(300, 3)).astype(np.float32)
    got = A.any_within(c, mp, 0.12)
    r2 = np.float32(0.12) * np.float32(0.12)
    for n in range(len(c)):
        d = mp - c[n]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        assert got[n] == bool((d2 < r2).any())
    assert not A.any_within(c, np.zeros((0, 3), np.float32), 0.5).any()


def test_spawn_hand_worked():
    # 4x4 image, identity pose, one pixel (col 2, row 1) with low alpha and depth 2:
    # x_c = ((2.5 - 2) / 2 * 2, (1.5 - 2) / 2 * 2, 2) = (0.5, -0.5, 2)
    alpha = np.ones((4, 4))
    alpha[1, 2] = 0.0
    depth = np.full((4, 4), 2.0)
    dep_in = np.full((4, 4), 2.0, np.float32)
    new, pts = A.spawn(alpha, depth, dep_in, 2.0, 2.0, 2.0, 2.0, np.eye(4), 0.5, 0.1, 10, 1.0, 0.2,
                       np.zeros((0, 3), np.float32))
    assert pts.tolist() == [[0.5, -0.5, 2.0]]
    assert new.tolist() == [[0.5, -0.5, 2.5]]  # voxel (0, -1, 2)
    # a Gaussian mean 0.1 from the centre suppresses it, one 0.3 away does not
    new2, _ = A.spawn(alpha, depth, dep_in, 2.0, 2.0, 2.0, 2.0, np.eye(4), 0.5, 0.1, 10, 1.0, 0.2,
                      np.array([[0.5, -0.4, 2.5]], np.float32))
    new3, _ = A.spawn(alpha, depth, dep_in, 2.0, 2.0, 2.0, 2.0, np.eye(4), 0.5, 0.1, 10, 1.0, 0.2,
                      np.array([[0.5, -0.2, 2.5]], np.float32))
    assert len(new2) == 0 and len(new3) == 1


def test_statistics_against_loops():
    rng = np.random.default_rng(3)
    n_anchors, k = 50, 4
    src = np.sort(rng.choice(n_anchors * k, size=120, replace=False))
    g = rng.normal(size=(120, 3))
    o = rng.uniform(0, 1, 120)
    vis = rng.integers(0, 3, 120)
    st = A.accumulate_stats(A.new_stats(n_anchors), src, k, g, o, vis)
    st = A.accumulate_stats(st, src[:60], k, g[:60], o[:60], vis[:60])
    for a in range(n_anchors):
        want = [0.0, 0, 0.0, 0]
        for rep in (120, 60):
            rows = [i for i in range(rep) if src[i] // k == a]
            want[0] += sum(np.linalg.norm(g[i]) for i in rows if vis[i])
            want[1] += sum(1 for i in rows if vis[i])
            want[2] += sum(o[i] for i in rows)
            want[3] += 1 if rows else 0
        assert np.isclose(st["g_sum"][a], want[0]) and st["g_cnt"][a] == want[1]
        assert np.isclose(st["o_sum"][a], want[2]) and st["visits"][a] == want[3]


def test_prune_and_grow_hand_worked():
    st = A.new_stats(4)
    st["visits"][:] = [0, 2, 2, 5]
    st["o_sum"][:] = [0.0, 0.3, 0.1, 4.0]
    assert A.prune(st, 0.1).tolist() == [0, 1, 3]  # anchor 2: 0.05 per visit < 0.1
    st["g_cnt"][:] = [0, 2, 1, 3]
    st["g_sum"][:] = [9.0, 1.0, 0.1, 3.3]  # averages -, 0.5, 0.1, 1.1
    k = 2
    src = np.array([2, 3, 4, 6, 7])  # anchors 1, 1, 2, 3, 3
    means = np.array([[0.2, 0.2, 0.2], [1.5, 0.2, 0.2], [5.0, 5, 5], [1.7, 0.1, 0.9], [2.5, 0, 0]], np.float32)
    anchors = np.array([[0.5, 0.5, 0.5]], np.float32)  # occupies voxel (0,0,0)
    new = A.grow(st, src, k, means, 0.4, 1.0, anchors)
    # hot anchors 1 and 3; their means fall in voxels (0,0,0) occupied, (1,0,0), (1,0,0), (2,0,0)
    assert new.tolist() == [[1.5, 0.5, 0.5], [2.5, 0.5, 0.5]]
