"""Pins of the pose-step oracle."""
import math

import numpy as np

import oracle


def test_exponential_identities():
    rng = np.random.default_rng(0)
    assert np.allclose(oracle.se3_exp(np.zeros(6)), np.eye(4), atol=0)
    for _ in range(5):
        xi = rng.normal(size=6)
        E = oracle.se3_exp(xi)
        assert np.allclose(E @ oracle.se3_exp(-xi), np.eye(4), atol=1e-12)
        R = E[:3, :3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and abs(np.linalg.det(R) - 1) < 1e-12
        # the rotation angle equals |phi| (Rodrigues)
        ang = math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))
        assert abs(ang - min(np.linalg.norm(xi[3:]), 2 * math.pi - np.linalg.norm(xi[3:]))) < 1e-9
    # a pure translation twist moves by rho
    E = oracle.se3_exp([0.1, -0.2, 0.3, 0, 0, 0])
    assert np.allclose(E[:3, 3], [0.1, -0.2, 0.3], atol=1e-15)


def test_plain_and_adam_steps_by_hand():
    T = np.eye(4)[None]
    g = np.array([[2.0, 0, 0, 0, 0, 0]])
    out = oracle.pose_step(T, g, (0.01, 0.02))
    assert np.allclose(out[0, :3, 3], [-0.02, 0, 0], atol=1e-15)
    # Adam's first bias-corrected step has magnitude lr in every non-zero component
    st = np.zeros((1, 13))
    g = np.array([[3.0, -4.0, 0, 0, 0, 0.5]])
    out = oracle.pose_step(T, g, (0.01, 0.02), adam=st)
    assert st[0, 12] == 1.0
    assert np.allclose(st[0, :6], 0.1 * g[0]) and np.allclose(st[0, 6:12], 0.001 * g[0] ** 2)
    xi = np.array([-0.01, 0.01, 0.0, 0.0, 0.0, -0.02])  # -lr * sign(g) per component
    R = out[0, :3, :3]
    assert abs(math.atan2(R[1, 0], R[0, 0]) - xi[5]) < 1e-12
    # translation = V rho with V = I + (1-cos t)/t^2 W + (t - sin t)/t^3 W^2 (closed form)
    t = abs(xi[5])
    W = np.array([[0, -xi[5], 0], [xi[5], 0, 0], [0, 0, 0]])
    V = np.eye(3) + (1 - math.cos(t)) / t ** 2 * W + (t - math.sin(t)) / t ** 3 * (W @ W)
    assert np.allclose(out[0, :3, 3], V @ xi[:3], atol=1e-9)


def _hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)


def test_exponential_matches_the_closed_form():
    # Rodrigues for the rotation and V = I + (1-cos t)/t^2 W + (t-sin t)/t^3 W^2
    # for the translation, on random twists (t = |phi|)
    rng = np.random.default_rng(4)
    for _ in range(20):
        xi = rng.normal(size=6) * rng.uniform(0.01, 2.0)
        rho, phi = xi[:3], xi[3:]
        t = np.linalg.norm(phi)
        W = _hat(phi)
        R = np.eye(3) + math.sin(t) / t * W + (1 - math.cos(t)) / t ** 2 * (W @ W)
        V = np.eye(3) + (1 - math.cos(t)) / t ** 2 * W + (t - math.sin(t)) / t ** 3 * (W @ W)
        E = oracle.se3_exp(xi)
        assert np.allclose(E[:3, :3], R, atol=1e-12)
        assert np.allclose(E[:3, 3], V @ rho, atol=1e-12)
        assert np.array_equal(E[3], [0, 0, 0, 1])


def test_the_step_updates_from_the_left():
    # T_cw <- Exp(xi) T_cw: a rotation step about z turns the translation of
    # T_cw with it (a right update, T_cw Exp(xi), would leave it in place)
    T = np.eye(4)
    T[:3, 3] = [1.0, 0.0, 0.0]
    g = np.array([[0, 0, 0, 0, 0, -2.0]])
    out = oracle.pose_step(T[None], g, (0.01, 0.02))  # xi = -lr g = (0, 0, 0, 0, 0, 0.04)
    th = 0.04
    assert np.allclose(out[0, :3, 3], [math.cos(th), math.sin(th), 0.0], atol=1e-15)
    assert np.allclose(out[0, :3, :3], [[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0],
                                        [0, 0, 1]], atol=1e-15)


def test_adam_second_step_by_hand():
    # two steps along rho_x with gradients 1 then 3: m = 0.9 * 0.1 + 0.1 * 3,
    # v = 0.999 * 0.001 + 0.001 * 9, bias corrections 1 - 0.9^2 and 1 - 0.999^2
    st = np.zeros((1, 13))
    T = np.eye(4)[None]
    oracle.pose_step(T, np.array([[1.0, 0, 0, 0, 0, 0]]), (0.01, 0.02), adam=st)
    out = oracle.pose_step(T, np.array([[3.0, 0, 0, 0, 0, 0]]), (0.01, 0.02), adam=st)
    m, v = 0.39, 0.009999
    step = -0.01 * (m / 0.19) / (math.sqrt(v / (1 - 0.999 ** 2)) + 1e-15)
    assert st[0, 12] == 2.0
    assert abs(st[0, 0] - m) < 1e-15 and abs(st[0, 6] - v) < 1e-15
    assert abs(out[0, 0, 3] - step) < 1e-15  # a pure translation step moves by rho
    assert np.allclose(out[0, :3, :3], np.eye(3), atol=0)
