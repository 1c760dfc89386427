"""Pins of the FP64 fusion oracle (Eq. 14) and of its Adam step."""
import math

import numpy as np

import oracle


def test_identical_renders_give_zero():
    rng = np.random.default_rng(0)
    c = rng.uniform(size=(2, 3, 5, 7))
    d = rng.uniform(1, 3, size=(2, 5, 7))
    out = oracle.distill_loss(c, c, d, d)
    assert out["L"] == 0.0
    for k in ("d_rgb_a", "d_rgb_b", "d_depth_a", "d_depth_b"):
        assert np.abs(out[k]).max() == 0.0


def test_hand_worked_two_pixels():
    # one keyframe, 1x2 image; colour differences (0.1, 0.2, 0.3) and (0, 0, 0.6),
    # depth differences 0.5 and -0.5
    a = np.array([[[[0.1, 0.0]], [[0.2, 0.0]], [[0.3, 0.6]]]])
    b = np.zeros_like(a)
    da = np.array([[[2.5, 1.5]]])
    db = np.array([[[2.0, 2.0]]])
    out = oracle.distill_loss(a, b, da, db)
    L_c = (0.01 + 0.04 + 0.09 + 0.36) / 6
    L_d = (0.25 + 0.25) / 2
    assert abs(out["L_c"] - L_c) < 1e-15 and abs(out["L_d"] - L_d) < 1e-15
    assert abs(out["L"] - (L_c + L_d)) < 1e-15
    assert abs(out["d_rgb_a"][0, 2, 0, 1] - 2 * 0.6 / 6) < 1e-15
    assert abs(out["d_depth_b"][0, 0, 0] + 2 * 0.5 / 2) < 1e-15


def test_gradients_central_differences():
    rng = np.random.default_rng(1)
    a, b = rng.uniform(size=(3, 3, 4, 5)), rng.uniform(size=(3, 3, 4, 5))
    da, db = rng.uniform(1, 2, size=(3, 4, 5)), rng.uniform(1, 2, size=(3, 4, 5))
    out = oracle.distill_loss(a, b, da, db)
    h = 1e-6
    for _ in range(5):
        idx = tuple(rng.integers(0, n) for n in a.shape)
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        num = (oracle.distill_loss(ap, b, da, db, grads=False)["L"] -
               oracle.distill_loss(am, b, da, db, grads=False)["L"]) / (2 * h)
        assert abs(num - out["d_rgb_a"][idx]) < 1e-8
        idx = tuple(rng.integers(0, n) for n in da.shape)
        dp, dm = db.copy(), db.copy()
        dp[idx] += h
        dm[idx] -= h
        num = (oracle.distill_loss(a, b, da, dp, grads=False)["L"] -
               oracle.distill_loss(a, b, da, dm, grads=False)["L"]) / (2 * h)
        assert abs(num - out["d_depth_b"][idx]) < 1e-8


def test_adam_first_and_second_step():
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = oracle.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-8)
    # first step: the bias-corrected moments are g and g^2
    assert np.allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)
    g2 = np.array([1.0, 1.0, 1.0])
    p2, m2, v2 = oracle.adam_step(p, g2, m, v, 2, lr=0.1, eps=0.0)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    assert np.allclose(p2, p - 0.1 * mh / np.sqrt(vh), rtol=1e-14, atol=0)
    assert math.isclose(m2[0], 0.9 * 0.05 + 0.1, rel_tol=1e-15)


def test_keyframes_are_averaged():
    # Eq. 14's 1/m: two copies of the same keyframe pair give the loss of one
    # (a sum over keyframes would double it), and a second keyframe with zero
    # difference halves it
    rng = np.random.default_rng(5)
    a, b = rng.uniform(size=(1, 3, 4, 6)), rng.uniform(size=(1, 3, 4, 6))
    da, db = rng.uniform(1, 2, size=(1, 4, 6)), rng.uniform(1, 2, size=(1, 4, 6))
    one = oracle.distill_loss(a, b, da, db, grads=False)["L"]
    two = oracle.distill_loss(np.concatenate([a, a]), np.concatenate([b, b]),
                              np.concatenate([da, da]), np.concatenate([db, db]), grads=False)["L"]
    half = oracle.distill_loss(np.concatenate([a, a]), np.concatenate([b, a]),
                               np.concatenate([da, da]), np.concatenate([db, da]), grads=False)["L"]
    assert abs(two - one) <= 1e-15 * one
    assert abs(half - one / 2) <= 1e-15 * one
