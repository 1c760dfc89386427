"""FP64 CPU oracle of the camera-pose step of coarse tracking (Sec. III-B).

TEST INFRASTRUCTURE: see the package docstring; never used by the product.

The paper optimises the pose with the photometric and depth losses but gives
no step rule.  The reading: a left update T_cw <- Exp(xi) T_cw with
xi = (rho, phi) in se(3), xi = -lr * g (plain step) or the Adam direction
(beta1 = 0.9, beta2 = 0.999, eps = 1e-15, bias-corrected), lr separate for
rho and phi.  Exp is the matrix exponential of the 4x4 twist [[phi^, rho], [0, 0]].

Pins: tests/test_oracle_pose.py (Exp(0) = I, Exp(xi) Exp(-xi) = I, rotation
part orthonormal with det 1, Rodrigues angle, the closed-form rotation and V
translation on random twists, the left update moving T_cw's translation,
hand-worked first and second Adam steps).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def twist(xi):
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    H = np.zeros((4, 4))
    H[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    H[:3, 3] = rho
    return H


def se3_exp(xi):
    return scipy.linalg.expm(twist(xi))


def pose_step(T_cw, grad, lr, adam=None):
    """One step for every view.  T_cw [V,4,4], grad [V,6], lr (rho, phi);
    adam: None or [V,13] state (m[6], v[6], step) updated in place.
    Returns the new T_cw."""
    T_cw = np.asarray(T_cw, np.float64).reshape(-1, 4, 4)
    grad = np.asarray(grad, np.float64).reshape(-1, 6)
    lrv = np.array([lr[0]] * 3 + [lr[1]] * 3)
    out = np.empty_like(T_cw)
    for v in range(T_cw.shape[0]):
        g = grad[v]
        if adam is None:
            xi = -lrv * g
        else:
            m, s = adam[v, :6], adam[v, 6:12]
            k = adam[v, 12] + 1.0
            adam[v, 12] = k
            m[:] = 0.9 * m + 0.1 * g
            s[:] = 0.999 * s + 0.001 * g * g
            mh = m / (1.0 - 0.9 ** k)
            sh = s / (1.0 - 0.999 ** k)
            xi = -lrv * mh / (np.sqrt(sh) + 1e-15)
        out[v] = se3_exp(xi) @ T_cw[v]
    return out
