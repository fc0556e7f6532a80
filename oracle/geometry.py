"""Maps from the reference box of the forest to a curved physical domain.

The paper runs its ventricle benchmarks on curved hexahedral meshes (Sec. 3.3, idealized
left ventricle).  Here the forest stays on the reference box X in [0, L_0] x [0, L_1]
(x [0, L_2]) and a smooth map x = Phi(X) gives the physical domain; an element of level l
with reference lower corner X_c is the image of [X_c, X_c + h_l], i.e. its element map is
x(xi) = Phi(X_c + (xi + 1) h_l / 2) with Jacobian J = DPhi(X) diag(h_l / 2).

Maps (``prob.geometry``, parameters ``prob.geo``):
  1  affine:  Phi(X) = A X + b, geo = (A row-major 3x3, b_0, b_1, b_2); 2D uses the leading
     2x2 block of A and b_0, b_1.
  2  shell:   an ellipsoidal shell sector, geo = (a_i, b_i, c_i, a_o, b_o, c_o, phi0, dphi,
     theta0, dtheta).  With s = X_0 / L_0, t = X_1 / L_1, u = X_2 / L_2 (3D),
        azimuth phi = phi0 + s dphi, polar angle theta = theta0 + t dtheta,
        semi-axes a(u) = a_i + u (a_o - a_i) (b, c likewise),
        x = (a sin(theta) cos(phi), b sin(theta) sin(phi), c cos(theta));
     in 2D, u = X_1 / L_1 and x = (a(u) cos(phi), b(u) sin(phi)).

DPhi[i][j] = d x_i / d X_j, written out by hand from these formulas.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

AFFINE = 1
SHELL = 2


def _affine(prob):
    g = np.asarray(prob.geo, dtype=np.float64)
    d = prob.dim
    A = g[:9].reshape(3, 3)[:d, :d]
    b = g[9:12][:d]
    return A, b


def phi(prob, X: np.ndarray) -> np.ndarray:
    """Physical points of reference points X (N, d)."""
    X = np.asarray(X, dtype=np.float64)
    d = prob.dim
    if prob.geometry == 0:
        return X.copy()
    if prob.geometry == AFFINE:
        A, b = _affine(prob)
        return X @ A.T + b[None, :]
    if prob.geometry == SHELL:
        ai, bi, ci, ao, bo, co, p0, dp, t0, dt = prob.geo[:10]
        L = prob.extent
        az = p0 + X[:, 0] / L[0] * dp
        if d == 2:
            u = X[:, 1] / L[1]
            a = ai + u * (ao - ai)
            b = bi + u * (bo - bi)
            return np.stack([a * np.cos(az), b * np.sin(az)], axis=1)
        th = t0 + X[:, 1] / L[1] * dt
        u = X[:, 2] / L[2]
        a = ai + u * (ao - ai)
        b = bi + u * (bo - bi)
        c = ci + u * (co - ci)
        return np.stack([a * np.sin(th) * np.cos(az), b * np.sin(th) * np.sin(az), c * np.cos(th)], axis=1)
    raise ValueError("unknown geometry %r" % (prob.geometry,))


def dphi(prob, X: np.ndarray) -> np.ndarray:
    """DPhi at reference points X: (N, d, d) with [n, i, j] = d x_i / d X_j."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if prob.geometry == 0:
        return np.broadcast_to(np.eye(d), (n, d, d)).copy()
    if prob.geometry == AFFINE:
        A, _ = _affine(prob)
        return np.broadcast_to(A, (n, d, d)).copy()
    if prob.geometry == SHELL:
        ai, bi, ci, ao, bo, co, p0, dp, t0, dt = prob.geo[:10]
        L = prob.extent
        az = p0 + X[:, 0] / L[0] * dp
        J = np.zeros((n, d, d))
        if d == 2:
            u = X[:, 1] / L[1]
            a = ai + u * (ao - ai)
            b = bi + u * (bo - bi)
            J[:, 0, 0] = -a * np.sin(az) * dp / L[0]
            J[:, 1, 0] = b * np.cos(az) * dp / L[0]
            J[:, 0, 1] = (ao - ai) * np.cos(az) / L[1]
            J[:, 1, 1] = (bo - bi) * np.sin(az) / L[1]
            return J
        th = t0 + X[:, 1] / L[1] * dt
        u = X[:, 2] / L[2]
        a = ai + u * (ao - ai)
        b = bi + u * (bo - bi)
        c = ci + u * (co - ci)
        st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(az), np.cos(az)
        J[:, 0, 0] = -a * st * sp * dp / L[0]
        J[:, 1, 0] = b * st * cp * dp / L[0]
        J[:, 2, 0] = 0.0
        J[:, 0, 1] = a * ct * cp * dt / L[1]
        J[:, 1, 1] = b * ct * sp * dt / L[1]
        J[:, 2, 1] = -c * st * dt / L[1]
        J[:, 0, 2] = (ao - ai) * st * cp / L[2]
        J[:, 1, 2] = (bo - bi) * st * sp / L[2]
        J[:, 2, 2] = (co - ci) * ct / L[2]
        return J
    raise ValueError("unknown geometry %r" % (prob.geometry,))
