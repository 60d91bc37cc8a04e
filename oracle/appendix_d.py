"""World-frame edge-hinge models QTP / QTS and the Quadratic/Cubic-shell energy of App. D (oracle; test
infrastructure only).

App. D rewrites the edge-based hinge energies with the directional curvature operator applied in the world
frame instead of the corotational one:

* QTP (App. D, Eq. 79): Psi = A_E k_b / 2 * sum_c (L_n x_c)^2 over the three world coordinates c, with
  L_n = c_h [1/h1, -(|X_P3|/(|X_23| h1) + |X_Q3|/(|X_23| h4)), -(|X_P2|/(|X_23| h1) + |X_Q2|/(|X_23| h4)),
  1/h4], c_h = 2/(h1 + h4); P and Q are the feet of the wings X1 and X4 on the hinge line X2-X3, h1 and h4
  their distances. Its Hessian is k_b A_E L_n^T L_n (x) I and its gradient that Hessian times x.
* QTS: eps = L_n N^T x - L_n N0^T X (N^T x = (n.x_1, ..., n.x_4), n the frame normal of the ES model),
  Psi = A_E k_b eps^2 / 2, gradient A_E k_b eps d eps/dx with d eps/dx_j = L_j n + sum_i L_i (dn/dx_j)^T x_i.
* Quadratic / Cubic shell energy in the paper's terms (Eq. 89): Psi' = A'_E k_b (kappa')^2 / 2 with
  A'_E = A_E / 3 and kappa' = theta l / A'_E, theta the bending angle at the hinge (its change from rest for
  the Cubic shell) and l the hinge length. For small deflections kappa_m = 2 theta / (h1 + h4) and
  Psi' = 3 Psi (App. D, after Eq. 89).

The operator here is written from App. D's printed form: feet as orthogonal projections, the printed ratios
as unsigned Euclidean distances (``signed=False``). With ``signed=True`` the ratios |X_P3|/|X_23| and
|X_P2|/|X_23| become the signed barycentric coordinates 1 - s_p and s_p of the foot, the reading the rest of
the oracle and the CUDA library use (both coincide on stencils whose angles at the hinge are acute). The
bending angle is atan2((n1 x n2) . e, n1 . n2) with n1, n2 the unit normals of T123 and T432 and e the unit
hinge direction, independent of the curvature operator.
"""
from __future__ import annotations

import numpy as np


def _foot(xv, xa, xb):
    """Orthogonal projection of xv on the line xa-xb and its signed coordinate s (foot = xa + s (xb - xa))."""
    e = xb - xa
    s = np.sum((xv - xa) * e, axis=-1) / np.sum(e * e, axis=-1)
    return xa + s[..., None] * e, s


def _len(a):
    return np.sqrt(np.sum(a * a, axis=-1))


def world_operator(X, signed=True):
    """L_n of App. D for rest stencils X [S,4,3] (wing 1, hinge 2-3, wing 4). Returns (L_n [S,4], A_E [S])."""
    X1, X2, X3, X4 = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    P, sp = _foot(X1, X2, X3)
    Q, sq = _foot(X4, X2, X3)
    h1, h4 = _len(X1 - P), _len(X4 - Q)
    l23 = _len(X3 - X2)
    if signed:
        p3, p2, q3, q2 = 1.0 - sp, sp, 1.0 - sq, sq
    else:
        p3, p2, q3, q2 = _len(X3 - P) / l23, _len(X2 - P) / l23, _len(X3 - Q) / l23, _len(X2 - Q) / l23
    ch = 2.0 / (h1 + h4)
    L = ch[:, None] * np.stack([1.0 / h1, -(p3 / h1 + q3 / h4), -(p2 / h1 + q2 / h4), 1.0 / h4], axis=1)
    area = 0.5 * _len(np.cross(X2 - X1, X3 - X1)) + 0.5 * _len(np.cross(X3 - X4, X2 - X4))
    return L, area


def qtp_energy_gradient(x, idx, X, kb, signed=True):
    """QTP bending energy [S] and gradient dPsi/dx_j [S,4,3] of the stencils idx [S,4] at world positions x."""
    L, A = world_operator(X, signed)
    xs = x[idx]
    Lx = np.einsum("sj,sjc->sc", L, xs)                   # L_n x_c for c = x, y, z (no origin subtracted)
    energy = 0.5 * kb * A * np.sum(Lx * Lx, axis=1)
    grad = (kb * A)[:, None, None] * np.einsum("sj,sc->sjc", L, Lx)
    return energy, grad


def qtp_hessian(X, kb, signed=True):
    """Scalar Hessian blocks k_b A_E L_n^T L_n [S,4,4] (the matrix is this (x) I_3)."""
    L, A = world_operator(X, signed)
    return (kb * A)[:, None, None] * np.einsum("si,sj->sij", L, L)


def qts_energy_gradient(x, idx, X, kb, normal, signed=True):
    """QTS bending energy [S] and gradient [S,4,3]. normal(xs) -> (n [S,3], dn/dx_j [S,4,3,3]) is the frame
    normal of the ES model at stencil positions xs [S,4,3]."""
    L, A = world_operator(X, signed)
    xs = x[idx]
    n, J = normal(xs)
    n0, _ = normal(X)
    eps = np.einsum("sj,sjc,sc->s", L, xs, n) - np.einsum("sj,sjc,sc->s", L, X, n0)
    energy = 0.5 * kb * A * eps * eps
    g = np.einsum("si,sic->sc", L, xs)                    # sum_i L_i x_i (world frame)
    deps = np.einsum("sj,sc->sjc", L, n) + np.einsum("sjab,sa->sjb", J, g)
    grad = (kb * A * eps)[:, None, None] * deps
    return energy, grad


def bending_angle(xs):
    """Signed bending angle at the hinge of stencils xs [S,4,3]: the angle from n(T123) to n(T432) about the
    hinge direction x2 -> x3."""
    x1, x2, x3, x4 = xs[:, 0], xs[:, 1], xs[:, 2], xs[:, 3]
    n1 = np.cross(x2 - x1, x3 - x1)
    n2 = np.cross(x3 - x4, x2 - x4)
    n1 /= _len(n1)[:, None]
    n2 /= _len(n2)[:, None]
    e = (x3 - x2) / _len(x3 - x2)[:, None]
    return np.arctan2(np.sum(np.cross(n1, n2) * e, axis=1), np.sum(n1 * n2, axis=1))


def quadratic_shell_energy(x, idx, X, kb):
    """Quadratic / Cubic shell bending energy of App. D Eq. 89 per stencil: A'_E k_b (theta l / A'_E)^2 / 2 with
    A'_E = (A_123 + A_432) / 3, theta the bending angle's change from rest, l the rest hinge length."""
    X1, X2, X3, X4 = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    A3 = (0.5 * _len(np.cross(X2 - X1, X3 - X1)) + 0.5 * _len(np.cross(X3 - X4, X2 - X4))) / 3.0
    l = _len(X3 - X2)
    theta = bending_angle(x[idx]) - bending_angle(X)
    kappa = theta * l / A3
    return 0.5 * A3 * kb * kappa * kappa
