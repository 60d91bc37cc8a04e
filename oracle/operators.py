"""Rest-state curvature operators (oracle; test infrastructure only).

Everything is float64 and vectorised over a leading stencil axis S; each formula is written once, in the
paper's notation, for one stencil.

Readings of the paper used here (the CUDA library implements the same readings independently):

* Signed feet. Eq. 6-7, Eq. 10 and Eq. 78 weight the hinge end points with unsigned ratios
  |X_P3|/|X_23|. For an obtuse triangle the foot P lies outside the hinge edge and the unsigned ratio no
  longer reproduces the foot, so affine displacements would bend. We use the signed barycentric
  coordinate s_p = (X_1 - X_2).(X_3 - X_2) / |X_23|^2 that App. B (after Eq. 71) defines, so the foot is
  P = (1 - s_p) X_2 + s_p X_3 exactly: |X_P3|/|X_23| -> 1 - s_p and |X_P2|/|X_23| -> s_p.
* Heights h_i are distances in the rest triangles (Eq. 4 says they are taken in the initial
  configuration).
* Triangle-stencil 2D coordinates (C_p, R) are the rest positions expressed in the initial corotational
  frame of App. A (origin X_1, x axis along X_12, z axis the rest normal of the central triangle), with
  the out-of-plane coordinate dropped.
* R (Eq. 34, Eq. 38): (m_s, m_t) of hinge i are the components of the outward unit normal of the central
  edge opposite vertex i in those 2D axes.
* D_b in Voigt order (kappa_xx, kappa_yy, 2 kappa_xy) with D_b = k_b [[1, nu, 0], [nu, 1, 0],
  [0, 0, (1 - nu)/2]], k_b = E t^3 / (12 (1 - nu^2)) (Section 3 Eq. 1, Section 4.3 after Eq. 16).
* Clamped edge stencil (Eq. 30-31): L_m built with the virtual node L' = M + N - L, then column 4 folded
  into column 1 (w_L' = w_L). Its stencil area is the area of the one real triangle (reading: the
  virtual triangle is not part of the surface).
"""
from __future__ import annotations

import numpy as np

from .topology import HINGE_EDGE, INTERIOR, FREE, CLAMPED


# ------------------------------------------------------------------ small batched helpers
def dot(a, b):
    return np.sum(a * b, axis=-1)


def norm(a):
    return np.sqrt(dot(a, a))


def tri_area(a, b, c):
    return 0.5 * norm(np.cross(b - a, c - a))


def height_and_foot(xv, xa, xb):
    """Distance h of xv from the line xa-xb and the signed foot coordinate s (foot = xa + s (xb - xa))."""
    e = xb - xa
    s = dot(xv - xa, e) / dot(e, e)
    foot = xa + s[..., None] * e
    return norm(xv - foot), s


# ------------------------------------------------------------------ material
def bending_rigidity(E, nu, t):
    """k_b = E t^3 / (12 (1 - nu^2)) (Section 4.3, after Eq. 16)."""
    return E * t ** 3 / (12.0 * (1.0 - nu * nu))


def bending_D(E, nu, t):
    """Plane-stress bending stiffness D_b = t^3 E / 12 in Voigt order with engineering twist (Eq. 1)."""
    kb = bending_rigidity(E, nu, t)
    return kb * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]])


# ------------------------------------------------------------------ edge-based hinge (Section 4.3)
def edge_operator(X):
    """Corotational edge-based hinge curvature operator L_m = 2 L_theta / (h1 + h4) (Eq. 9-10).

    X: [S,4,3] rest positions (x1, x2, x3, x4). Returns (L_m [S,4], area A_E [S] = A_123 + A_432).
    """
    x1, x2, x3, x4 = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    h1, sp = height_and_foot(x1, x2, x3)
    h4, sq = height_and_foot(x4, x2, x3)
    L_theta = np.stack([1.0 / h1,
                        -((1.0 - sp) / h1 + (1.0 - sq) / h4),
                        -(sp / h1 + sq / h4),
                        1.0 / h4], axis=1)
    L_m = (2.0 / (h1 + h4))[:, None] * L_theta
    area = tri_area(x1, x2, x3) + tri_area(x4, x3, x2)
    return L_m, area


def edge_clamped_operator(X):
    """Clamped boundary edge stencil L-M-N-L' (Eq. 30-31).

    X: [S,3,3] rest positions of (L, M, N). Returns (L'_m [S,4] with a zero 4th column, area [S]).
    """
    L, M, N = X[:, 0], X[:, 1], X[:, 2]
    X4 = np.stack([L, M, N, M + N - L], axis=1)
    L_m, _ = edge_operator(X4)
    L_m = L_m.copy()
    L_m[:, 0] += L_m[:, 3]
    L_m[:, 3] = 0.0
    return L_m, tri_area(L, M, N)


# ------------------------------------------------------------------ triangle-centred stencils
def rest_frame(X):
    """Initial corotational frame of a triangle stencil (App. A Eq. 65): origin X_1, x along X_12, z along
    X_12 x X_13, y = z x x. Returns (ex, ey, ez) each [S,3]."""
    e12 = X[:, 1] - X[:, 0]
    e13 = X[:, 2] - X[:, 0]
    ex = e12 / norm(e12)[:, None]
    ez = np.cross(e12, e13)
    ez = ez / norm(ez)[:, None]
    ey = np.cross(ez, ex)
    return ex, ey, ez


def local_2d(X):
    """Rest stencil positions in the initial corotational frame, out-of-plane part dropped: [S,6,2]."""
    ex, ey, _ = rest_frame(X)
    d = X - X[:, :1]
    return np.stack([dot(d, ex[:, None]), dot(d, ey[:, None])], axis=-1)


def directional_operator(X):
    """Directional curvature operator L_p = -H theta (App. C Eq. 76-78), signed feet. X: [S,6,3].

    Row i (hinge across the central edge a_i-b_i opposite vertex i, neighbour i+3) is
    -(2 / (h_i + h_{i+3})) * theta_i with theta_i = -w_i/h_i - w_{i+3}/h_{i+3}
    + ((1 - s_i)/h_i + (1 - s_{i+3})/h_{i+3}) w_a + (s_i/h_i + s_{i+3}/h_{i+3}) w_b.
    """
    S = X.shape[0]
    Lp = np.zeros((S, 3, 6))
    for i, (a, b) in enumerate(HINGE_EDGE):
        hi, si = height_and_foot(X[:, i], X[:, a], X[:, b])
        hn, sn = height_and_foot(X[:, i + 3], X[:, a], X[:, b])
        theta = np.zeros((S, 6))
        theta[:, i] = -1.0 / hi
        theta[:, i + 3] = -1.0 / hn
        theta[:, a] = (1.0 - si) / hi + (1.0 - sn) / hn
        theta[:, b] = si / hi + sn / hn
        Lp[:, i, :] = -(2.0 / (hi + hn))[:, None] * theta
    return Lp


def transform_R(X):
    """FVM transform R (Eq. 38): column i = ((m_s)^2, (m_t)^2, 2 m_s m_t) of the outward unit normal of
    the central edge opposite vertex i, in the 2D rest frame."""
    P = local_2d(X)
    S = X.shape[0]
    R = np.zeros((S, 3, 3))
    for i, (a, b) in enumerate(HINGE_EDGE):
        t = P[:, b] - P[:, a]
        t = t / norm(t)[:, None]
        m = np.stack([t[:, 1], -t[:, 0]], axis=1)  # outward for a counter-clockwise triangle
        R[:, 0, i] = m[:, 0] ** 2
        R[:, 1, i] = m[:, 1] ** 2
        R[:, 2, i] = 2.0 * m[:, 0] * m[:, 1]
    return R


def quadratic_fit_matrix(X):
    """C_p (Eq. 49): row j = (X_j^2/2, Y_j^2/2, X_j Y_j/2) in the 2D rest frame. Returns [S,6,3]."""
    P = local_2d(X)
    x, y = P[..., 0], P[..., 1]
    return np.stack([0.5 * x * x, 0.5 * y * y, 0.5 * x * y], axis=-1)


def smoothed_operator(Lp, Cp):
    """Smoothed hinge operator L_g = (L_p C_p)^-1 L_p (Eq. 50)."""
    return np.linalg.solve(Lp @ Cp, Lp)


def fold_boundary(L, bc):
    """Condense virtual neighbour columns (Eq. 58-61). L: [S,r,6]; bc: [S,3] per hinge.

    Clamped hinge i (Eq. 59, w_L' = w_L): column i+3 is added to column i.
    Free hinge i (Eq. 60-61, w_L' = w_M + w_N - w_L): column i+3 is added to the columns of the edge end
    points a_i, b_i and subtracted from column i. Several boundary edges superimpose.
    """
    L = L.copy()
    for i, (a, b) in enumerate(HINGE_EDGE):
        c = L[:, :, i + 3].copy()
        cl = bc[:, i] == CLAMPED
        fr = bc[:, i] == FREE
        L[cl, :, i] += c[cl]
        L[fr, :, a] += c[fr]
        L[fr, :, b] += c[fr]
        L[fr, :, i] -= c[fr]
        L[(cl | fr), :, i + 3] = 0.0
    return L


def triangle_stencil_operators(X, bc, family, D_b):
    """Rest-state operator of triangle stencils for one hinge family.

    X: [S,6,3] rest positions with virtual nodes; bc: [S,3]; family 'F' (FVM hinge) or 'S' (smoothed).
    Returns (L [S,3,6] folded, Dmat [S,3,3], area [S]) such that the plate energy is
    (area/2) sum_c (L x_c)^T Dmat (L x_c):

    * FVM hinge: L = L_p, Dmat = R^T D_b R (Eq. 39-41). On stencils with a free edge the twist row of R
      is zeroed (Section 4.4, boundary conditions: mixed second derivative set to zero).
    * Smoothed hinge: L = L_g, Dmat = D_b (Eq. 52-53).
    """
    Lp = directional_operator(X)
    area = tri_area(X[:, 0], X[:, 1], X[:, 2])
    if family == "F":
        L = fold_boundary(Lp, bc)
        R = transform_R(X)
        has_free = np.any(bc == FREE, axis=1)
        R[has_free, 2, :] = 0.0
        Dmat = np.einsum("sji,jk,skl->sil", R, D_b, R)
    elif family == "S":
        Lg = smoothed_operator(Lp, quadratic_fit_matrix(X))
        L = fold_boundary(Lg, bc)
        Dmat = np.broadcast_to(D_b, (X.shape[0], 3, 3)).copy()
    else:
        raise ValueError(family)
    return L, Dmat, area
