"""Pins of the oracle's rest-state operators against properties the paper's construction fixes.

* Every curvature operator annihilates constants and affine functions of the rest tangent plane
  (zero curvature of a flat or rigidly moved stencil; Section 4.2 remarks, Eq. 12), including obtuse
  stencils (signed feet) and after the free-edge fold (Eq. 60-61).
* The smoothed hinge operator inverts the quadratic fit: L_g C_p = I_3 (Eq. 49-50).
* The clamped edge operator equals the printed Eq. 31 on an acute stencil.
* For an FVM hinge with a free edge the fold makes that hinge's directional curvature vanish.
"""
import numpy as np
import pytest

from oracle import operators as op
from oracle.topology import FREE, CLAMPED, INTERIOR, HINGE_EDGE, build_stencils

RNG = np.random.default_rng(12)


def random_flat_tri_stencils(S, obtuse=False, tilt=True):
    """Random triangle-centred stencils lying in a random plane: [S,6,3] and the plane's (u, v) axes."""
    P = np.zeros((S, 6, 2))
    P[:, 0] = [0.0, 0.0]
    P[:, 1] = [1.0, 0.0]
    P[:, 2] = RNG.uniform([0.2, 0.5], [0.8, 1.2], size=(S, 2))
    if obtuse:
        P[:, 2, 0] = RNG.uniform(1.3, 1.8, size=S)     # obtuse angle at vertex 2
        P[:, 2, 1] = RNG.uniform(0.2, 0.4, size=S)
    for i, (a, b) in enumerate(HINGE_EDGE):
        # neighbour on the far side of the hinge edge (a valid, non-inverted neighbour triangle)
        mid = 0.5 * (P[:, a] + P[:, b])
        alpha = RNG.uniform(0.6, 1.4, size=(S, 1))
        beta = RNG.uniform(-0.3, 0.3, size=(S, 1))
        P[:, 3 + i] = mid + alpha * (mid - P[:, i]) + beta * (P[:, b] - P[:, a])
    # random rigid placement in 3D
    Q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    u, v = Q[:, 0], Q[:, 1]
    X = P[..., :1] * u + P[..., 1:] * v + RNG.standard_normal(3)
    return X, P, u, v


@pytest.mark.parametrize("obtuse", [False, True])
def test_edge_operator_kills_affine(obtuse):
    X, P, u, v = random_flat_tri_stencils(64, obtuse)
    E4 = X[:, [0, 1, 2, 3]]   # wing 1 = vertex 1, hinge 2-3, wing 4 across it
    L, area = op.edge_operator(E4)
    assert np.all(area > 0)
    assert np.max(np.abs(L.sum(axis=1))) < 1e-12 * np.abs(L).max()
    for f in (lambda x: x @ u, lambda x: x @ v, lambda x: 3.0 * (x @ u) - 2.0 * (x @ v) + 1.5):
        w = f(E4)
        assert np.max(np.abs(np.sum(L * w, axis=1))) < 1e-11 * np.abs(L).max()


def test_edge_operator_unsigned_form_on_acute_stencil():
    """On an acute stencil, where feet fall inside the hinge, the signed-feet operator equals Eq. 10."""
    X = np.array([[[0.4, 0.9, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.6, -0.7, 0.0]]])
    L, _ = op.edge_operator(X)
    x1, x2, x3, x4 = X[0]
    P = np.array([0.4, 0.0, 0.0])
    Q = np.array([0.6, 0.0, 0.0])
    h1, h4, e = 0.9, 0.7, 1.0
    n = np.linalg.norm
    Lt = [1 / h1, -(n(P - x3) / (e * h1) + n(Q - x3) / (e * h4)), -(n(P - x2) / (e * h1) + n(Q - x2) / (e * h4)),
          1 / h4]
    np.testing.assert_allclose(L[0], 2.0 / (h1 + h4) * np.array(Lt), rtol=1e-14)


def test_clamped_edge_operator_matches_eq31():
    X3 = np.array([[[0.3, 0.8, 0.0], [0.0, 0.0, 0.0], [1.2, 0.0, 0.0]]])   # L, M, N
    L, area = op.edge_clamped_operator(X3)
    h1 = 0.8
    c = 1.2
    P = np.array([0.3, 0.0, 0.0])
    Qr = np.array([1.2 - 0.3, 0.0, 0.0])  # foot of the reflected node L' = M + N - L
    n = np.linalg.norm
    x2, x3 = X3[0, 1], X3[0, 2]
    expect = (1 / h1) * np.array([2 / h1, -(n(P - x3) + n(Qr - x3)) / (c * h1), -(n(P - x2) + n(Qr - x2)) / (c * h1), 0])
    np.testing.assert_allclose(L[0], expect, rtol=1e-14)
    assert area[0] == pytest.approx(0.5 * 1.2 * 0.8)


@pytest.mark.parametrize("obtuse", [False, True])
def test_directional_and_smoothed_operators_kill_affine(obtuse):
    X, P, u, v = random_flat_tri_stencils(64, obtuse)
    Lp = op.directional_operator(X)
    Lg = op.smoothed_operator(Lp, op.quadratic_fit_matrix(X))
    for L in (Lp, Lg):
        scale = np.abs(L).max()
        for f in (lambda x: np.ones(x.shape[:-1]), lambda x: x @ u, lambda x: x @ v):
            w = f(X)
            assert np.max(np.abs(np.einsum("srk,sk->sr", L, w))) < 1e-10 * scale


def test_smoothed_operator_inverts_quadratic_fit():
    X, *_ = random_flat_tri_stencils(64)
    Lp = op.directional_operator(X)
    Cp = op.quadratic_fit_matrix(X)
    Lg = op.smoothed_operator(Lp, Cp)
    np.testing.assert_allclose(Lg @ Cp, np.broadcast_to(np.eye(3), (64, 3, 3)), atol=1e-10)


def test_smoothed_operator_exact_on_quadratic():
    """L_g d = (c4, c5, c6) for d = c1 + c2 X + c3 Y + c4 X^2/2 + c5 Y^2/2 + c6 XY/2 in the rest frame (Eq. 48)."""
    X, *_ = random_flat_tri_stencils(32)
    P = op.local_2d(X)
    c = RNG.standard_normal((32, 6))
    x, y = P[..., 0], P[..., 1]
    d = (c[:, :1] + c[:, 1:2] * x + c[:, 2:3] * y + c[:, 3:4] * x * x / 2 + c[:, 4:5] * y * y / 2
         + c[:, 5:6] * x * y / 2)
    Lg = op.smoothed_operator(op.directional_operator(X), op.quadratic_fit_matrix(X))
    np.testing.assert_allclose(np.einsum("srk,sk->sr", Lg, d), c[:, 3:], atol=1e-9)


def test_free_fold_keeps_affine_and_zeroes_fvm_hinge():
    X, P, u, v = random_flat_tri_stencils(16)
    for i, (a, b) in enumerate(HINGE_EDGE):
        bc = np.zeros((16, 3), np.int8)
        bc[:, i] = FREE
        Xv = X.copy()
        Xv[:, 3 + i] = X[:, a] + X[:, b] - X[:, i]          # virtual node
        Lp = op.directional_operator(Xv)
        Lf = op.fold_boundary(Lp, bc)
        assert np.all(Lf[:, :, 3 + i] == 0.0)
        assert np.max(np.abs(Lf[:, i, :])) < 1e-12 * np.abs(Lp).max()    # theta_i == 0 after the free fold
        for f in (lambda x: x @ u, lambda x: x @ v):
            w = f(Xv)
            assert np.max(np.abs(np.einsum("srk,sk->sr", Lf, w))) < 1e-10 * np.abs(Lp).max()
        Lg = op.fold_boundary(op.smoothed_operator(Lp, op.quadratic_fit_matrix(Xv)), bc)
        for f in (lambda x: x @ u, lambda x: x @ v):
            assert np.max(np.abs(np.einsum("srk,sk->sr", Lg, f(Xv)))) < 1e-9 * np.abs(Lg).max()


def test_clamped_fold_keeps_constants():
    X, *_ = random_flat_tri_stencils(16)
    bc = np.zeros((16, 3), np.int8)
    bc[:, 1] = CLAMPED
    Lc = op.fold_boundary(op.directional_operator(X), bc)
    assert np.max(np.abs(Lc.sum(axis=2))) < 1e-12 * np.abs(Lc).max()
    np.testing.assert_array_equal(Lc[:, :, 4], 0.0)


def test_R_maps_directional_to_generalised_curvature():
    """For a uniform curvature tensor K, the directional curvature across the edge with outward normal m is
    m^T K m; R^T (K_xx, K_yy, K_xy) reproduces those three values (Eq. 36-38, the FVM superposition
    written as a map from generalised to directional curvature)."""
    X, *_ = random_flat_tri_stencils(8)
    R = op.transform_R(X)
    P = op.local_2d(X)
    K = RNG.standard_normal((8, 2, 2))
    K = K + np.swapaxes(K, 1, 2)
    for i, (a, b) in enumerate(HINGE_EDGE):
        t = P[:, b] - P[:, a]
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        m = np.stack([t[:, 1], -t[:, 0]], 1)
        kn = np.einsum("si,sij,sj->s", m, K, m)
        kvec = np.stack([K[:, 0, 0], K[:, 1, 1], K[:, 0, 1]], 1)
        np.testing.assert_allclose(np.einsum("sr,sr->s", R[:, :, i], kvec), kn, rtol=1e-12, atol=1e-12)
        # outward: the normal points away from the opposite vertex
        assert np.all(np.einsum("si,si->s", m, P[:, i] - P[:, a]) < 0)


def test_topology_counts_and_relabel():
    import shellgen as sg
    xy, tris = sg.grid(4, 3)
    topo = build_stencils(tris, xy.shape[0], sg.grid_side_edges(4, 3, "x0"))
    nx, ny = 4, 3
    n_edges = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    n_boundary = 2 * (nx + ny)
    assert len(topo["edge"]) == n_edges - n_boundary
    assert len(topo["edge_clamped"]) == ny
    assert len(topo["tri"]) == len(tris)
    # every free boundary hinge is hinge 3 (edge 1->2) after relabelling when it is the only free one
    bc = topo["tri_bc"]
    nfree = np.sum(bc == FREE, axis=1)
    assert np.all(bc[nfree >= 1, 2] == FREE)
    for k in range(3):
        assert np.all((topo["tri"][:, 3 + k] < 0) == (bc[:, k] != INTERIOR))


def test_topology_rejects_bad_orientation():
    tris = np.array([[0, 1, 2], [1, 2, 3]])     # shared edge traversed the same way twice
    with pytest.raises(ValueError):
        build_stencils(tris, 4)
