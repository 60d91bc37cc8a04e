"""Pins of the oracle's energies, forces, matrix and step against invariants and finite differences.

* Forces are exact negative gradients: central differences of the total energy on small meshes in
  random non-planar states, for all six models, every boundary type and the membrane.
* Rigid motions: energy unchanged, forces rotate with the body, net force and net torque vanish; the rest
  state is force free.
* The plate force equals -K_b x (Eq. 21-22); the matrix is symmetric positive semi-definite and its
  null space for a free flat plate contains {1, X, Y} (x) I_3.
* Integrator: a free unconstrained mesh falls exactly as v_n = n dt g, x_n = x_0 + dt^2 g n(n+1)/2; for a
  plate without membrane one eigenmode of M^-1 K decays by exactly 1/(1 + dt^2 omega^2) per step
  (backward Euler, Eq. 62-63, is exact for a linear force).
"""
import numpy as np
import pytest

import shellgen as sg
from oracle import system as osys
from oracle.energies import FIXED

RNG = np.random.default_rng(3)
MODELS = sg.MODELS


def small_scene(model, bc):
    n = 4
    if model in sg.SHELL_MODELS:
        sc = sg.cylinder_panel(n, model, radius=0.7, load=0.0)
        rest = sc.rest
        tris = sc.tris
        xy = None
    else:
        xy, tris = sg.grid(n, n)
        rest = sg.flat3(xy)
    clamped = sg.grid_side_edges(n, n, "x0") if bc == "clamped" else np.zeros((0, 2), np.int32)
    return rest, tris, clamped


def total_energy(m, x):
    a, b, _, _ = osys.energy(m, x, np.zeros_like(x))
    return a + b


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("bc", ["free", "clamped"])
def test_force_is_negative_gradient(model, bc):
    rest, tris, clamped = small_scene(model, bc)
    m = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2, clamped_edges=clamped, factor=False)
    x = rest + 0.03 * RNG.standard_normal(rest.shape)
    f = osys.forces(m, x)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd[i, c] = -(total_energy(m, xp) - total_energy(m, xm)) / (2 * h)
    assert np.abs(fd - f).max() < 1e-7 * np.abs(f).max()


@pytest.mark.parametrize("model", MODELS)
def test_rigid_motion_invariance(model):
    rest, tris, _ = small_scene(model, "free")
    m = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2, factor=False)
    np.testing.assert_allclose(osys.forces(m, rest), 0.0, atol=1e-9)
    x = rest + 0.05 * RNG.standard_normal(rest.shape)
    Q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    xr = x @ Q.T + RNG.standard_normal(3)
    e0, e1 = total_energy(m, x), total_energy(m, xr)
    assert e1 == pytest.approx(e0, rel=1e-11)
    f0, f1 = osys.forces(m, x), osys.forces(m, xr)
    np.testing.assert_allclose(f1, f0 @ Q.T, atol=1e-9 * np.abs(f0).max())
    assert np.abs(f0.sum(axis=0)).max() < 1e-9 * np.abs(f0).max()
    torque = np.cross(x, f0).sum(axis=0)
    assert np.abs(torque).max() < 1e-9 * np.abs(f0).max()


@pytest.mark.parametrize("model", ["EP", "FP", "SP"])
def test_plate_force_is_constant_hessian_times_x(model):
    xy, tris = sg.grid(5, 5)
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2, membrane=False,
                         clamped_edges=sg.grid_side_edges(5, 5, "y0"), factor=False)
    Kb, _ = osys.stiffness_matrices(m)
    # clamped stencils measure along the fixed rest normal, so compare on transverse motion only
    x = rest.copy()
    x[:, 2] = 0.1 * RNG.standard_normal(rest.shape[0])
    f = osys.forces(m, x)
    np.testing.assert_allclose(f[:, 2], -(Kb @ x[:, 2]), atol=1e-10 * np.abs(f).max())
    # without clamped edges the (x) I_3 form holds for every coordinate
    m2 = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2, membrane=False, factor=False)
    Kb2, _ = osys.stiffness_matrices(m2)
    x = rest + 0.1 * RNG.standard_normal(rest.shape)
    np.testing.assert_allclose(osys.forces(m2, x), -(Kb2 @ x), atol=1e-10 * np.abs(Kb2 @ x).max())


@pytest.mark.parametrize("model", MODELS)
def test_matrix_symmetric_psd_and_null_space(model):
    xy, tris = sg.grid(5, 4)
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2, factor=False)
    Kb, Km = osys.stiffness_matrices(m)
    for K in (Kb, Km):
        K = K.toarray()
        np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
        w = np.linalg.eigvalsh(K)
        assert w.min() > -1e-10 * w.max()
    K = Kb.toarray()
    for field in (np.ones(rest.shape[0]), xy[:, 0], xy[:, 1]):
        assert np.abs(K @ field).max() < 1e-9 * np.abs(K).max()
    assert np.sum(np.linalg.eigvalsh(K) < 1e-9 * np.abs(K).max()) >= 3


def test_fixed_normal_stencils_only_on_clamped_boundaries():
    xy, tris = sg.grid(4, 4)
    rest = sg.flat3(xy)
    for model in MODELS:
        m = osys.build_model(tris, rest, model, 1e5, 0.3, 1e-2, 1.0, 1e-2,
                             clamped_edges=sg.grid_side_edges(4, 4, "x0"), factor=False)
        nfixed = sum(int(np.sum(st.mode == FIXED)) for st in m.stencils)
        assert nfixed == 4   # one clamped stencil per clamped boundary edge (edge hinge) or triangle


def test_free_fall_is_exact():
    for model in ("EP", "SS"):
        sc = sg.plate_clamped_x0(4, model=model)
        m = osys.build_model(sc.tris, sc.rest, model, 1e5, 0.3, 1e-3, 1000.0, 0.01, gravity=(0.0, -3.0, -9.81))
        g = np.array([0.0, -3.0, -9.81])
        x, v = osys.step(m, sc.rest, np.zeros_like(sc.rest), 7)
        n = 7
        np.testing.assert_allclose(v, np.broadcast_to(n * 0.01 * g, v.shape), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(x - sc.rest, np.broadcast_to(0.01 ** 2 * g * n * (n + 1) / 2, x.shape),
                                   rtol=1e-9, atol=1e-13)


def test_eigenmode_damping_without_membrane():
    xy, tris = sg.grid(4, 4)
    rest = sg.flat3(xy)
    pinned = ~sg.grid_interior_mask(4, 4)
    dt = 0.05
    m = osys.build_model(tris, rest, "SP", 1e5, 0.3, 1e-2, 1000.0, dt, pinned=pinned, membrane=False)
    Kb, _ = osys.stiffness_matrices(m)
    free = ~pinned
    K = Kb.toarray()[np.ix_(free, free)]
    Mf = m.mass[free]
    # generalised eigenproblem K u = w^2 M u via symmetric scaling
    S = np.diag(1.0 / np.sqrt(Mf))
    w2, U = np.linalg.eigh(S @ K @ S)
    k = len(w2) // 2
    u = S @ U[:, k]
    v0 = np.zeros_like(rest)
    v0[free, 2] = u
    x1, v1 = osys.step(m, rest, v0, 1)
    np.testing.assert_allclose(v1[free, 2], u / (1.0 + dt * dt * w2[k]), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(v1[:, :2], 0.0, atol=1e-14)
