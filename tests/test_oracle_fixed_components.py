"""Pins of the oracle's per-component constraints (Section 6.1, hemisphere: x fixed on the nodes of the y-z
plane, y on those of the x-z plane, z as well on the hole's edge in the y-z plane) against facts that do not
come from the oracle's own constraint handling:

* the linearised step with fixed components equals the solution of the system with those rows and columns
  deleted (elimination, dense solve), the textbook form of a Dirichlet condition;
* the quasi-static solve of a coarse hemisphere ends at the minimiser of the total potential over the free
  components (L-BFGS from the rest shape);
* the hemisphere's mesh, loads and constraints are symmetric under x -> -x and y -> -y, so for a model whose
  energy is mirror-invariant (ES, FS) the equilibrium is symmetric and the symmetry constraints carry no
  reaction: f + f_ext vanishes at the fixed components too. A constraint on the wrong component (a swapped
  bit) carries one.
* the smoothed-hinge operator (Eq. 49-50) is not mirror-invariant on a curved stencil: its quadratic fit is
  centred at the frame origin X_1 (App. A), and there the directional operator does not annihilate linear
  functions of the projected coordinates, so SS carries reactions at the symmetry constraints.
"""
import dataclasses

import numpy as np
import pytest
import scipy.optimize
from scipy.spatial import cKDTree

import shellgen as sg
from oracle import newton as nw
from oracle import operators as op
from oracle import system as osys


def coarse(model, load=20.0, n_around=16, n_rings=5):
    return sg.hemisphere(model, n_around=n_around, n_rings=n_rings, load=load)


def test_bits_and_pinned():
    sc = coarse("ES")
    fd = sc.fixed_dofs.copy()
    fd[5] = 7
    m = osys.build_model(sc.tris, sc.rest, "ES", sc.E, sc.nu, sc.thickness, sc.density, sc.dt,
                         fixed_dofs=fd, factor=False)
    assert m.pinned[5] and m.pinned.sum() == 1
    assert np.array_equal(m.fixed[:, 0], (fd & 1) > 0) and np.array_equal(m.fixed[:, 2], (fd & 4) > 0)
    assert m.partial


@pytest.mark.parametrize("model", ["ES", "SS"])
def test_step_with_fixed_components_equals_elimination(model):
    sc = dataclasses.replace(coarse(model), dt=1e-3)
    m = osys.from_scenario(sc)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(sc.rest.shape)
    x = sc.rest + 0.01 * rng.standard_normal(sc.rest.shape)
    _, vn = osys.step(m, x, v, 1)
    Kb, Km = osys.stiffness_matrices(m)
    A3 = np.kron(np.diag(m.mass) + m.dt ** 2 * (Kb + Km).toarray(), np.eye(3))
    b = (m.mass[:, None] * v + m.dt * (osys.forces(m, x) + m.f_ext)).ravel()
    free = ~m.fixed.ravel()
    ve = np.zeros(A3.shape[0])
    ve[free] = np.linalg.solve(A3[np.ix_(free, free)], b[free])
    np.testing.assert_allclose(vn.ravel(), ve, rtol=0, atol=1e-10 * np.abs(ve).max())
    assert np.all(vn[m.fixed] == 0.0)


@pytest.mark.parametrize("model", ["ES", "SS"])
def test_static_hemisphere_reaches_the_energy_minimiser(model):
    sc = coarse(model, n_around=12, n_rings=4)
    m = osys.from_scenario(sc, factor=False)
    x, it, nr = nw.solve_static(m, sc.rest, eps_f=1e-7, eps_u=0.1, max_iters=400)
    assert nr < 1e-7 and np.all(x[m.fixed] == sc.rest[m.fixed])
    free = ~m.fixed

    def fun(z):
        xx = sc.rest.copy()
        xx[free] = z
        e = osys.membrane_energy(m, xx) + osys.bending_energy(m, xx) - float(np.sum(m.f_ext * xx))
        return e, -nw.static_residual(m, xx)[free]

    res = scipy.optimize.minimize(fun, sc.rest[free], jac=True, method="L-BFGS-B",
                                  options={"maxiter": 50000, "ftol": 1e-16, "gtol": 1e-10})
    xmin = sc.rest.copy()
    xmin[free] = res.x
    assert np.linalg.norm(x - xmin) <= 2e-5 * np.linalg.norm(x - sc.rest)


def _mirror_index(X, axis):
    Y = X.copy()
    Y[:, axis] *= -1.0
    d, idx = cKDTree(X).query(Y)
    assert d.max() < 1e-9
    return idx


@pytest.mark.parametrize("model", ["ES", "FS"])
def test_symmetry_constraints_carry_no_reaction(model):
    sc = coarse(model)
    m = osys.from_scenario(sc, factor=False)
    x, _, _ = nw.solve_static(m, sc.rest, eps_f=1e-8, eps_u=0.1, max_iters=400)
    full = osys.forces(m, x) + m.f_ext               # reactions included: not masked
    assert np.abs(full).max() <= 1e-8 * 20.0 * 10
    u = x - sc.rest
    for axis in (0, 1):
        idx = _mirror_index(sc.rest, axis)
        um = u[idx].copy()
        um[:, axis] *= -1.0
        assert np.abs(um - u).max() <= 1e-9 * np.abs(u).max()
    # the same solve with bits 0 and 1 swapped constrains the components that move: reactions appear
    fd = sc.fixed_dofs.copy()
    fd = (fd & 4) | ((fd & 1) << 1) | ((fd & 2) >> 1)
    m2 = osys.build_model(sc.tris, sc.rest, model, sc.E, sc.nu, sc.thickness, sc.density, sc.dt,
                          load_vtx=sc.load_vtx, load_f=sc.load_f, fixed_dofs=fd, factor=False)
    x2, _, _ = nw.solve_static(m2, sc.rest, eps_f=1e-8, eps_u=0.1, max_iters=400)
    assert np.abs(osys.forces(m2, x2) + m2.f_ext).max() > 1e-2 * 20.0


def test_smoothed_hinge_depends_on_the_frame_origin_on_curved_stencils():
    rng = np.random.default_rng(1)
    D = op.bending_D(1.0, 0.3, 1.0)
    perm = [1, 0, 2, 4, 3, 5]   # mirror image relabelled: vertices 1 <-> 2 (the origin moves), hinges alike
    for curved, invariant in ((False, True), (True, False)):
        X = np.array([[10.0, 0, 0], [9.2388, 3.8268, 0], [9.0369, 3.7432, 2.0791], [6.9165, 6.9165, 2.0791],
                      [9.7815, 0, 2.0791], [0, 0, 0]])
        X[5] = X[0] + X[1] - X[2]
        if not curved:   # flatten onto the triangle's plane
            n = np.cross(X[1] - X[0], X[2] - X[0])
            n /= np.linalg.norm(n)
            X = X - np.outer((X - X[0]) @ n, n)
        Xm = X.copy()
        Xm[:, 0] *= -1.0
        Xm = Xm[perm]
        w = rng.standard_normal(6)
        for fam in "FS":
            L0, D0, A0 = op.triangle_stencil_operators(X[None], np.zeros((1, 3), int), fam, D)
            L1, D1, A1 = op.triangle_stencil_operators(Xm[None], np.zeros((1, 3), int), fam, D)
            e0 = A0[0] * (L0[0] @ w) @ D0[0] @ (L0[0] @ w)
            e1 = A1[0] * (L1[0] @ w[perm]) @ D1[0] @ (L1[0] @ w[perm])
            same = abs(e0 - e1) <= 1e-12 * abs(e0)
            assert same == (invariant or fam == "F"), (curved, fam, e0, e1)
    # and so SS carries reactions at the hemisphere's symmetry constraints
    sc = coarse("SS")
    m = osys.from_scenario(sc, factor=False)
    x, _, _ = nw.solve_static(m, sc.rest, eps_f=1e-8, eps_u=0.1, max_iters=400)
    assert np.abs(osys.forces(m, x) + m.f_ext).max() > 1e-2
