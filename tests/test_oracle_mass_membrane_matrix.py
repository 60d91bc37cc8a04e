"""Pins of the oracle's lumped mass and constant membrane matrix against closed forms.

* Lumped mass (m_i = sum over incident triangles of rho t A / 3; the paper gives no mass matrix, Section 5):
  the masses of a flat mesh add up to rho t times its area, known here from the geometry alone (a unit
  square, jittered inside or not), and on the regular right-triangle grid a vertex carries rho t s^2 times
  (incident triangles) / 6: s^2 inside (six triangles), s^2 / 3 at the corners on the split diagonal, s^2 / 6
  at the other two corners, s^2 / 2 on the sides.
* Constant membrane block (2 (mu + lam) A t grad(phi_a).grad(phi_b) (x) I_3 per triangle; reading of the
  membrane term, Section 3): for a displacement u(X) = G X linear in the rest coordinates, the hat functions
  reproduce u exactly, so u^T K_m u = 2 (mu + lam) t |G|_F^2 times the mesh area, on any mesh; the rows of
  interior vertices of K_m u vanish (patch test); and the weight is the smallest that bounds the membrane
  Hessian: an equibiaxial linear field attains the bound (u^T K_m u equals the second derivative of the
  membrane energy along u), a uniaxial one stays strictly below it.
"""
import numpy as np
import pytest

import shellgen as sg
from oracle import system as osys
from oracle.energies import lame

E, NU, T, RHO = 2.0e6, 0.3, 2e-3, 750.0


def _plate(n, jitter_amount=0.0, seed=3):
    xy, tris = sg.grid(n, n)
    if jitter_amount:
        xy = sg.jitter(xy, 1.0 / n, jitter_amount, sg.grid_interior_mask(n, n), seed)
    return xy, tris, sg.flat3(xy)


@pytest.mark.parametrize("jit", [0.0, 0.2])
def test_lumped_mass_sums_to_rho_t_area(jit):
    n = 9
    xy, tris, rest = _plate(n, jit)
    m = osys.build_model(tris, rest, "EP", E, NU, T, RHO, 1e-2, factor=False)
    # the jitter moves interior vertices only: the mesh still tiles the unit square, area 1
    assert m.mass.sum() == pytest.approx(RHO * T * 1.0, rel=1e-13)


def test_lumped_mass_per_vertex_on_regular_grid():
    n = 8
    s = 1.0 / n
    xy, tris, rest = _plate(n)
    m = osys.build_model(tris, rest, "SP", E, NU, T, RHO, 1e-2, factor=False)
    unit = RHO * T * s * s
    mass = m.mass.reshape(n + 1, n + 1)   # vertex index j * (n + 1) + i (row j along y)
    interior = mass[1:-1, 1:-1]
    np.testing.assert_allclose(interior, unit, rtol=1e-13)
    # corners: (0,0) and (1,1) lie on the split diagonal of their cell (two triangles), the others have one
    corners = {(0, 0): 2, (n, n): 2, (0, n): 1, (n, 0): 1}
    for (j, i), k in corners.items():
        assert mass[j, i] == pytest.approx(unit * k / 6.0, rel=1e-13), (j, i)
    # non-corner side vertices have three incident triangles
    sides = np.concatenate([mass[0, 1:-1], mass[-1, 1:-1], mass[1:-1, 0], mass[1:-1, -1]])
    np.testing.assert_allclose(sides, unit * 0.5, rtol=1e-13)


def _membrane_matrix(tris, rest):
    m = osys.build_model(tris, rest, "EP", E, NU, T, RHO, 1e-2, factor=False)
    _, Km = osys.stiffness_matrices(m)
    return m, Km


@pytest.mark.parametrize("jit", [0.0, 0.2])
def test_membrane_matrix_energy_of_linear_field(jit):
    n = 7
    xy, tris, rest = _plate(n, jit, seed=5)
    _, Km = _membrane_matrix(tris, rest)
    mu, lam = lame(E, NU)
    rng = np.random.default_rng(11)
    for _ in range(3):
        G = rng.standard_normal((3, 2))
        u = xy @ G.T                                  # [V,3], u(X) = G X
        quad = float(np.einsum("vc,vw,wc->", u, Km.toarray(), u))
        expect = 2.0 * (mu + lam) * T * 1.0 * float(np.sum(G * G))   # area of the unit square
        assert quad == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("jit", [0.0, 0.2])
def test_membrane_matrix_patch_test(jit):
    n = 7
    xy, tris, rest = _plate(n, jit, seed=8)
    _, Km = _membrane_matrix(tris, rest)
    G = np.random.default_rng(2).standard_normal((3, 2))
    u = xy @ G.T
    y = Km @ u
    interior = sg.grid_interior_mask(n, n)
    scale = np.abs(Km).max() * np.abs(u).max()
    assert np.abs(y[interior]).max() < 1e-12 * scale
    assert np.abs(y[~interior]).max() > 1e-3 * scale    # boundary rows carry the traction


def _second_derivative_of_membrane_energy(m, u, h=1e-4):
    x0 = m.rest
    e = [osys.membrane_energy(m, x0 + k * h * u) for k in (-2, -1, 0, 1, 2)]
    # fourth-order central difference
    return (-e[0] + 16 * e[1] - 30 * e[2] + 16 * e[3] - e[4]) / (12 * h * h)


def test_membrane_weight_is_attained_by_equibiaxial_and_bounds_uniaxial():
    n = 6
    xy, tris, rest = _plate(n, 0.2, seed=4)
    m, Km = _membrane_matrix(tris, rest)
    K = Km.toarray()
    # equibiaxial in-plane stretch: |e|^2 = |grad u|^2 / 1 and (tr e)^2 = 2 |e|^2, the bound holds with equality
    u = np.zeros_like(rest)
    u[:, :2] = xy
    d2 = _second_derivative_of_membrane_energy(m, u)
    quad = float(np.einsum("vc,vw,wc->", u, K, u))
    assert quad == pytest.approx(d2, rel=1e-6)
    # uniaxial stretch: the energy's curvature is (2 mu + lam) t A |G|^2, below 2 (mu + lam) t A |G|^2
    u = np.zeros_like(rest)
    u[:, 0] = xy[:, 0]
    d2 = _second_derivative_of_membrane_energy(m, u)
    quad = float(np.einsum("vc,vw,wc->", u, K, u))
    mu, lam = lame(E, NU)
    assert d2 == pytest.approx((2 * mu + lam) * T, rel=1e-6)
    assert quad == pytest.approx(2 * (mu + lam) * T, rel=1e-12)
    assert quad > d2 * (1 + 1e-3)
