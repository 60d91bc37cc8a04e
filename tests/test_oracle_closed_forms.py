"""Pins of the oracle against closed forms of Kirchhoff-Love plate/shell theory and the paper's printed
benchmark.

* A rest-flat plate deflected to the quadratic w = 1/2 X^T K X has KL energy density
  1/2 kappa^T D_b kappa with kappa = (K_xx, K_yy, 2 K_xy) (Section 3, Eq. 1-2).
  - Smoothed hinge (SP): exact on every interior stencil of any mesh (the fit is exact for quadratic
    surfaces, Eq. 48-50).
  - FVM hinge (FP): exact on every interior stencil of regular right-triangle and equilateral meshes.
  - Edge hinge (EP): derived per edge. On the right-triangle grid the hinge across a horizontal, vertical
    and diagonal edge measures K_yy + K_xy, K_xx + K_xy and -2 K_xy; on an equilateral mesh the hinge with
    in-plane edge normal m measures (4 m^T K m - tr K)/3. The energy is 1/2 k_b A_E kappa_m^2 (Eq. 16).
* Rest-flat shells bent onto a cylinder of radius R measure curvature 1/R; a cylinder of rest radius R0
  re-bent to R1 has energy proportional to (1/R1 - 1/R0)^2 (Eq. 2, Eq. 23-24, 42-43, 54-55).
* Timoshenko's simply supported square plate (Section 6.1): FP/SP converge to the analytic centre
  deflection on regular meshes and EP only on the equilateral mesh (golden fixtures).
* Membrane: uniaxial, equibiaxial and pure-rotation closed forms of the plane-stress linear membrane.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import shellgen as sg
from oracle import operators as op
from oracle import system as osys
from oracle.energies import lame, membrane_energy_force, membrane_rest, stencil_energy

E, NU, T = 1e6, 0.3, 1e-3
RNG = np.random.default_rng(7)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def quad_surface(xy, K):
    return 0.5 * np.einsum("vi,ij,vj->v", xy, K, xy)


def random_K():
    K = RNG.standard_normal((2, 2))
    return K + K.T


def tri_mesh(kind, n=10):
    if kind == "equilateral":
        return sg.equilateral_grid(n, n, 1.0 / n)
    xy, tris = sg.grid(n, n)
    if kind == "jittered":
        xy = sg.jitter(xy, 1.0 / n, 0.2, sg.grid_interior_mask(n, n), 11)
    return xy, tris


@pytest.mark.parametrize("model,mesh", [("SP", "regular"), ("SP", "jittered"), ("SP", "equilateral"),
                                        ("FP", "regular"), ("FP", "equilateral")])
def test_triangle_hinge_plate_matches_kl_per_stencil(model, mesh):
    xy, tris = tri_mesh(mesh)
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, model, E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    interior = np.all(st.idx >= 0, axis=1)
    D_b = op.bending_D(E, NU, T)
    area = op.tri_area(st.rest[:, 0], st.rest[:, 1], st.rest[:, 2])
    for _ in range(3):
        K = random_K()
        x = rest.copy()
        x[:, 2] = quad_surface(xy, K)
        kappa = np.array([K[0, 0], K[1, 1], 2 * K[0, 1]])
        dens = 0.5 * kappa @ D_b @ kappa
        e = stencil_energy(x, st)
        np.testing.assert_allclose(e[interior], area[interior] * dens, rtol=1e-9)


def test_fvm_hinge_not_exact_on_jittered_mesh():
    """FP/FS are mesh dependent on irregular meshes (Section 6.1, Section 7)."""
    xy, tris = tri_mesh("jittered")
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, "FP", E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    interior = np.all(st.idx >= 0, axis=1)
    K = np.diag([1.0, 0.3])
    x = rest.copy()
    x[:, 2] = quad_surface(xy, K)
    area = op.tri_area(st.rest[:, 0], st.rest[:, 1], st.rest[:, 2])
    kappa = np.array([1.0, 0.3, 0.0])
    dens = 0.5 * kappa @ op.bending_D(E, NU, T) @ kappa
    ratio = stencil_energy(x, st)[interior] / (area[interior] * dens)
    assert np.ptp(ratio) > 1e-2


def _edge_directions(st):
    e = st.rest[:, 2] - st.rest[:, 1]
    return e / np.linalg.norm(e, axis=1, keepdims=True)


def test_edge_hinge_right_triangle_grid_closed_form():
    xy, tris = tri_mesh("regular")
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, "EP", E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    kb = op.bending_rigidity(E, NU, T)
    AE = st.W[:, 0, 0] / kb
    d = _edge_directions(st)
    horiz = np.abs(d[:, 1]) < 1e-12
    vert = np.abs(d[:, 0]) < 1e-12
    diag = ~(horiz | vert)
    assert horiz.sum() and vert.sum() and diag.sum()
    for _ in range(3):
        K = random_K()
        x = rest.copy()
        x[:, 2] = quad_surface(xy, K)
        e = stencil_energy(x, st)
        kap = np.where(horiz, K[1, 1] + K[0, 1], np.where(vert, K[0, 0] + K[0, 1], -2.0 * K[0, 1]))
        np.testing.assert_allclose(e, 0.5 * kb * AE * kap ** 2, rtol=1e-9, atol=1e-12 * np.abs(e).max())
    # grid-aligned cylinders: the direction-averaged density equals the KL density k_b/2 K^2
    for K in (np.diag([2.0, 0.0]), np.diag([0.0, 2.0])):
        x = rest.copy()
        x[:, 2] = quad_surface(xy, K)
        e = stencil_energy(x, st)
        dens = sum(np.mean(e[s] / AE[s]) for s in (horiz, vert, diag))
        assert dens == pytest.approx(0.5 * kb * 4.0, rel=1e-10)


def test_edge_hinge_equilateral_closed_form():
    xy, tris = tri_mesh("equilateral")
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, "EP", E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    kb = op.bending_rigidity(E, NU, T)
    AE = st.W[:, 0, 0] / kb
    d = _edge_directions(st)
    mvec = np.stack([d[:, 1], -d[:, 0]], axis=1)
    # interior stencils away from the trimmed outline are equilateral
    L = np.linalg.norm(st.rest[:, 2] - st.rest[:, 1], axis=1)
    h1 = np.linalg.norm(np.cross(st.rest[:, 0] - st.rest[:, 1], st.rest[:, 2] - st.rest[:, 1]), axis=1) / L
    equi = np.abs(h1 - L * math.sqrt(3) / 2) < 1e-9
    equi &= np.abs(AE - L * L * math.sqrt(3) / 2) < 1e-9
    assert equi.sum() > 50
    for _ in range(3):
        K = random_K()
        x = rest.copy()
        x[:, 2] = quad_surface(xy, K)
        e = stencil_energy(x, st)
        kap = (4.0 * np.einsum("si,ij,sj->s", mvec, K, mvec) - np.trace(K)) / 3.0
        np.testing.assert_allclose(e[equi], 0.5 * kb * AE[equi] * kap[equi] ** 2, rtol=1e-9,
                                   atol=1e-12 * np.abs(e).max())


@pytest.mark.parametrize("model", ["ES", "FS", "SS"])
def test_flat_shell_bent_to_cylinder(model):
    """Rest-flat shell rolled onto radius R: interior energy -> (k_b/2)/R^2 per unit area as s -> 0."""
    n = 24
    R = 2.0
    width = 1.0
    xy, tris = sg.grid(n, n, 1.0, width)
    rest = sg.flat3(xy)
    x = sg.roll_to_cylinder(xy, R, width)
    m = osys.build_model(tris, rest, model, E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    interior = np.all(st.idx >= 0, axis=1)
    kb = op.bending_rigidity(E, NU, T)
    e = stencil_energy(x, st)
    if model == "ES":
        AE = st.W[:, 0, 0] / kb
        d = _edge_directions(st)
        along_axis = np.abs(d[:, 1]) < 1e-12          # hinges parallel to the axis see the full curvature
        across = np.abs(d[:, 0]) < 1e-12              # hinges across the axis see none
        kap = np.sqrt(2.0 * e / (kb * AE))
        np.testing.assert_allclose(kap[interior & along_axis], 1.0 / R, rtol=2e-3)
        assert np.max(kap[interior & across]) < 1e-3 / R
    else:
        area = op.tri_area(st.rest[:, 0], st.rest[:, 1], st.rest[:, 2])
        ratio = e[interior].sum() / (area[interior].sum() * 0.5 * kb / R ** 2)
        assert ratio == pytest.approx(1.0, rel=5e-3)


@pytest.mark.parametrize("model", ["ES", "FS", "SS"])
def test_curved_rest_rebent_scales_with_curvature_change(model):
    n = 20
    width = 0.8
    R0 = 1.5
    xy, tris = sg.grid(n, n, 1.0, width)
    rest = sg.roll_to_cylinder(xy, R0, width)
    m = osys.build_model(tris, rest, model, E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    interior = np.all(st.idx >= 0, axis=1)
    assert np.sum(stencil_energy(rest, st)) < 1e-20
    psi = {}
    for R1 in (1.0, 1.2, 2.0, 3.0):
        psi[R1] = np.sum(stencil_energy(sg.roll_to_cylinder(xy, R1, width), st)[interior])
    ref = psi[1.0] / (1 / 1.0 - 1 / R0) ** 2
    for R1 in (1.2, 2.0, 3.0):
        assert psi[R1] / (1 / R1 - 1 / R0) ** 2 == pytest.approx(ref, rel=3e-2)


def test_shell_and_plate_agree_for_small_deflection():
    """EP/ES, FP/FS, SP/SS give the same energy to leading order for small deflections (Section 6.1)."""
    n = 8
    xy, tris = sg.grid(n, n)
    rest = sg.flat3(xy)
    x = rest.copy()
    x[:, 2] = 1e-4 * np.sin(3.0 * xy[:, 0]) * np.cos(2.0 * xy[:, 1])
    for p, s in (("EP", "ES"), ("FP", "FS"), ("SP", "SS")):
        mp = osys.build_model(tris, rest, p, E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
        ms = osys.build_model(tris, rest, s, E, NU, T, 1.0, 1e-2, membrane=False, factor=False)
        ep = osys.bending_energy(mp, x)
        es = osys.bending_energy(ms, x)
        assert es == pytest.approx(ep, rel=1e-6)


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def timoshenko_ratio(model, mesh, n):
    g = _read_golden("timoshenko_ss_square.txt")
    rest, tris, bmask = sg.simply_supported_square(n, g["a"], mesh)
    m = osys.build_model(tris, rest, model, g["E"], g["nu"], g["h"], 1.0, 1.0, pinned=bmask, membrane=False,
                         factor=False)
    Kb, _ = osys.stiffness_matrices(m)
    nodal_area = np.zeros(rest.shape[0])
    np.add.at(nodal_area, tris.ravel(), np.repeat(m.tri_area / 3.0, 3))
    free = ~bmask
    w = spla.spsolve(Kb.tocsr()[free][:, free].tocsc(), g["B"] * nodal_area[free])
    wref = g["C"] * g["B"] * g["a"] ** 4 * (1 - g["nu"] ** 2) / (g["E"] * g["h"] ** 3)
    return w.max() / wref


def test_timoshenko_plate_convergence():
    rows = []
    with open(os.path.join(GOLDEN, "paper_models.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b, c = line.split()
                rows.append((a, b, c == "1"))
    for model, mesh, converges in rows:
        r16 = timoshenko_ratio(model, mesh, 16)
        r32 = timoshenko_ratio(model, mesh, 32)
        if converges:
            assert abs(r32 - 1.0) < 0.03, (model, mesh, r32)
            assert abs(r32 - 1.0) <= abs(r16 - 1.0) + 1e-9, (model, mesh, r16, r32)
        else:
            assert abs(r32 - 1.0) > 0.2, (model, mesh, r32)


# ------------------------------------------------------------------ membrane
def _one_triangle():
    X = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0]]])
    Dm_inv, area = membrane_rest(X)
    return X, Dm_inv, area


def _deform(X, Fmat, Q=np.eye(3)):
    return (Q @ (Fmat @ X[0].T)).T[None]


def test_membrane_uniaxial_equibiaxial_rotation():
    X, Dm_inv, area = _one_triangle()
    mu, lam = lame(E, NU)
    e = 1e-3
    F = np.diag([1 + e, 1.0, 1.0])
    en, _ = membrane_energy_force(_deform(X, F), Dm_inv, area, E, NU, T)
    assert en[0] == pytest.approx(0.5 * area[0] * T * E * e * e / (1 - NU * NU), rel=1e-9)
    F = np.diag([1 + e, 1 + e, 1.0])
    en, _ = membrane_energy_force(_deform(X, F), Dm_inv, area, E, NU, T)
    assert en[0] == pytest.approx(area[0] * T * e * e * (2 * mu + 2 * lam), rel=1e-9)
    Q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    en, f = membrane_energy_force(_deform(X, np.eye(3), Q), Dm_inv, area, E, NU, T)
    assert abs(en[0]) < 1e-20
    assert np.abs(f).max() < 1e-12
    # a large rigid rotation of a stretched state changes neither energy nor force magnitude
    F = np.diag([1 + e, 1 - 0.5 * e, 1.0])
    e1, f1 = membrane_energy_force(_deform(X, F), Dm_inv, area, E, NU, T)
    e2, f2 = membrane_energy_force(_deform(X, F, Q), Dm_inv, area, E, NU, T)
    assert e2[0] == pytest.approx(e1[0], rel=1e-12)
    np.testing.assert_allclose(f2[0], (Q @ f1[0].T).T, atol=1e-12 * np.abs(f1).max())
