"""App. D: the world-frame edge-hinge models QTP / QTS and the factor 3 against the Quadratic / Cubic shell.

* App. D's operator L_n, written from its printed form (feet by orthogonal projection, unsigned distance
  ratios), equals the corotational edge operator L_m of Eq. 9-10 on stencils whose feet lie on the hinge; on
  obtuse stencils the printed form no longer annihilates constants (so translations would bend), and the
  signed-foot reading restores L_n = L_m.
* Because every row of L_n sums to zero, applying it in the world frame equals applying it to x - x_o:
  QTP's energy, gradient and Hessian equal EP's, and QTS's equal ES's, on deformed meshes.
* Quadratic / Cubic shell energy (Eq. 89, from the dihedral angle): for small out-of-plane deflections of a
  flat plate it is three times the EP energy, stencil by stencil, with an error that falls quadratically with
  the deflection (App. D, after Eq. 89).
"""
import numpy as np
import pytest

import shellgen as sg
from oracle import appendix_d as ad
from oracle import operators as op
from oracle import system as osys
from oracle.energies import frame_normal, stencil_energy, stencil_forces

E, NU, T = 3e6, 0.35, 2e-3
KB = op.bending_rigidity(E, NU, T)


def _random_stencils(S, rng, foot_lo, foot_hi):
    """Flat stencils X [S,4,3] with hinge X2-X3, wing feet at signed coordinates in [foot_lo, foot_hi], then
    a random rotation and translation."""
    X = np.zeros((S, 4, 3))
    L = rng.uniform(0.5, 2.0, S)
    X[:, 2, 0] = L
    s1, s4 = rng.uniform(foot_lo, foot_hi, S), rng.uniform(foot_lo, foot_hi, S)
    X[:, 0, 0], X[:, 0, 1] = s1 * L, rng.uniform(0.3, 1.5, S)
    X[:, 3, 0], X[:, 3, 1] = s4 * L, -rng.uniform(0.3, 1.5, S)
    for s in range(S):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        X[s] = X[s] @ Q.T + rng.standard_normal(3)
    return X


def test_printed_world_operator_equals_corotational_on_acute_stencils():
    rng = np.random.default_rng(1)
    X = _random_stencils(200, rng, 0.05, 0.95)
    Ln, An = ad.world_operator(X, signed=False)
    Lm, Am = op.edge_operator(X)
    np.testing.assert_allclose(Ln, Lm, rtol=1e-12, atol=1e-12 * np.abs(Lm).max())
    np.testing.assert_allclose(An, Am, rtol=1e-13)
    np.testing.assert_allclose(ad.world_operator(X, signed=True)[0], Lm, rtol=1e-12, atol=1e-12 * np.abs(Lm).max())


def test_printed_world_operator_fails_constants_on_obtuse_stencils():
    rng = np.random.default_rng(2)
    X = _random_stencils(100, rng, 1.2, 1.8)    # both feet beyond X3: obtuse angles at the hinge
    Ln, _ = ad.world_operator(X, signed=False)
    scale = np.abs(Ln).max(axis=1)
    assert np.all(np.abs(Ln.sum(axis=1)) > 1e-3 * scale)
    Ls, _ = ad.world_operator(X, signed=True)
    np.testing.assert_allclose(Ls.sum(axis=1), 0.0, atol=1e-12 * scale.max())
    np.testing.assert_allclose(Ls, op.edge_operator(X)[0], rtol=1e-12, atol=1e-12 * scale.max())


def _free_model(model, tris, rest):
    m = osys.build_model(tris, rest, model, E, NU, T, 1000.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    assert st.kind == "edge" and np.all(st.idx >= 0)      # no clamped edges: interior hinges only
    return m, st


def test_qtp_equals_ep_energy_gradient_and_hessian():
    xy, tris = sg.grid(7, 5)
    rest = sg.flat3(xy)
    m, st = _free_model("EP", tris, rest)
    x = rest + 0.05 * np.random.default_rng(3).standard_normal(rest.shape)
    eq, gq = ad.qtp_energy_gradient(x, st.idx, st.rest, KB, signed=False)
    ee = stencil_energy(x, st)
    np.testing.assert_allclose(eq, ee, rtol=1e-11, atol=1e-13 * ee.max())
    np.testing.assert_allclose(-gq, stencil_forces(x, st), rtol=1e-10, atol=1e-11 * np.abs(gq).max())
    # Hessian k_b A_E L_n^T L_n assembled = the constant bending matrix K_b of the EP model
    V = len(rest)
    H = np.zeros((V, V))
    blocks = ad.qtp_hessian(st.rest, KB, signed=False)
    for s in range(len(st)):
        H[np.ix_(st.idx[s], st.idx[s])] += blocks[s]
    Kb, _ = osys.stiffness_matrices(m)
    np.testing.assert_allclose(H, Kb.toarray(), rtol=1e-11, atol=1e-12 * np.abs(H).max())


def test_qts_equals_es_energy_and_gradient():
    width = 0.5 * np.pi / 2
    xy, tris = sg.grid(8, 6, 1.0, width)
    rest = sg.roll_to_cylinder(xy, 0.5, width)
    m, st = _free_model("ES", tris, rest)
    x = rest + 0.02 * np.random.default_rng(4).standard_normal(rest.shape)
    eq, gq = ad.qts_energy_gradient(x, st.idx, st.rest, KB, lambda xs: frame_normal(xs, "edge"), signed=True)
    ee = stencil_energy(x, st)
    np.testing.assert_allclose(eq, ee, rtol=1e-10, atol=1e-12 * ee.max())
    np.testing.assert_allclose(-gq, stencil_forces(x, st), rtol=1e-9, atol=1e-10 * np.abs(gq).max())


@pytest.mark.parametrize("mesh", ["regular", "jittered"])
def test_quadratic_shell_energy_is_three_times_ep_for_small_deflection(mesh):
    n = 8
    xy, tris = sg.grid(n, n)
    if mesh == "jittered":
        xy = sg.jitter(xy, 1.0 / n, 0.2, sg.grid_interior_mask(n, n), 9)
    rest = sg.flat3(xy)
    m = osys.build_model(tris, rest, "EP", E, NU, T, 1000.0, 1e-2, membrane=False, factor=False)
    st = m.stencils[0]
    w = np.random.default_rng(5).standard_normal(len(rest))
    errs = []
    for eps in (1e-4, 1e-5):
        x = rest.copy()
        x[:, 2] = eps * w
        ratio = ad.quadratic_shell_energy(x, st.idx, st.rest, KB) / stencil_energy(x, st)
        errs.append(np.abs(ratio - 3.0).max())
    assert errs[0] < 1e-4 and errs[1] < 1e-6
    assert errs[1] < 0.02 * errs[0]       # O(eps^2): a tenfold smaller deflection, a hundredfold smaller error
