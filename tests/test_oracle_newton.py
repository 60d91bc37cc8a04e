"""Pins of the oracle's Newton iterations (exact backward Euler, Section 5 Eq. 62-63, and the quasi-static
Newton-Raphson of Eq. 64) and of the membrane tangent they use, against facts that do not come from the
Newton loop itself:

* the closed-form membrane Hessian equals central differences of the oracle's membrane forces at rotated,
  stretched and compressed states; its projected form is positive semi-definite and equals the exact one in
  tension; its frozen-rotation part is the linear constant-strain stiffness at rest and is bounded by the
  isotropic block of the linearised step;
* the Newton step's velocity is the minimiser of the incremental potential found by L-BFGS, reached in a few
  iterations where the chord iteration with the constant matrix is still far off;
* the quasi-static solve ends below eps_f at the minimiser of the total potential (L-BFGS), its first step
  moves the largest nodal displacement by exactly eps_u, and it needs at least w_tip / eps_u iterations.
"""
import dataclasses

import numpy as np
import pytest
import scipy.optimize

import shellgen as sg
from oracle import newton as nw
from oracle import system as osys
from oracle.energies import lame, membrane_energy_force, membrane_rest, membrane_stiffness_blocks

E, NU, T = 1e6, 0.3, 1e-3
X1 = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0]]])


def _fd_hessian(x, Dm, A, h=1e-6):
    H = np.zeros((9, 9))
    for k in range(9):
        xp, xm = x.copy(), x.copy()
        xp.reshape(-1)[k] += h
        xm.reshape(-1)[k] -= h
        fp = membrane_energy_force(xp, Dm, A, E, NU, T)[1].reshape(-1)
        fm = membrane_energy_force(xm, Dm, A, E, NU, T)[1].reshape(-1)
        H[:, k] = -(fp - fm) / (2 * h)
    return H


def _as9(H):
    return H[0].transpose(0, 2, 1, 3).reshape(9, 9)


@pytest.mark.parametrize("stretch", [0.25, -0.12, 0.0])
def test_membrane_hessian_matches_finite_differences(stretch):
    rng = np.random.default_rng(int(1000 * abs(stretch)) + 1)
    Dm, A = membrane_rest(X1)
    for _ in range(3):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        Fm = np.eye(3) + stretch * np.eye(3) + 0.1 * rng.standard_normal((3, 3))
        x = (Q @ (Fm @ X1[0].T)).T[None] + rng.standard_normal(3)
        H = _as9(nw.membrane_hessian_blocks(x, Dm, A, E, NU, T, project=False))
        Hfd = _fd_hessian(x, Dm, A)
        assert np.abs(H - Hfd).max() <= 2e-8 * np.abs(Hfd).max()
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_projected_hessian_is_psd_and_exact_in_tension():
    rng = np.random.default_rng(5)
    Dm, A = membrane_rest(X1)
    for s in (-0.3, -0.1, 0.05, 0.3):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        x = (Q @ ((1 + s) * np.eye(3) @ X1[0].T)).T[None]
        Hp = _as9(nw.membrane_hessian_blocks(x, Dm, A, E, NU, T, project=True))
        assert np.linalg.eigvalsh(Hp).min() >= -1e-9 * np.abs(Hp).max()
        He = _as9(nw.membrane_hessian_blocks(x, Dm, A, E, NU, T, project=False))
        if s > 0:     # equibiaxial tension: kappa = mu - c / tr S > 0 and Q > 0, nothing to clamp
            np.testing.assert_allclose(Hp, He, rtol=0, atol=1e-12 * np.abs(He).max())
        else:         # compression: the exact Hessian has negative directions, the projection removes them
            assert np.linalg.eigvalsh(He).min() < -1e-6 * np.abs(He).max()


def test_frozen_part_is_linear_stiffness_at_rest_and_below_the_isotropic_block():
    Dm, A = membrane_rest(X1)
    Hf = _as9(nw.membrane_tangent_blocks(X1, Dm, A, E, NU, T))
    np.testing.assert_allclose(Hf, _fd_hessian(X1.copy(), Dm, A), rtol=0, atol=1e-8 * np.abs(Hf).max())
    np.testing.assert_allclose(Hf, _as9(nw.membrane_hessian_blocks(X1, Dm, A, E, NU, T)), rtol=0,
                               atol=1e-12 * np.abs(Hf).max())
    rng = np.random.default_rng(9)
    Kiso = np.kron(membrane_stiffness_blocks(Dm, A, E, NU, T)[0], np.eye(3))
    for _ in range(5):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        x = (Q @ ((np.eye(3) + 0.2 * rng.standard_normal((3, 3))) @ X1[0].T)).T[None]
        Hf = _as9(nw.membrane_tangent_blocks(x, Dm, A, E, NU, T))
        assert np.linalg.eigvalsh(Hf).min() >= -1e-9 * np.abs(Hf).max()
        assert np.linalg.eigvalsh(Kiso - Hf).min() >= -1e-9 * np.abs(Kiso).max()


def _swinging(model, seed=1):
    """A cylinder panel held on one straight edge, moving: a rotating motion the constant matrix resists."""
    sc = sg.cylinder_panel(5, model, ny=4, E=2e5, load=0.0, gravity=(0.0, 0.0, -9.81), dt=2e-2)
    side = sc.clamped_edges[: len(sc.clamped_edges) // 2]
    pinned = np.zeros(sc.n_verts, np.uint8)
    pinned[np.unique(side)] = 1
    sc = dataclasses.replace(sc, clamped_edges=side.astype(np.int32), pinned=pinned)
    m = osys.from_scenario(sc)
    rng = np.random.default_rng(seed)
    v = 0.5 * rng.standard_normal(sc.x0.shape)
    v[m.pinned] = 0.0
    return m, sc.x0.copy(), v


@pytest.mark.parametrize("model", ["EP", "SS"])
def test_newton_step_minimises_the_incremental_potential(model):
    m, x, v = _swinging(model)
    xn, vn, it = nw.step_newton(m, x, v, 1, max_iters=30, rtol=1e-11)
    assert it[0] <= 16          # linear rate ~0.2 per iteration: the constant bending Hessian is not exact
    free = ~m.pinned

    def fun(z):
        vv = np.zeros_like(v)
        vv[free] = z.reshape(-1, 3)
        g = osys.residual_nonlinear(m, x, v, vv)
        return osys.incremental_potential(m, x, v, vv), g[free].ravel()

    res = scipy.optimize.minimize(fun, vn[free].ravel() * 0.0, jac=True, method="L-BFGS-B",
                                  options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-13})
    vmin = np.zeros_like(v)
    vmin[free] = res.x.reshape(-1, 3)
    assert np.linalg.norm(vn - vmin) <= 1e-5 * np.linalg.norm(vn)
    # the chord iteration with the constant matrix is still far from it after as many solves
    _, vc, _ = osys.step_nonlinear(m, x, v, 1, max_iters=it[0], rtol=0.0)
    assert np.linalg.norm(vc - vn) > 1e2 * np.linalg.norm(vmin - vn)


@pytest.mark.parametrize("model", ["EP", "FP", "SP"])
def test_static_solve_reaches_the_energy_minimiser(model):
    sc = sg.cantilever(model, nx=8, ny=2, total_load=1.0)
    m = osys.from_scenario(sc, factor=False)
    eps_u = 0.1
    x, it, nr = nw.solve_static(m, sc.rest, eps_f=1e-6, eps_u=eps_u, max_iters=400)
    assert nr < 1e-6
    tip = sg.cantilever_tip(sc)
    w = x[tip, 2] - sc.rest[tip, 2]
    assert it >= w / eps_u
    # the first step is limited: its largest nodal displacement is exactly eps_u
    x1, it1, _ = nw.solve_static(m, sc.rest, eps_f=0.0, eps_u=eps_u, max_iters=1)
    assert it1 == 1 and np.abs(x1 - sc.rest).max() == pytest.approx(eps_u, rel=1e-12)
    # independent minimisation of the total potential Psi(x) - f_ext . x over the free vertices
    free = ~m.pinned

    def fun(z):
        xx = sc.rest.copy()
        xx[free] = z.reshape(-1, 3)
        e = osys.membrane_energy(m, xx) + osys.bending_energy(m, xx) - float(np.sum(m.f_ext * xx))
        return e, -nw.static_residual(m, xx)[free].ravel()

    # started from the rest shape, not from the Newton result
    res = scipy.optimize.minimize(fun, sc.rest[free].ravel(), jac=True, method="L-BFGS-B",
                                  options={"maxiter": 50000, "ftol": 1e-16, "gtol": 1e-10})
    xmin = sc.rest.copy()
    xmin[free] = res.x.reshape(-1, 3)
    assert np.linalg.norm(x - xmin) <= 3e-4 * np.linalg.norm(x - sc.rest)
