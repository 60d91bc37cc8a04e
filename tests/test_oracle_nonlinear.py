"""Pins of the oracle's exact backward-Euler step (chord iteration, Section 5, Eq. 62-63 without the
linearisation) against facts that do not come from the chord loop itself."""
import dataclasses

import numpy as np
import pytest
import scipy.optimize

import shellgen as sg
from oracle import system as osys


def _perturbed(sc, seed=0, dx=1e-3, dv=0.05):
    m = osys.from_scenario(sc)
    rng = np.random.default_rng(seed)
    x = sc.x0 + dx * rng.standard_normal(sc.x0.shape)
    v = dv * rng.standard_normal(sc.x0.shape)
    x[m.pinned] = sc.x0[m.pinned]
    v[m.pinned] = 0.0
    return m, x, v


@pytest.mark.parametrize("model", ["EP", "FS", "SS"])
def test_first_chord_iterate_is_the_linearised_step(model):
    """v_1 = A^-1 (M v + dt (f(x) + f_ext)) is exactly the linearised backward-Euler step."""
    sc = sg.cylinder_panel(6, model) if model[1] == "S" else sg.plate_clamped_x0(6, model=model)
    m, x, v = _perturbed(sc)
    xl, vl = osys.step(m, x, v, 1)
    xn, vn, it = osys.step_nonlinear(m, x, v, 1, max_iters=1)
    assert it == [1]
    assert np.allclose(vn, vl, rtol=0, atol=1e-14 * np.abs(vl).max())
    assert np.allclose(xn, xl, rtol=0, atol=1e-14 * np.abs(xl).max())


@pytest.mark.parametrize("model", ["EP", "FP", "SP"])
def test_linear_forces_converge_in_one_iteration(model):
    """Without the (nonlinear, corotated) membrane and without clamped edges (whose fixed-normal energy has
    a projected Hessian), the plate force is exactly -K_b x (the (x) I_3 form) and A is its exact Hessian
    shifted by the mass, so the first chord iterate already solves backward Euler."""
    sc = sg.plate_clamped_x0(8, model=model)
    pinned = np.zeros(sc.n_verts, np.uint8)
    pinned[np.unique(sc.clamped_edges)] = 1          # hold the clamped side by its vertices instead
    sc = dataclasses.replace(sc, clamped_edges=np.zeros((0, 2), np.int32), pinned=pinned)
    m = osys.from_scenario(sc, membrane=False)
    rng = np.random.default_rng(3)
    x = sc.x0 + 1e-2 * rng.standard_normal(sc.x0.shape)
    v = rng.standard_normal(sc.x0.shape)
    x[m.pinned] = sc.x0[m.pinned]
    v[m.pinned] = 0.0
    r0 = np.linalg.norm(osys.residual_nonlinear(m, x, v, np.zeros_like(v)))
    _, vn, it = osys.step_nonlinear(m, x, v, 1, max_iters=5, rtol=1e-11)
    assert it == [1]
    assert np.linalg.norm(osys.residual_nonlinear(m, x, v, vn)) <= 1e-11 * r0


@pytest.mark.parametrize("model", ["ES", "SS"])
def test_chord_solution_minimises_the_incremental_potential(model):
    """Backward Euler is the minimiser of the incremental potential; an independent quasi-Newton minimisation
    (L-BFGS on the energy, free vertices) lands on the chord iteration's velocity."""
    sc = sg.cylinder_panel(4, model)
    m, x, v = _perturbed(sc, seed=1, dx=2e-3, dv=0.5)
    _, vc, it = osys.step_nonlinear(m, x, v, 1, max_iters=200, rtol=1e-12)
    free = ~m.pinned

    def f(z):
        vn = np.zeros_like(v)
        vn[free] = z.reshape(-1, 3)
        e = osys.incremental_potential(m, x, v, vn)
        g = osys.residual_nonlinear(m, x, v, vn)[free].ravel()
        return e, g

    res = scipy.optimize.minimize(f, np.zeros(3 * free.sum()), jac=True, method="L-BFGS-B",
                                  options={"maxiter": 20000, "gtol": 1e-13, "ftol": 1e-16})
    vm = np.zeros_like(v)
    vm[free] = res.x.reshape(-1, 3)
    assert np.linalg.norm(vm - vc) <= 1e-6 * np.linalg.norm(vc), (it, res.message)


def test_chord_iteration_reduces_the_linearisation_error():
    """On a stiff curved shell the linearised step leaves a nonlinear residual that the chord iteration
    reduces (linearly, by about 0.6 per iteration for this strongly perturbed stiff panel); the residual
    after k iterations decreases monotonically."""
    sc = sg.cylinder_panel(6, "SS")
    m, x, v = _perturbed(sc, seed=2, dx=5e-3, dv=1.0)
    r0 = np.linalg.norm(osys.residual_nonlinear(m, x, v, np.zeros_like(v)))
    res = []
    for k in (1, 2, 4, 8):
        _, vk, _ = osys.step_nonlinear(m, x, v, 1, max_iters=k, rtol=0.0)
        res.append(np.linalg.norm(osys.residual_nonlinear(m, x, v, vk)) / r0)
    assert all(b < a for a, b in zip(res, res[1:])), res
    assert res[0] > 1e-9 and res[-1] < res[0] / 5, res
