"""Per-component constraints on the GPU against the oracle (Section 6.1's hemisphere: x fixed on the nodes of
the y-z plane, y on those of the x-z plane, z as well on the hole's edge in the y-z plane), through the C ABI.
The kernels keep the scalar matrix and project every product, right-hand side, residual and preconditioned
vector onto the free components (the step kernel's Newton-capable variant).

* Quasi-static hemisphere (Eq. 64, eps_u = 0.1): the GPU's equilibrium equals the oracle's (same shifted
  Newton steps) to 1e-7 with the same number of steps (+-1), the fixed components stay at rest, the free
  residual meets eps_f; the full 1088-node shell with SS, coarser meshes with ES and FS.
* Linearised backward-Euler steps with fixed components: FP64 to 1e-10 of the oracle's 3V solve, FP32 with
  refinement to 1e-6; fixed components keep their positions exactly.
* Exact backward Euler by Newton with fixed components: 1e-9 of the oracle's Newton.
* A batch holding a hemisphere and an unconstrained plate gives each its states of stepping alone.
"""
import dataclasses

import numpy as np
import pytest

import shellgen as sg
from oracle import newton as nw
from oracle import system as osys

gb = pytest.importorskip("paper_2502_10872_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.load_library()


def rel(a, b, ref):
    return np.linalg.norm(a - b) / max(np.linalg.norm(ref), 1e-300)


def fixed_mask(sc):
    return ((sc.fixed_dofs[:, None] >> np.arange(3)[None, :]) & 1).astype(bool)


@pytest.mark.parametrize("model,n_around,n_rings", [("SS", 64, 17), ("ES", 32, 9), ("FS", 32, 9)])
def test_static_hemisphere_matches_oracle(model, n_around, n_rings):
    sc = sg.hemisphere(model, n_around=n_around, n_rings=n_rings)
    m = osys.from_scenario(sc, factor=False)
    xo, it_o, _ = nw.solve_static(m, sc.rest, eps_f=1e-6, eps_u=0.1, max_iters=600, shift=True)
    h = gb.create_from_scenario(sc, precision="fp64")
    st = gb.shell_solve_static(h, eps_f=1e-6, eps_u=0.1, max_iters=600)
    x, v = gb.shell_get_state(h)
    ia, ib = sg.hemisphere_probes(sc)
    print(model, n_around * n_rings, "u_min oracle %.5f gpu %.5f, v_max oracle %.5f gpu %.5f, steps oracle %d gpu %d"
          % (xo[ia, 0] - sc.rest[ia, 0], x[ia, 0] - sc.rest[ia, 0], xo[ib, 1] - sc.rest[ib, 1],
             x[ib, 1] - sc.rest[ib, 1], it_o, st["nl_iterations"]))
    fx = fixed_mask(sc)
    assert np.array_equal(x[fx], sc.rest[fx])
    assert np.linalg.norm(nw.static_residual(m, x)) < 1e-6
    assert rel(x, xo, xo - sc.rest) <= 1e-7
    assert abs(st["nl_iterations"] - it_o) <= 1
    assert np.all(v == 0.0)


def swinging_hemisphere(model, seed=3):
    sc = sg.hemisphere(model, n_around=32, n_rings=9, load=0.0, density=500.0, dt=2e-2)
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(sc.rest.shape)
    v0[fixed_mask(sc)] = 0.0
    return dataclasses.replace(sc, v0=v0, gravity=(0.0, 0.0, -9.81), steps=5)


@pytest.mark.parametrize("model", ["ES", "FS", "SS"])
def test_linearised_steps_with_fixed_components(model):
    sc = swinging_hemisphere(model)
    m = osys.from_scenario(sc)
    xo, vo = osys.step(m, sc.x0, sc.v0, sc.steps)
    fx = fixed_mask(sc)
    for prec, tol in (("fp64", 1e-10), ("fp32_refine", 1e-6)):
        h = gb.create_from_scenario(sc, precision=prec)
        gb.shell_step(h, sc.steps)
        x, v = gb.shell_get_state(h)
        print(model, prec, "rel_x %.2e rel_v %.2e" % (rel(x, xo, xo - sc.x0), rel(v, vo, vo)))
        assert np.array_equal(x[fx], sc.x0[fx]) and np.all(v[fx] == 0.0)
        assert rel(x, xo, xo - sc.x0) <= tol
        assert rel(v, vo, vo) <= tol


def test_newton_backward_euler_with_fixed_components():
    sc = swinging_hemisphere("SS")
    m = osys.from_scenario(sc, factor=False)
    xo, vo, its = nw.step_newton(m, sc.x0, sc.v0, 2, max_iters=60, rtol=1e-11)
    h = gb.create_from_scenario(sc, precision="fp64")
    gb.shell_set_nonlinear(h, 60, 1e-11)
    gb.shell_set_newton(h, True)
    gits = [gb.shell_step(h, 1)["nl_iterations"] for _ in range(2)]
    x, v = gb.shell_get_state(h)
    print("newton iterations oracle", its, "gpu", gits)
    assert all(abs(a - b) <= 1 for a, b in zip(its, gits))
    assert rel(x, xo, xo - sc.x0) <= 1e-9
    assert rel(v, vo, vo) <= 1e-9


def test_batch_with_constrained_instance_equals_alone():
    scs = [swinging_hemisphere("SS"), sg.plate_clamped_x0(14, model="EP")]
    alone = []
    for sc in scs:
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        gb.shell_step(h, 3)
        alone.append(gb.shell_get_state(h))
    b = gb.shell_batch_create(1 << 40)
    hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
    for h in hs:
        gb.shell_batch_admit(b, h)
    rc, _ = gb.shell_batch_step(b, 3)
    assert rc == 0
    x, v = gb.shell_batch_get_states(b)
    _, offs = gb.shell_batch_state_layout(b)
    for k in range(2):
        xs, vs = x[offs[k]:offs[k + 1]], v[offs[k]:offs[k + 1]]
        assert np.array_equal(xs, alone[k][0]) and np.array_equal(vs, alone[k][1]), k
    gb.shell_batch_destroy(b)


def test_invalid_fixed_bits_rejected():
    sc = sg.hemisphere("ES", n_around=16, n_rings=5)
    bad = sc.fixed_dofs.copy()
    bad[3] = 8
    with pytest.raises(Exception):
        gb.create_from_scenario(dataclasses.replace(sc, fixed_dofs=bad), precision="fp64")
