"""Newton iterations on the GPU against the oracle (Section 5: exact backward Euler by a Newton-type minimisation
of the incremental potential, Eq. 62-63; the quasi-static Newton-Raphson of Eq. 64 with the eps_u limiter),
through the C ABI.

* Exact backward Euler by Newton (FP64): positions and velocities after several steps equal the oracle's Newton
  solution (both iterate to ||R|| <= 1e-11 ||R(0)||) to 1e-9, with the same number of Newton iterations per
  step (+-1), 15-26 iterations (linear rate: the membrane Hessian is clamped where triangles are compressed,
  and a shell's constant bending Hessian is not its exact one); FP32 + refinement to 1e-6.
* Quasi-static cantilever of Section 6.1 (17 x 3 nodes, end shear 4, eps_u = 0.1): the GPU's equilibrium equals
  the oracle's (same shifted Newton steps) to 1e-7, with the same number of steps (+-1); its residual meets
  eps_f; the iteration limit reports NOT_CONVERGED without committing.
* A batch mixing Newton, chord and linearised instances gives each instance's states of stepping it alone.
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


def swinging(model, n=10, ny=8, seed=1, amp=0.1):
    """Cylinder panel held by the vertices of one straight edge, moving under gravity."""
    sc = sg.cylinder_panel(n, model, ny=ny, E=2e5, load=0.0, gravity=(0.0, 0.0, -9.81), dt=2e-2)
    side = sc.clamped_edges[: len(sc.clamped_edges) // 2]
    pinned = np.zeros(sc.n_verts, np.uint8)
    pinned[np.unique(side)] = 1
    rng = np.random.default_rng(seed)
    v0 = amp * rng.standard_normal(sc.x0.shape)
    v0[pinned.astype(bool)] = 0.0
    return dataclasses.replace(sc, clamped_edges=np.zeros((0, 2), np.int32), pinned=pinned, v0=v0)


def hanging_plate(model, seed=2):
    """Plate of 24 x 15 cells (400 vertices: two 256-row chunks, a ragged tail) held by the vertices of one edge,
    falling under gravity with a random initial velocity (its bending Hessian is exact)."""
    xy, tris = sg.grid(24, 15)
    rest = sg.flat3(xy)
    pinned = np.zeros(len(rest), np.uint8)
    pinned[sg.grid_side_vertices(24, 15, "x0")] = 1
    rng = np.random.default_rng(seed)
    v0 = 0.2 * rng.standard_normal(rest.shape)
    v0[pinned.astype(bool)] = 0.0
    sc = sg.plate_clamped_x0(24, model=model, E=1e5, dt=2e-2)
    return dataclasses.replace(sc, tris=tris, rest=rest, x0=rest.copy(), v0=v0, pinned=pinned,
                               clamped_edges=np.zeros((0, 2), np.int32))


@pytest.mark.parametrize("model,kind,its_max", [("EP", "plate", 30), ("FP", "plate", 30), ("SP", "plate", 30),
                                                ("SS", "shell", 30)])
def test_newton_backward_euler_fp64_matches_oracle(model, kind, its_max):
    sc = hanging_plate(model) if kind == "plate" else swinging(model)
    m = osys.from_scenario(sc, factor=False)
    xo, vo, its = nw.step_newton(m, sc.x0, sc.v0, 3, max_iters=60, rtol=1e-11)
    h = gb.create_from_scenario(sc, precision="fp64")
    gb.shell_set_nonlinear(h, 60, 1e-11)
    gb.shell_set_newton(h, True)
    gits = []
    for _ in range(3):
        st = gb.shell_step(h, 1)
        gits.append(st["nl_iterations"])
    x, v = gb.shell_get_state(h)
    print(model, "newton iterations oracle", its, "gpu", gits)
    assert max(its) <= its_max
    assert rel(x, xo, xo - sc.x0) <= 1e-9
    assert rel(v, vo, vo) <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, gits))


@pytest.mark.parametrize("model", ["SP", "SS"])
def test_newton_backward_euler_fp32_refine_matches_oracle(model):
    sc = hanging_plate(model) if model == "SP" else swinging(model)
    m = osys.from_scenario(sc, factor=False)
    xo, vo, _ = nw.step_newton(m, sc.x0, sc.v0, 3, max_iters=60, rtol=1e-11)
    h = gb.create_from_scenario(sc, precision="fp32_refine")
    gb.shell_set_nonlinear(h, 60, 1e-7)
    gb.shell_set_newton(h, True)
    st = gb.shell_step(h, 3)
    x, v = gb.shell_get_state(h)
    assert st["steps_done"] == 3 and st["nl_iterations"] < 60
    assert rel(x, xo, xo - sc.x0) <= 1e-6
    assert rel(v, vo, vo) <= 1e-6


@pytest.mark.parametrize("model", ["EP", "FP", "SP", "SS"])
def test_static_cantilever_matches_oracle(model):
    sc = sg.cantilever(model)
    m = osys.from_scenario(sc, factor=False)
    xo, it_o, nr_o = nw.solve_static(m, sc.rest, eps_f=1e-8, eps_u=0.1, max_iters=400, shift=True)
    h = gb.create_from_scenario(sc, precision="fp64")
    st = gb.shell_solve_static(h, eps_f=1e-8, eps_u=0.1, max_iters=400)
    x, v = gb.shell_get_state(h)
    tip = sg.cantilever_tip(sc)
    print(model, "w_tip oracle %.5f gpu %.5f, steps oracle %d gpu %d, |f + f_ext| gpu %.2e"
          % (xo[tip, 2] - sc.rest[tip, 2], x[tip, 2] - sc.rest[tip, 2], it_o, st["nl_iterations"],
             st["rel_residual"]))
    assert st["rel_residual"] < 1e-8
    assert np.linalg.norm(nw.static_residual(m, x)) < 1e-7
    # both stop below eps_f = 1e-8; the softest mode (about 0.3 N/m) turns that into ~3e-8 of position
    assert rel(x, xo, xo - sc.rest) <= 1e-7
    assert abs(st["nl_iterations"] - it_o) <= 1
    assert np.all(v == 0.0)


def test_static_iteration_limit_commits_nothing():
    sc = sg.cantilever("FP")
    h = gb.create_from_scenario(sc, precision="fp64")
    st = gb.shell_solve_static(h, eps_f=1e-7, eps_u=0.1, max_iters=10, check=False)
    assert st["rc"] == gb.SHELL_ERR_NOT_CONVERGED
    x, _ = gb.shell_get_state(h)
    assert np.array_equal(x, sc.rest)


def test_static_fp32_refine_cantilever():
    sc = sg.cantilever("SP")
    m = osys.from_scenario(sc, factor=False)
    xo, _, _ = nw.solve_static(m, sc.rest, eps_f=1e-7, eps_u=0.1, max_iters=400, shift=True)
    h = gb.create_from_scenario(sc, precision="fp32_refine")
    st = gb.shell_solve_static(h, eps_f=1e-3, eps_u=0.1, max_iters=400)
    x, _ = gb.shell_get_state(h)
    assert st["rel_residual"] < 1e-3
    assert rel(x, xo, xo - sc.rest) <= 1e-4    # an equilibrium to eps_f = 1e-3 (about 1e-4 of the tip load)


def test_mixed_batch_with_newton_instance_equals_alone():
    scs = [swinging("SS"), sg.plate_clamped_x0(14, model="EP"), hanging_plate("FS", seed=3)]
    modes = [("newton", 12), ("linear", 0), ("chord", 6)]

    def setup(h, mode):
        kind, k = mode
        if kind != "linear":
            gb.shell_set_nonlinear(h, k, 1e-9)
        if kind == "newton":
            gb.shell_set_newton(h, True)

    alone = []
    for sc, mode in zip(scs, modes):
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        setup(h, mode)
        gb.shell_step(h, 3)
        alone.append(gb.shell_get_state(h))
    b = gb.shell_batch_create(1 << 40)
    hs = []
    for sc, mode in zip(scs, modes):
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        setup(h, mode)
        gb.shell_batch_admit(b, h)
        hs.append(h)
    rc, _ = gb.shell_batch_step(b, 3)
    assert rc == 0
    x, v = gb.shell_batch_get_states(b)
    _, offs = gb.shell_batch_state_layout(b)
    for k in range(3):
        xs, vs = x[offs[k]:offs[k + 1]], v[offs[k]:offs[k + 1]]
        assert np.array_equal(xs, alone[k][0]) and np.array_equal(vs, alone[k][1]), k
    gb.shell_batch_destroy(b)
