"""Exact backward Euler on the GPU (chord iteration with the constant matrix, shell_set_nonlinear) against the
oracle's chord iteration, and its consistency with the linearised step, batching and the no-alloc entry."""
import numpy as np
import pytest

import shellgen as sg
from oracle import system as osys

gb = pytest.importorskip("paper_2502_10872_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.load_library()


def rel(a, b, ref):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(ref), 1e-300))


def _scene(name):
    if name == "cyl12_SS":
        return sg.cylinder_panel(12, "SS")
    if name == "cyl12_ES":
        return sg.cylinder_panel(12, "ES")
    return sg.plate_clamped_x0(16, model="FP")


@pytest.mark.parametrize("name", ["cyl12_SS", "cyl12_ES", "plate16_FP"])
def test_fixed_chord_iterations_match_oracle_fp64(name):
    """K chord iterations per step (rtol 0: always K solves) for 3 steps, FP64: equal to the oracle's."""
    sc = _scene(name)
    K = 4
    m = osys.from_scenario(sc)
    xo, vo, its = osys.step_nonlinear(m, sc.x0, sc.v0, 3, max_iters=K, rtol=0.0)
    assert its == [K] * 3
    h = gb.create_from_scenario(sc, precision="fp64")
    gb.shell_set_nonlinear(h, K, 0.0)
    st = gb.shell_step(h, 3)
    assert st["steps_done"] == 3 and st["nl_iterations"] == K
    xg, vg = gb.shell_get_state(h)
    assert rel(xg, xo, xo - sc.x0) <= 1e-10
    assert rel(vg, vo, vo) <= 1e-10


def test_converged_chord_iteration_matches_oracle():
    """Chord iteration to ||R|| <= 1e-8 ||R(0)||: the GPU commits a state whose backward-Euler residual (by
    the oracle) meets the tolerance, close to the oracle's converged state. (The chord iteration contracts
    slowly when dt^2 K dominates M: the constant isotropic membrane block resists in-plane rotations that
    the corotated energy leaves free, ~400 iterations for 1e-4 at dt = 5e-3 here; at dt = 5e-4, 16.)"""
    sc = sg.cylinder_panel(12, "SS", dt=5e-4)
    m = osys.from_scenario(sc)
    x0 = sc.x0.copy()
    v0 = sc.v0.copy()
    h = gb.create_from_scenario(sc, precision="fp64")
    gb.shell_set_nonlinear(h, 60, 1e-8)
    st = gb.shell_step(h, 1)
    assert st["steps_done"] == 1 and 1 <= st["nl_iterations"] < 60
    xg, vg = gb.shell_get_state(h)
    r0 = np.linalg.norm(osys.residual_nonlinear(m, x0, v0, np.zeros_like(v0)))
    assert np.linalg.norm(osys.residual_nonlinear(m, x0, v0, vg)) <= 2e-8 * r0
    xo, vo, its = osys.step_nonlinear(m, x0, v0, 1, max_iters=60, rtol=1e-8)
    assert abs(its[0] - st["nl_iterations"]) <= 1
    assert rel(vg, vo, vo) <= 1e-7


def test_fixed_chord_iterations_fp32_refine():
    """FP32 forces and PCG with FP64 refinement: the chord iterate agrees with the FP64 oracle to the FP32
    force rounding (the bound of the linearised FP32 path, 1e-6)."""
    sc = sg.cylinder_panel(12, "FS")
    m = osys.from_scenario(sc)
    xo, vo, _ = osys.step_nonlinear(m, sc.x0, sc.v0, 2, max_iters=3, rtol=0.0)
    h = gb.create_from_scenario(sc, precision="fp32_refine", refine_rtol=1e-10)
    gb.shell_set_nonlinear(h, 3, 0.0)
    st = gb.shell_step(h, 2)
    assert st["nl_iterations"] == 3
    xg, _ = gb.shell_get_state(h)
    assert rel(xg, xo, xo - sc.x0) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_one_chord_iteration_is_the_linearised_step_bitwise(precision):
    sc = sg.cylinder_panel(12, "SS")
    ha = gb.create_from_scenario(sc, precision=precision)
    hb = gb.create_from_scenario(sc, precision=precision)
    gb.shell_set_nonlinear(hb, 1, 1e-8)
    gb.shell_step(ha, 4)
    gb.shell_step(hb, 4)
    xa, va = gb.shell_get_state(ha)
    xb, vb = gb.shell_get_state(hb)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_nonlinear_alone_in_batch_and_noalloc_agree_bitwise():
    """Exact and linearised instances mixed in one batch (the batch issues the largest number of chord
    launches; finished instances skip them) give the states of each instance stepped alone, and so does the
    entry point without allocation."""
    scs = [sg.cylinder_panel(10, "SS"), sg.plate_clamped_x0(12, model="EP"), sg.cylinder_panel(8, "FS")]
    iters = [5, 0, 3]
    alone = []
    for sc, k in zip(scs, iters):
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        gb.shell_set_nonlinear(h, k, 1e-6)
        gb.shell_step(h, 3)
        alone.append(gb.shell_get_state(h))
    b = gb.shell_batch_create(1 << 40)
    hs = []
    for sc, k in zip(scs, iters):
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        gb.shell_set_nonlinear(h, k, 1e-6)
        gb.shell_batch_admit(b, h)
        hs.append(h)
    _, stats = gb.shell_batch_step(b, 3)
    for k, h in enumerate(hs):
        xa, va = alone[k]
        xb, vb = gb.shell_get_state(h)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb), k
    assert [s["nl_iterations"] for s in stats.values()][1] == 0
    gb.shell_batch_destroy(b)
    h = gb.create_from_scenario(scs[0], precision="fp32_refine")
    gb.shell_set_nonlinear(h, iters[0], 1e-6)
    st = gb.shell_step_noalloc(h, 3)
    assert st["steps_done"] == 3
    xc, vc = gb.shell_get_state(h)
    assert np.array_equal(xc, alone[0][0]) and np.array_equal(vc, alone[0][1])


def test_set_nonlinear_rejects_bad_arguments():
    h = gb.create_from_scenario(sg.plate_clamped_x0(8, model="EP"))
    for k, r in [(-1, 1e-8), (3, -1.0), (3, float("nan"))]:
        with pytest.raises(gb.ShellError):
            gb.shell_set_nonlinear(h, k, r)
