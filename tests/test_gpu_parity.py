"""GPU-vs-oracle parity of the whole step through the C ABI (needs a GB300).

Metric (per result): rel_x = |x - x*| / |x* - X| (displacement relative, origin independent), rel_v =
|v - v*| / |v*|, energies relative per component. Bars: 1e-10 in FP64; the FP32 path with FP64
refinement states its own bound per case (<= 1e-6 for the solve, and the measured force-rounding error).
Sizes span several 256-row chunks with ragged tails (multi-CTA teams and their global barrier), every
model, every boundary type, point loads, gravity, rest-curved and rest-flat shells.
"""
import numpy as np
import pytest

import shellgen as sg
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
    d = np.linalg.norm(ref)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def run_both(sc, steps, precision="fp64", **kw):
    m = osys.from_scenario(sc)
    xo, vo = osys.step(m, sc.x0, sc.v0, steps)
    h = gb.create_from_scenario(sc, precision=precision, **kw)
    st = gb.shell_step(h, steps)
    xg, vg = gb.shell_get_state(h)
    return m, h, st, (xg, vg), (xo, vo)


def test_plate16_edge_hinge_fp64_100_steps():
    """16 x 16 edge-hinge plate, one edge clamped, gravity, 100 steps (the small end-to-end workload)."""
    sc = sg.plate_clamped_x0(16, model="EP")
    m, h, st, (xg, vg), (xo, vo) = run_both(sc, 100)
    assert st["steps_done"] == 100
    assert rel(xg, xo, xo - sc.rest) <= 1e-10
    assert rel(vg, vo, vo) <= 1e-10
    eg = gb.shell_energy(h)
    eo = np.array(osys.energy(m, xo, vo))
    for k in range(4):
        assert abs(eg[k] - eo[k]) <= 1e-9 * abs(eo[k]) + 1e-18, (k, eg, eo)


@pytest.mark.parametrize("model", sg.MODELS)
def test_all_models_plate_scene_fp64(model):
    """Ragged plate (21 x 13 cells, 308 vertices -> 2 chunks), x0 edge clamped, gravity, a point load."""
    sc = sg.plate_clamped_x0(21, model=model)
    xy, tris = sg.grid(21, 13)
    sc.tris, sc.rest = tris, sg.flat3(xy)
    sc.x0, sc.v0 = sc.rest.copy(), np.zeros_like(sc.rest)
    sc.pinned = np.zeros(sc.rest.shape[0], np.uint8)
    sc.pinned[sg.grid_side_vertices(21, 13, "x0")] = 1
    sc.clamped_edges = sg.grid_side_edges(21, 13, "x0")
    sc.load_vtx = np.array([sc.rest.shape[0] - 1], np.int32)
    sc.load_f = np.array([[0.0, 0.3, -0.5]])
    sc.E = 2e5
    m, h, st, (xg, vg), (xo, vo) = run_both(sc, 25)
    assert rel(xg, xo, xo - sc.rest) <= 1e-10, model
    assert rel(vg, vo, vo) <= 1e-10, model


@pytest.mark.parametrize("model", sg.MODELS)
def test_all_models_cylinder_scene_fp64(model):
    """Cylinder panel 30 x 23 cells (744 vertices, 3 chunks), both straight edges clamped, point load; plate
    models rest flat and start curved."""
    sc = sg.cylinder_panel(30, model, ny=23, radius=0.6, dt=5e-3)
    m, h, st, (xg, vg), (xo, vo) = run_both(sc, 20)
    assert rel(xg, xo, xo - sc.x0) <= 1e-10, model


@pytest.mark.parametrize("model", sg.MODELS)
def test_matrix_matches_oracle(model):
    """The device-assembled constant matrix equals the oracle's M + dt^2 (K_b + K_m) (pinned rows identity)."""
    rng = np.random.default_rng(2)
    sc = sg.cylinder_panel(14, model, ny=9, radius=0.8) if model in sg.SHELL_MODELS else sg.plate_clamped_x0(14, model)
    m = osys.from_scenario(sc, factor=False)
    A = osys.system_matrix(m)
    h = gb.create_from_scenario(sc)
    u = rng.standard_normal(sc.x0.shape)
    ag = gb.shell_apply_matrix(h, u)
    ao = A @ u
    assert rel(ag, ao, ao) <= 1e-13


@pytest.mark.parametrize("model", sg.MODELS)
def test_forces_and_energy_at_deformed_state(model):
    """shell_forces / shell_energy at a random deformed state (all stencils, free and clamped boundaries)."""
    rng = np.random.default_rng(5)
    if model in sg.SHELL_MODELS:
        sc = sg.cylinder_panel(17, model, ny=11, radius=0.8)
    else:
        sc = sg.plate_clamped_x0(17, model=model)
    x = sc.x0 + 0.01 * rng.standard_normal(sc.x0.shape)
    v = 0.1 * rng.standard_normal(sc.x0.shape)
    m = osys.from_scenario(sc, factor=False)
    h = gb.create_from_scenario(sc)
    gb.shell_set_state(h, x, v)
    fg = gb.shell_forces(h)
    fo = osys.forces(m, x)
    assert rel(fg, fo, fo) <= 1e-12
    eg = gb.shell_energy(h)
    eo = np.array(osys.energy(m, x, v))
    np.testing.assert_allclose(eg, eo, rtol=1e-11, atol=1e-300)


def test_cylinder128_shell_models_fp64():
    """128 x 128 cylinder panel (16,641 vertices, 66 chunks, a multi-CTA team), each shell operator, 10 steps."""
    for model in ("ES", "FS", "SS"):
        sc = sg.cylinder_panel(128, model)
        m, h, st, (xg, vg), (xo, vo) = run_both(sc, 10)
        assert rel(xg, xo, xo - sc.x0) <= 1e-10, model


@pytest.mark.parametrize("model", ["ES", "FS", "SS"])
def test_cylinder128_fp32_refine(model):
    """FP32 forces and PCG with FP64 refinement on the 128 x 128 cylinder: solve to refine_rtol = 1e-10;
    the remaining difference to the FP64 oracle is the FP32 rounding of the force (stated bound 1e-6)."""
    sc = sg.cylinder_panel(128, model)
    m, h, st, (xg, vg), (xo, vo) = run_both(sc, 10, precision="fp32_refine", refine_rtol=1e-10)
    assert st["refine_rounds"] >= 1
    assert st["rel_residual"] <= 1e-10
    assert rel(xg, xo, xo - sc.x0) <= 1e-6, model


def test_alone_equals_in_batch_bitwise():
    """An instance's result is bit-identical alone and inside a batch of other instances (both precisions)."""
    scs = sg.mixed_batch(12, seed=9, side_lo=6, side_hi=40, steps=5)
    for prec in ("fp64", "fp32_refine"):
        alone = []
        for sc in scs:
            h = gb.create_from_scenario(sc, precision=prec)
            gb.shell_step(h, 5)
            alone.append(gb.shell_get_state(h))
            gb.shell_destroy(h)
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision=prec) for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        rc, stats = gb.shell_batch_step(b, 5)
        assert rc == 0
        assert all(s["steps_done"] == 5 for s in stats.values())
        for slot in list(b.members):
            gb.shell_batch_retire(b, slot)
        for k, h in enumerate(hs):
            x, v = gb.shell_get_state(h)
            assert np.array_equal(x, alone[k][0]), (prec, k)
            assert np.array_equal(v, alone[k][1]), (prec, k)


def test_not_converged_commits_nothing():
    sc = sg.plate_clamped_x0(12, model="SP")
    h = gb.create_from_scenario(sc, pcg_max_it=1)
    x0, v0 = gb.shell_get_state(h)
    st = gb.shell_step(h, 3, check=False)
    assert st["rc"] == gb.SHELL_ERR_NOT_CONVERGED
    assert st["steps_done"] == 0
    x1, v1 = gb.shell_get_state(h)
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)


def test_invalid_meshes_rejected():
    with pytest.raises(gb.ShellError) as e:
        gb.shell_create([[0, 1, 2], [1, 2, 3]], [[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], "SP", 1e6, 0.3,
                        1e-3, 1000.0)
    assert e.value.code == gb.SHELL_ERR_BAD_ORIENTATION
    xy, tris = sg.grid(2, 2)
    curved = sg.roll_to_cylinder(xy, 0.5, 1.0)
    with pytest.raises(gb.ShellError) as e:
        gb.shell_create(tris, curved, "SP", 1e6, 0.3, 1e-3, 1000.0)   # plate model on a curved rest shape
    assert e.value.code == gb.SHELL_ERR_INVALID_ARG
    with pytest.raises(gb.ShellError) as e:
        gb.shell_create(tris, sg.flat3(xy), "SP", 1e6, 0.3, 1e-3, 1000.0, clamped_edges=[[0, 4]])  # interior edge
    assert e.value.code == gb.SHELL_ERR_INVALID_ARG


def test_full_size_jittered_plate_fp64_step_satisfies_system():
    """512^2-vertex jittered smoothed-hinge plate (E = 1e7, t = 5e-4, dt = 1/60: dt^2 K dominates M by ~4e6,
    the stiffest workload), FP64. After 2 steps, one more step is checked against the oracle's own system at
    that state: the normwise backward error |A v' - b| / (| |A| |v'| | + |b|) <= 1e-13 (PCG stops at a
    relative residual of 1e-13; the recursive residual of CG drifts from the true one by O(eps |A| |v|)), and
    x' = x + dt v'."""
    sc = sg.jittered_plate(512)
    h = gb.create_from_scenario(sc, precision="fp64", pcg_max_it=100000)
    gb.shell_step(h, 2)
    x, v = gb.shell_get_state(h)
    st = gb.shell_step(h, 1)
    x1, v1 = gb.shell_get_state(h)
    m = osys.from_scenario(sc, factor=False)
    A = osys.system_matrix(m)
    b = osys.rhs(m, x, v)
    eta = np.linalg.norm(A @ v1 - b) / (np.linalg.norm(abs(A) @ abs(v1)) + np.linalg.norm(b))
    assert eta <= 1e-13, (eta, st)
    np.testing.assert_allclose(x1, x + sc.dt * v1, rtol=0, atol=1e-15 * np.abs(x).max())


def test_full_size_jittered_plate_fp32_refine_matches_oracle():
    """Same workload in the mode it states: FP32 forces and PCG with FP64 refinement to 1e-6, and the FP64 path,
    against the oracle's trajectory (direct solves) after 1, 3 and 6 steps: rel_x <= 1e-6 for FP32 +
    refinement (measured 1-2e-9) and <= 1e-10 for FP64 (measured 4-5e-11)."""
    sc = sg.jittered_plate(512)
    h64 = gb.create_from_scenario(sc, precision="fp64", pcg_max_it=100000)
    h32 = gb.create_from_scenario(sc, precision="fp32_refine", refine_rtol=1e-6, refine_max=40, pcg_max_it=60000)
    m = osys.from_scenario(sc)
    xo, vo = sc.x0, sc.v0
    done = 0
    for target in (1, 3, 6):
        gb.shell_step(h64, target - done)
        st = gb.shell_step(h32, target - done)
        assert st["rel_residual"] <= 1e-6
        xo, vo = osys.step(m, xo, vo, target - done)
        done = target
        x64, _ = gb.shell_get_state(h64)
        x32, v32 = gb.shell_get_state(h32)
        e64 = rel(x64, xo, xo - sc.rest)
        e32 = rel(x32, xo, xo - sc.rest)
        print(f"jitter512 step {target}: rel_x fp64 {e64:.2e}, fp32_refine {e32:.2e}, rel_v fp32_refine "
              f"{rel(v32, vo, vo):.2e}")
        assert e64 <= 1e-10, (target, e64)
        assert e32 <= 1e-6, (target, e32)


def test_bench_batch_sampled_instances_match_oracle():
    """The benchmark's batch (256 mixed instances, 930,819 vertices, FP32 + refinement with the default
    refinement target) in the benchmark's launch configuration (autotuned) and its step count (53 steps: the
    autotuner's 30, 3 warm-up and 20 timed); sampled instances (the largest, the smallest, one per model) against
    the oracle at every 10th step and at the end: rel_x <= 1e-6 (the per-result error the benchmark states)."""
    scs = sg.mixed_batch(256, seed=4, steps=500)
    b = gb.shell_batch_create(1 << 50)
    hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
    for h in hs:
        gb.shell_batch_admit(b, h)
    tuned = gb.shell_batch_autotune(b, 2)
    done = tuned["steps"]
    sizes = [sc.n_verts for sc in scs]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for model in sg.MODELS:
        pick.add(next(k for k, sc in enumerate(scs) if sc.model == model))
    models = {k: osys.from_scenario(scs[k]) for k in pick}
    states = {k: osys.step(models[k], scs[k].x0, scs[k].v0, done) for k in pick}
    worst = 0.0
    while done < 53:
        n = min(10, 53 - done)
        rc, _ = gb.shell_batch_step(b, n)
        assert rc == 0
        done += n
        for k in sorted(pick):
            sc = scs[k]
            states[k] = osys.step(models[k], states[k][0], states[k][1], n)
            xo = states[k][0]
            xg, _ = gb.shell_get_state(hs[k])
            e = rel(xg, xo, xo - sc.x0)
            worst = max(worst, e)
            assert e <= 1e-6, (k, sc.name, done, e)
    print("bench batch, sampled instances: max rel_x vs the oracle over 53 steps", worst)
    gb.shell_batch_destroy(b)


def test_autotune_changes_speed_not_results():
    """The autotuner re-plans the solve launch on real steps; the states equal an untuned batch bitwise."""
    scs = sg.mixed_batch(10, seed=21, side_lo=6, side_hi=48)
    out = []
    n_tune = None
    for tune in (True, False):
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        if tune:
            info = gb.shell_batch_autotune(b, 1)
            assert info["ctas_per_sm"] >= 1
            n_tune = info["steps"]
            gb.shell_batch_step(b, 2)
        else:
            gb.shell_batch_step(b, n_tune + 2)
        out.append([gb.shell_get_state(h) for h in hs])
        gb.shell_batch_destroy(b)
    for (xa, va), (xb, vb) in zip(*out):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_batch_packed_states_roundtrip():
    """shell_batch_get/set_states move every resident instance's state in one packed copy each way, in slot
    order, identical to the per-handle transfers."""
    scs = sg.mixed_batch(5, seed=33, side_lo=4, side_hi=20)
    b = gb.shell_batch_create(1 << 40)
    hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
    for h in hs:
        gb.shell_batch_admit(b, h)
    gb.shell_batch_step(b, 2)
    slots, offs = gb.shell_batch_state_layout(b)
    x, v = gb.shell_batch_get_states(b)
    for k, slot in enumerate(slots):
        xa, va = gb.shell_get_state(b.members[int(slot)])
        assert np.array_equal(x[offs[k]:offs[k + 1]], xa) and np.array_equal(v[offs[k]:offs[k + 1]], va)
    gb.shell_batch_set_states(b, x + 0.25, v * 2.0)
    for k, slot in enumerate(slots):
        xa, va = gb.shell_get_state(b.members[int(slot)])
        assert np.array_equal(xa, x[offs[k]:offs[k + 1]] + 0.25) and np.array_equal(va, v[offs[k]:offs[k + 1]] * 2.0)
    gb.shell_batch_destroy(b)


def test_batch_step_states_equals_set_step_get():
    """shell_batch_step_states (copies in, steps, copies out, one wait) gives the states and statistics of
    shell_batch_set_states + shell_batch_step + shell_batch_get_states, bitwise; NULL buffers keep the device
    states or copy nothing; zero steps only copy."""
    scs = sg.mixed_batch(6, seed=35, side_lo=4, side_hi=40)
    runs = []
    for fused in (False, True):
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        gb.shell_batch_step(b, 2)
        x, v = gb.shell_batch_get_states(b)
        x, v = np.ascontiguousarray(x * 1.0001), np.ascontiguousarray(v * 0.5)
        if fused:
            xo, vo = np.empty_like(x), np.empty_like(v)
            rc, st = gb.shell_batch_step_states(b, 3, x, v, xo, vo)
            rc2, _ = gb.shell_batch_step_states(b, 2)                  # device states kept, nothing copied
            x2, v2 = np.empty_like(x), np.empty_like(v)
            gb.shell_batch_step_states(b, 0, None, None, x2, v2)        # zero steps: copy out only
        else:
            gb.shell_batch_set_states(b, x, v)
            rc, st = gb.shell_batch_step(b, 3)
            xo, vo = gb.shell_batch_get_states(b)
            rc2, _ = gb.shell_batch_step(b, 2)
            x2, v2 = gb.shell_batch_get_states(b)
        assert rc == 0 and rc2 == 0
        runs.append((xo, vo, x2, v2, {k: (s["steps_done"], s["total_pcg_iterations"]) for k, s in st.items()}))
        gb.shell_batch_destroy(b)
    for a, c in zip(runs[0][:4], runs[1][:4]):
        assert np.array_equal(a, c)
    assert runs[0][4] == runs[1][4]


def test_batch_states_from_page_locked_buffers():
    """Page-locked host buffers are read and written in place by the state kernels (no staging copy); the
    states, statistics and every later step equal those of pageable buffers (staged copies), bitwise: set,
    step and get in one call, in separate calls, and in place (the same buffers in and out)."""
    import torch
    scs = sg.mixed_batch(6, seed=36, side_lo=4, side_hi=40)
    runs = []
    for pinned in (False, True):
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        gb.shell_batch_step(b, 2)
        x0, v0 = gb.shell_batch_get_states(b)

        def buf(a):
            if not pinned:
                return np.array(a)
            t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
            t[...] = a
            return t
        x, v = buf(x0 * 1.0001), buf(v0 * 0.5)
        xo, vo = buf(np.zeros_like(x0)), buf(np.zeros_like(v0))
        rc, st = gb.shell_batch_step_states(b, 3, x, v, xo, vo)
        gb.shell_batch_set_states(b, xo, vo)
        rc2, _ = gb.shell_batch_step(b, 1)
        gb.shell_batch_get_states(b, x, v)
        rc3, _ = gb.shell_batch_step_states(b, 2, x, v, x, v)        # in place
        assert rc == 0 and rc2 == 0 and rc3 == 0
        runs.append((np.array(xo), np.array(vo), np.array(x), np.array(v),
                     {k: (s["steps_done"], s["total_pcg_iterations"]) for k, s in st.items()}))
        gb.shell_batch_destroy(b)
    for a, c in zip(runs[0][:4], runs[1][:4]):
        assert np.array_equal(a, c)
    assert runs[0][4] == runs[1][4]


@pytest.mark.parametrize("case", ["cyl96_SS", "jitter160_SP", "batch6"])
def test_shared_memory_staging_is_bitwise_neutral(case):
    """FP32 products that stage each 256-row block's gathered vector entries in shared memory read the same
    values in the same order as products gathering from global memory: states agree bitwise, through every
    multigrid level (A, P and R lists) and the FP64 refinement."""
    if case == "cyl96_SS":
        scs = [sg.cylinder_panel(96, "SS")]
    elif case == "jitter160_SP":
        scs = [sg.jittered_plate(160, steps=20)]
    else:
        scs = sg.mixed_batch(6, seed=41, side_lo=16, side_hi=72)
    out = []
    for no_staging in (False, True):
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision="fp32_refine", no_staging=no_staging) for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        _, stats = gb.shell_batch_step(b, 6)
        assert all(s["status"] == 0 and s["steps_done"] == 6 for s in stats.values())
        out.append([gb.shell_get_state(h) for h in hs])
        levels = [gb.shell_info(h)["amg_levels"] for h in hs]
        gb.shell_batch_destroy(b)
    assert max(levels) >= 3     # the multigrid path (coarse lists) is exercised
    for (xa, va), (xb, vb) in zip(*out):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_state_round_trip_leaves_steps_bitwise_unchanged():
    """Reading the states and writing them back between steps (packed batch transfer, or per handle) changes
    nothing: the next steps equal those of an untouched batch bitwise (the warm start's velocity history is
    kept)."""
    scs = sg.mixed_batch(4, seed=52, side_lo=6, side_hi=30)
    out = []
    for round_trip in (False, True):
        b = gb.shell_batch_create(1 << 40)
        hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
        for h in hs:
            gb.shell_batch_admit(b, h)
        for _ in range(4):
            if round_trip:
                x, v = gb.shell_batch_get_states(b)
                gb.shell_batch_set_states(b, x, v)
                xa, va = gb.shell_get_state(hs[0])
                gb.shell_set_state(hs[0], xa, va)
            gb.shell_batch_step(b, 1)
        out.append([gb.shell_get_state(h) for h in hs])
        gb.shell_batch_destroy(b)
    for (xa, va), (xb, vb) in zip(*out):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
