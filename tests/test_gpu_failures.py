"""Failure detection on the GPU, in the forms that fault nothing: failures are made on the host (a non-finite
state set through the C ABI) or by a device-side wait that runs out (a team-barrier wait bound of 1 ns), and
the tests check the status the host reads, that nothing is committed, and that the next steps are normal.

* NaN in the state -> SHELL_ERR_NONFINITE, the state is left as set, steps_done 0; a finite state clears the
  failure and stepping resumes.
* One instance of a batch fails (NaN) while the others step: the batch returns the first error, the failed
  slot reports it with no committed step, the others commit every step, bitwise equal to stepping alone.
* A team barrier whose wait bound is exceeded -> SHELL_ERR_TIMEOUT on a multi-CTA instance: the abandoned
  launches commit nothing (state bitwise unchanged), and after restoring the default bound the next steps
  equal those of an instance that never timed out, bitwise.
"""
import numpy as np
import pytest

import shellgen as sg

gb = pytest.importorskip("paper_2502_10872_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.load_library()


def _free_vertex(sc):
    pinned = np.asarray(sc.pinned).astype(bool)
    return int(np.flatnonzero(~pinned)[len(pinned) // 3])


@pytest.mark.parametrize("precision,which", [("fp64", "x"), ("fp32_refine", "x"), ("fp32_refine", "v")])
def test_nonfinite_state_is_reported_and_not_committed(precision, which):
    sc = sg.cylinder_panel(24, "SS", ny=18)
    h = gb.create_from_scenario(sc, precision=precision)
    gb.shell_step(h, 2)
    x, v = gb.shell_get_state(h)
    bad_x, bad_v = x.copy(), v.copy()
    k = _free_vertex(sc)
    (bad_x if which == "x" else bad_v)[k, 1] = np.nan
    gb.shell_set_state(h, bad_x, bad_v)
    st = gb.shell_step(h, 3, check=False)
    assert st["rc"] == gb.SHELL_ERR_NONFINITE and st["steps_done"] == 0 and st["status"] == gb.SHELL_ERR_NONFINITE
    xs, vs = gb.shell_get_state(h)
    assert np.array_equal(xs, bad_x, equal_nan=True) and np.array_equal(vs, bad_v, equal_nan=True)
    # a finite state clears the failure; the next steps are those of a handle that never failed
    gb.shell_set_state(h, x, v)
    st = gb.shell_step(h, 2)
    assert st["steps_done"] == 2
    ref = gb.create_from_scenario(sc, precision=precision)
    gb.shell_step(ref, 4)
    xa, va = gb.shell_get_state(ref)
    xb, vb = gb.shell_get_state(h)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_one_failing_instance_leaves_the_batch_stepping():
    scs = [sg.plate_clamped_x0(20, model="FP"), sg.cylinder_panel(16, "ES"), sg.cylinder_panel(30, "SS", ny=20)]
    alone = []
    for sc in scs:
        h = gb.create_from_scenario(sc, precision="fp32_refine")
        gb.shell_step(h, 3)
        alone.append(gb.shell_get_state(h))
    hs = [gb.create_from_scenario(sc, precision="fp32_refine") for sc in scs]
    x1 = scs[1].x0.copy()
    x1[_free_vertex(scs[1]), 2] = np.inf
    gb.shell_set_state(hs[1], x1, None)
    b = gb.shell_batch_create(1 << 40)
    slots = [gb.shell_batch_admit(b, h) for h in hs]
    rc, stats = gb.shell_batch_step(b, 3, check=False)
    assert rc == gb.SHELL_ERR_NONFINITE
    assert stats[slots[1]]["status"] == gb.SHELL_ERR_NONFINITE and stats[slots[1]]["steps_done"] == 0
    for k in (0, 2):
        assert stats[slots[k]]["status"] == 0 and stats[slots[k]]["steps_done"] == 3
    for k in (0, 2):
        gb.shell_batch_retire(b, slots[k])
        xs, vs = gb.shell_get_state(hs[k])
        assert np.array_equal(xs, alone[k][0]) and np.array_equal(vs, alone[k][1]), k
    gb.shell_batch_destroy(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_team_barrier_timeout_commits_nothing_and_recovers(precision):
    sc = sg.cylinder_panel(96, "FS", ny=96)                 # 9,409 vertices: a multi-CTA team
    ref = gb.create_from_scenario(sc, precision=precision)
    h = gb.create_from_scenario(sc, precision=precision)
    b = gb.shell_batch_create(1 << 40)
    slot = gb.shell_batch_admit(b, h)
    rc, stats = gb.shell_batch_step(b, 2)
    assert rc == 0 and stats[slot]["team_ctas"] > 1
    x, v = gb.shell_batch_get_states(b)
    gb.shell_batch_set_wait_limit(b, 1)                      # 1 ns: the first CTA that waits at a barrier gives up
    rc, stats = gb.shell_batch_step(b, 3, check=False)
    assert rc == gb.SHELL_ERR_TIMEOUT
    assert stats[slot]["steps_done"] == 0
    xt, vt = gb.shell_batch_get_states(b)
    assert np.array_equal(xt, x) and np.array_equal(vt, v)
    gb.shell_batch_set_wait_limit(b, 0)                      # back to the default bound
    rc, stats = gb.shell_batch_step(b, 2)
    assert rc == 0 and stats[slot]["steps_done"] == 2
    gb.shell_step(ref, 4)
    xa, va = gb.shell_get_state(ref)
    xb, vb = gb.shell_batch_get_states(b)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    gb.shell_batch_destroy(b)
