"""shell_step_noalloc: the step entry point for callers that cannot allocate device memory after set-up
(a frozen allocator in a real-time loop, or a host framework that owns the device-memory budget). Its launch
scratch is a static device array instead of tables allocated on first use. This file is collected last, so a
run that stops at the first failure has run every other test before it."""
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


def rel(a, b, ref):
    return np.linalg.norm(a - b) / max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("precision,case", [("fp64", "plate"), ("fp32_refine", "cylinder")])
def test_noalloc_step_matches_shell_step(precision, case):
    sc = (sg.plate_clamped_x0(40, model="SP") if case == "plate"
          else sg.cylinder_panel(60, "FS", ny=45, dt=5e-3))     # 1,681 / 2,806 vertices: multi-CTA teams
    ref = gb.create_from_scenario(sc, precision=precision)
    new = gb.create_from_scenario(sc, precision=precision)
    for call in range(2):                                        # two calls in a row share the static array
        a = gb.shell_step(ref, 4)
        b = gb.shell_step_noalloc(new, 4)
        assert b["rc"] == 0 and b["steps_done"] == 4
        assert b["total_pcg_iterations"] == a["total_pcg_iterations"]
        xa, va = gb.shell_get_state(ref)
        xb, vb = gb.shell_get_state(new)
        assert rel(xb, xa, xa - sc.rest) <= 1e-10, call
        assert rel(vb, va, va) <= 1e-10, call
        # results do not depend on the launch's team size or scratch placement: the states agree bitwise
        assert np.array_equal(xb, xa) and np.array_equal(vb, va), call
