"""Continuous batching (paper_2502_10872_gb300.serving): requests admitted by an HBM budget while others are
stepping give the same result as alone (bitwise: reductions do not depend on the co-resident instances)."""
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


def make_requests(n, seed=3):
    from paper_2502_10872_gb300.serving import Request
    rng = np.random.default_rng(seed)
    scs = sg.mixed_batch(n, seed=seed, side_lo=5, side_hi=36)
    reqs, t = [], 0.0
    for k, sc in enumerate(scs):
        t += float(rng.exponential(0.002))
        reqs.append(Request(k, t, sc, int(rng.integers(2, 9))))
    return reqs


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_served_results_equal_alone(precision):
    from paper_2502_10872_gb300.serving import Server
    reqs = make_requests(8)
    srv = Server(budget_bytes=1 << 40, precision=precision, keep_states=True)
    rep = srv.run(reqs)
    srv.close()
    s = rep.summary()
    assert s["completed"] == len(reqs) and s["failed"] == 0
    for r in reqs:
        h = gb.create_from_scenario(r.scenario, precision=precision)
        gb.shell_step(h, r.steps)
        x, v = gb.shell_get_state(h)
        assert r.done_steps == r.steps
        assert np.array_equal(x, r.final_state[0]), r.rid
        assert np.array_equal(v, r.final_state[1]), r.rid
        gb.shell_destroy(h)


def test_budget_limits_residency():
    from paper_2502_10872_gb300.serving import Server
    reqs = make_requests(6, seed=5)
    sizes = []
    for r in reqs:
        h = gb.create_from_scenario(r.scenario, precision="fp32_refine")
        sizes.append(gb.shell_info(h)["device_bytes"])
        gb.shell_destroy(h)
    budget = sorted(sizes)[-1] + sorted(sizes)[-2]          # at most two of the largest at once
    srv = Server(budget_bytes=budget, precision="fp32_refine")
    rep = srv.run(reqs)
    srv.close()
    assert rep.summary()["completed"] == len(reqs)
    # an instance larger than the whole budget is refused with SHELL_ERR_BUDGET
    b = gb.shell_batch_create(1024)
    h = gb.create_from_scenario(reqs[0].scenario)
    assert gb.shell_batch_admit(b, h, check=False) == gb.SHELL_ERR_BUDGET
    gb.shell_batch_destroy(b)
