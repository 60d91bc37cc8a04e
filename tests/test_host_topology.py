"""Host-side stencil and matrix-structure logic of the library (no GPU): every index in range, counts equal
to the oracle's independent topology, nonzero pattern equal to the oracle's matrix pattern."""
import numpy as np
import pytest

import shellgen as sg
import paper_2502_10872_gb300 as gb
from oracle import system as osys
from oracle.topology import build_stencils


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    from paper_2502_10872_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        gb.build()
    gb.load_library()


def scenes():
    yield sg.plate_clamped_x0(7)
    yield sg.cylinder_panel(9, "SS", ny=5)
    xy, tris = sg.equilateral_grid(6, 5, 0.2)
    yield sg.Scenario("equi", tris, sg.flat3(xy), sg.flat3(xy), np.zeros((xy.shape[0], 3)), "SP", 1e6, 0.3, 1e-3,
                      1000.0, np.zeros(xy.shape[0], np.uint8), np.zeros((0, 2), np.int32), (0, 0, 0),
                      np.zeros(0, np.int32), np.zeros((0, 3)), 1e-2, 1)
    yield sg.jittered_plate(40, steps=1)
    for sc in sg.mixed_batch(6, seed=3, side_lo=3, side_hi=20):
        yield sc


@pytest.mark.parametrize("model", sg.MODELS)
def test_topology_matches_oracle(model):
    for sc in scenes():
        s = gb.shell_topology_summary(sc.tris, sc.n_verts, model, sc.clamped_edges)
        assert s["bad_indices"] == 0
        topo = build_stencils(sc.tris, sc.n_verts, sc.clamped_edges)
        if model[0] == "E":
            assert s["edge_stencils"] == len(topo["edge"])
            assert s["clamped_edge_stencils"] == len(topo["edge_clamped"])
            assert s["n_slots"] == 3 * sc.n_tris + 4 * (len(topo["edge"]) + len(topo["edge_clamped"]))
        else:
            assert s["virtual_tri_stencils"] == int(np.sum(np.any(topo["tri"][:, 3:] < 0, axis=1)))
            assert s["n_slots"] == 6 * sc.n_tris
        rest = sc.rest if model in sg.SHELL_MODELS or np.ptp(sc.rest[:, 2]) == 0 else sc.x0
        if model in sg.PLATE_MODELS and np.ptp(sc.rest[:, 2]) > 0:
            continue
        m = osys.build_model(sc.tris, sc.rest, model, 1e6, 0.3, 1e-3, 1000.0, 1e-2,
                             clamped_edges=sc.clamped_edges, factor=False)
        Kb, Km = osys.stiffness_matrices(m)
        pattern = (abs(Kb) + abs(Km) + __import__("scipy.sparse", fromlist=["eye"]).eye(sc.n_verts)).tocsr()
        pattern.eliminate_zeros()
        # structural nonzeros may exceed numerical ones only where entries cancel exactly
        assert s["nnz"] >= pattern.nnz
        assert s["nnz"] - pattern.nnz <= 0.02 * s["nnz"]
        assert s["nnz_stored"] >= s["nnz"]


def test_topology_errors():
    with pytest.raises(gb.ShellError) as e:
        gb.shell_topology_summary([[0, 1, 2], [0, 1, 3]], 4, "SP")
    assert e.value.code == gb.SHELL_ERR_BAD_ORIENTATION
    with pytest.raises(gb.ShellError) as e:
        gb.shell_topology_summary([[0, 1, 2], [1, 0, 3], [0, 1, 4]], 5, "SP")
    assert e.value.code == gb.SHELL_ERR_NON_MANIFOLD
    with pytest.raises(gb.ShellError) as e:
        gb.shell_topology_summary([[0, 1, 5]], 4, "SP")
    assert e.value.code == gb.SHELL_ERR_INVALID_ARG
    with pytest.raises(gb.ShellError):
        gb.shell_topology_summary([[0, 1, 2], [2, 1, 3]], 4, "EP", clamped_edges=[[1, 2]])   # interior edge
