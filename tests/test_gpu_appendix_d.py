"""App. D's world-frame edge-hinge models on the GPU: the EP and ES force kernels against the oracle's QTP and
QTS energies and gradients (written from App. D's world-frame operator, not from the corotational one), on
deformed free meshes, through the C ABI (shell_forces, shell_energy). The CPU tests pin QTP = EP and QTS = ES
exactly; this checks that the CUDA kernels compute those energies and forces (bar 1e-12, FP64)."""
import numpy as np
import pytest

import shellgen as sg
from oracle import appendix_d as ad
from oracle import operators as op
from oracle import system as osys
from oracle.energies import frame_normal, membrane_energy_force

gb = pytest.importorskip("paper_2502_10872_gb300")
pytestmark = pytest.mark.gpu

E, NU, T, RHO = 2e6, 0.3, 1.5e-3, 1000.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.load_library()


@pytest.mark.parametrize("model", ["EP", "ES"])
def test_edge_hinge_kernels_match_world_frame_qtp_qts(model):
    nx, ny = 37, 23                                        # 912 vertices: several force tiles, ragged tail
    if model == "EP":
        xy, tris = sg.grid(nx, ny)
        rest = sg.flat3(sg.jitter(xy, 1.0 / nx, 0.15, sg.grid_interior_mask(nx, ny), 3))
    else:
        width = 0.6 * np.pi / 2
        xy, tris = sg.grid(nx, ny, 1.0, width)
        rest = sg.roll_to_cylinder(xy, 0.6, width)
    rng = np.random.default_rng(17)
    x = rest + 2e-3 * rng.standard_normal(rest.shape)
    m = osys.build_model(tris, rest, model, E, NU, T, RHO, 1e-2, factor=False)
    st = m.stencils[0]
    assert st.kind == "edge" and np.all(st.idx >= 0)
    kb = op.bending_rigidity(E, NU, T)
    if model == "EP":
        eb, gb_ = ad.qtp_energy_gradient(x, st.idx, st.rest, kb, signed=True)
    else:
        eb, gb_ = ad.qts_energy_gradient(x, st.idx, st.rest, kb, lambda xs: frame_normal(xs, "edge"), signed=True)
    em, fm = membrane_energy_force(x[m.tris], m.Dm_inv, m.tri_area, E, NU, T)
    f = np.zeros_like(x)
    np.add.at(f, m.tris.ravel(), fm.reshape(-1, 3))
    np.add.at(f, st.idx, -gb_)
    h = gb.shell_create(tris, rest, model, E, NU, T, RHO, init_xyz=x)
    fg = gb.shell_forces(h)
    eg = gb.shell_energy(h)
    assert np.linalg.norm(fg - f) <= 1e-12 * np.linalg.norm(f)
    assert abs(eg[1] - eb.sum()) <= 1e-12 * eb.sum()
    assert abs(eg[0] - em.sum()) <= 1e-12 * em.sum()
    gb.shell_destroy(h)
