"""Host set-up of the multigrid preconditioner (no GPU): the transfer operators with the damped-Jacobi sweeps
folded in (Rs = R (I - omega A D^-1), Ps = Rs^T), which let the solve kernel run a level in two team phases,
give the same V(1,1) cycle as the plain sequence of pre-smoothing, residual, restriction, coarse correction
and post-smoothing. Built from the library's own set-up source (tests/amg_host_check.cpp) and run on the
constant step matrices of plate and shell scenes (assembled by the oracle, used here only as SPD inputs of
the right structure)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import shellgen as sg
from oracle import system as osys

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("amg") / "amg_host_check")
    subprocess.run([gxx, "-O1", "-std=c++17", "-o", exe, os.path.join(HERE, "amg_host_check.cpp")], check=True)
    return exe


def write_csr(path, A):
    A = A.tocsr()
    A.sort_indices()
    with open(path, "wb") as f:
        np.array([A.shape[0], A.nnz], dtype=np.int32).tofile(f)
        A.indptr.astype(np.int32).tofile(f)
        A.indices.astype(np.int32).tofile(f)
        A.data.astype(np.float64).tofile(f)


def scenes():
    yield "plate EP 40", sg.plate_clamped_x0(40, model="EP")
    yield "cylinder SS 32", sg.cylinder_panel(32, "SS")
    yield "jittered SP 48", sg.jittered_plate(48, steps=1)
    yield "plate FP 130", sg.plate_clamped_x0(130, model="FP")   # 17,161 rows: the threaded set-up path
    for k, sc in enumerate(sg.mixed_batch(3, seed=9, side_lo=20, side_hi=40)):
        yield f"mixed {k} {sc.model}", sc


@pytest.mark.parametrize("name,sc", list(scenes()), ids=lambda v: v if isinstance(v, str) else "")
def test_folded_transfers_give_the_plain_cycle(checker, tmp_path, name, sc):
    m = osys.from_scenario(sc, factor=False)
    path = str(tmp_path / "A.bin")
    write_csr(path, osys.system_matrix(m))
    out = subprocess.run([checker, path], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("OK"), out.stdout
