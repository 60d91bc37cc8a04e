"""Build the in-tree CUDA library ``libshells.so`` for sm_103a (nvcc + g++, no cmake).

The translation units compile in parallel; the result is placed next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libshells.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CU = ["kernels_setup.cu", "kernels_force.cu", "kernels_solve.cu"]
CPP = ["host_mesh.cpp", "amg_setup.cpp", "halo.cpp", "api.cpp"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    ch = cuda_home()
    nvcc = os.path.join(ch, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I" + os.path.join(ch, "include"), "-I" + CSRC]
    jobs = []
    for f in CU:
        o = os.path.join(OUT_DIR, f + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
               "-c", os.path.join(CSRC, f), "-o", o] + inc
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, o))
    for f in CPP:
        o = os.path.join(OUT_DIR, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o] + inc
        jobs.append((cmd, o))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose or ptxas_info:
        for (cmd, _), out in zip(jobs, outs):
            if out.strip():
                print(out)
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp] + [o for _, o in jobs] + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
