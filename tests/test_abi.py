"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every entry point
that include/shell.h declares, and refuses to compute without a GB300 (no CPU fallback)."""
import os
import re

import pytest

import paper_2502_10872_gb300 as gb
from paper_2502_10872_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        gb.build()
    return gb.load_library()


def header_functions():
    src = open(os.path.join(ROOT, "include", "shell.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shell_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_api():
    names = header_functions()
    for n in ("shell_create", "shell_step", "shell_energy", "shell_forces", "shell_destroy", "shell_batch_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(binding.EXPORTS)


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gb.ShellError) as e:
        gb.shell_create([[0, 1, 2]], [[0, 0, 0], [1, 0, 0], [0, 1, 0]], "SP", 1e6, 0.3, 1e-3, 1000.0,
                        use_torch_allocator=False)
    assert e.value.code == gb.SHELL_ERR_NO_DEVICE


def test_options_defaults(lib):
    o = gb.make_options(use_torch_allocator=False, stream=0)
    assert o.dt == 1e-2 and o.pcg_max_it == 20000 and o.refine_max == 20
    assert lib.shell_strerror(gb.SHELL_ERR_NOT_CONVERGED).decode().startswith("linear solve")


def test_binding_structs_match_header_layout():
    import ctypes as C
    # shell_options: double, int32(+pad), double, double, int32, int32, 4 pointers
    assert C.sizeof(binding.shell_options) == 8 + 8 + 8 + 8 + 4 + 4 + 4 * 8 + 8
    assert C.sizeof(binding.shell_step_stats) == 4 * 4 + 8 + 8 + 8 + 8 + 8
    assert C.sizeof(binding.shell_bc) == 8 + 8 + 8 + 24 + 8 + 8 + 8 + 8


def test_binding_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field offset and struct size of the ctypes mirrors equals the C compiler's for include/shell.h."""
    import ctypes as C
    import shutil
    import subprocess
    from pathlib import Path
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"shell_mesh": binding.shell_mesh, "shell_material": binding.shell_material,
               "shell_bc": binding.shell_bc, "shell_options": binding.shell_options,
               "shell_step_stats": binding.shell_step_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "shell.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    inc = Path(__file__).resolve().parents[1] / "include"
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", str(inc), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_batch_stats_mapping():
    """The per-call batch statistics are a read-only mapping over the resident slots (ascending), each slot's
    fields read from the C array when first accessed; slots outside the batch are absent."""
    arr = (binding.shell_step_stats * 8)()
    for k in range(8):
        arr[k].steps_done = k
        arr[k].total_pcg_iterations = 10 * k
    st = binding.BatchStats(arr, (1, 4, 6))
    assert list(st) == [1, 4, 6] and len(st) == 3
    assert st[4]["steps_done"] == 4 and st[6]["total_pcg_iterations"] == 60
    assert 2 not in st and st.get(2) is None
    with pytest.raises(KeyError):
        st[0]
    assert [s["steps_done"] for s in st.values()] == [1, 4, 6]
    assert dict(st.items())[1]["status"] == 0
    assert st[4] is st[4]   # built once
    assert st.raw(6).total_pcg_iterations == 60 and st.raw(2) is None


def test_batch_resident_slots_follow_membership():
    assert "__del__" in binding.Batch.__dict__   # a collected batch frees its device memory
    b = binding.Batch(None, None)
    b.members = {5: None, 2: None}
    assert b.resident_slots() == (2, 5)
    b.members[0] = None
    b._changed()
    assert b.resident_slots() == (0, 2, 5)
