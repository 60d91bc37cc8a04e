"""ctypes binding of the C ABI in ``include/shell.h`` (argument marshalling only).

Every function here forwards to the CUDA library ``libshells.so`` built in-tree by
``paper_2502_10872_gb300._build``; there is no CPU implementation behind it. If the library is missing the
import of a function raises :class:`LibraryNotBuilt`; without a GB300 the calls return
``SHELL_ERR_NO_DEVICE`` (raised as :class:`ShellError`).

Device memory is allocated through PyTorch's caching allocator when PyTorch with CUDA is available (the
library's allocator hooks), and work runs on PyTorch's current stream unless a stream is given.
"""
from __future__ import annotations

import ctypes as C
import os
from collections.abc import Mapping
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshells.so")

SHELL_OK = 0
ERRORS = {
    -1: "SHELL_ERR_INVALID_ARG", -2: "SHELL_ERR_NON_MANIFOLD", -3: "SHELL_ERR_BAD_ORIENTATION",
    -4: "SHELL_ERR_DEGENERATE", -5: "SHELL_ERR_SINGULAR_OPERATOR", -6: "SHELL_ERR_OOM", -7: "SHELL_ERR_BUDGET",
    -8: "SHELL_ERR_NOT_CONVERGED", -9: "SHELL_ERR_NONFINITE", -10: "SHELL_ERR_TIMEOUT", -11: "SHELL_ERR_CUDA",
    -12: "SHELL_ERR_NO_DEVICE", -13: "SHELL_ERR_BUSY", -14: "SHELL_ERR_STATIC_LIMIT",
}
for _c, _n in ERRORS.items():
    globals()[_n] = _c
MODELS = {"EP": 0, "ES": 1, "FP": 2, "FS": 3, "SP": 4, "SS": 5}
PRECISIONS = {"fp64": 0, "fp32_refine": 1}
PRECONDITIONERS = {"auto": 0, "jacobi": 1, "amg": 2}

# symbols declared in include/shell.h
EXPORTS = (
    "shell_default_options", "shell_strerror", "shell_create", "shell_step", "shell_step_noalloc",
    "shell_set_nonlinear", "shell_energy",
    "shell_forces",
    "shell_apply_matrix", "shell_get_state", "shell_set_state", "shell_get_state_device", "shell_set_state_device", "shell_info",
    "shell_destroy", "shell_topology_summary", "shell_batch_create", "shell_batch_admit", "shell_batch_retire", "shell_batch_step",
    "shell_batch_capacity", "shell_batch_step_times", "shell_batch_set_profiling", "shell_batch_kernel_times",
    "shell_batch_autotune", "shell_batch_set_launch", "shell_batch_get_states", "shell_batch_set_states",
    "shell_batch_step_states",
    "shell_batch_state_layout", "shell_batch_set_wait_limit", "shell_set_newton", "shell_solve_static",
    "shell_batch_destroy",
)


class LibraryNotBuilt(RuntimeError):
    pass


class ShellError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"{ERRORS.get(code, code)}: {_strerror(code)}"
        super().__init__(f"{what}: {msg}" if what else msg)


# ------------------------------------------------------------------------------------------ structs
class shell_mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("tris", C.c_void_p), ("rest_xyz", C.c_void_p),
                ("init_xyz", C.c_void_p), ("init_vel", C.c_void_p)]


class shell_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("thickness", C.c_double), ("density", C.c_double)]


class shell_bc(C.Structure):
    _fields_ = [("pinned", C.c_void_p), ("n_clamped", C.c_int32), ("clamped_edges", C.c_void_p),
                ("gravity", C.c_double * 3), ("n_loads", C.c_int32), ("load_vtx", C.c_void_p),
                ("load_f", C.c_void_p), ("fixed_dofs", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class shell_options(C.Structure):
    _fields_ = [("dt", C.c_double), ("precision", C.c_int32), ("pcg_rtol", C.c_double),
                ("refine_rtol", C.c_double), ("pcg_max_it", C.c_int32), ("refine_max", C.c_int32),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("preconditioner", C.c_int32), ("no_staging", C.c_int32)]


class shell_step_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int32), ("pcg_iterations", C.c_int32), ("refine_rounds", C.c_int32),
                ("status", C.c_int32), ("total_pcg_iterations", C.c_int64), ("rel_residual", C.c_double),
                ("total_refine_rounds", C.c_int64), ("last_solve_us", C.c_double), ("team_ctas", C.c_int32),
                ("nl_iterations", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# ------------------------------------------------------------------------------------------ loading
_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libshells.so`` (raises :class:`LibraryNotBuilt` if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LibraryNotBuilt(f"{path} not found: run paper_2502_10872_gb300._build.build() (nvcc, sm_103a)")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "shell_default_options": (None, [C.POINTER(shell_options)]),
        "shell_strerror": (C.c_char_p, [C.c_int]),
        "shell_create": (C.c_int, [C.POINTER(shell_mesh), C.POINTER(shell_material), C.c_int32, C.POINTER(shell_bc),
                                   C.POINTER(shell_options), C.POINTER(P)]),
        "shell_step": (C.c_int, [P, C.c_int32, C.POINTER(shell_step_stats)]),
        "shell_step_noalloc": (C.c_int, [P, C.c_int32, C.POINTER(shell_step_stats)]),
        "shell_set_nonlinear": (C.c_int, [P, C.c_int32, C.c_double]),
        "shell_energy": (C.c_int, [P, P]),
        "shell_forces": (C.c_int, [P, P]),
        "shell_apply_matrix": (C.c_int, [P, P, P]),
        "shell_get_state": (C.c_int, [P, P, P]),
        "shell_set_state": (C.c_int, [P, P, P]),
        "shell_get_state_device": (C.c_int, [P, P, P]),
        "shell_set_state_device": (C.c_int, [P, P, P]),
        "shell_info": (C.c_int, [P, P]),
        "shell_destroy": (C.c_int, [P]),
        "shell_topology_summary": (C.c_int, [C.c_int32, C.c_int32, P, C.c_int32, P, C.c_int32, P]),
        "shell_batch_create": (C.c_int, [C.POINTER(shell_options), C.c_size_t, C.POINTER(P)]),
        "shell_batch_admit": (C.c_int, [P, P, C.POINTER(C.c_int32)]),
        "shell_batch_retire": (C.c_int, [P, C.c_int32]),
        "shell_batch_step": (C.c_int, [P, C.c_int32, C.POINTER(shell_step_stats)]),
        "shell_batch_capacity": (C.c_int, [P]),
        "shell_batch_step_times": (C.c_int, [P, P, C.c_int32]),
        "shell_batch_set_profiling": (C.c_int, [P, C.c_int32]),
        "shell_batch_kernel_times": (C.c_int, [P, P]),
        "shell_batch_autotune": (C.c_int, [P, C.c_int32, P, P]),
        "shell_batch_set_launch": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32]),
        "shell_batch_get_states": (C.c_int, [P, P, P]),
        "shell_batch_set_states": (C.c_int, [P, P, P]),
        "shell_batch_step_states": (C.c_int, [P, C.c_int32, P, P, P, P, C.POINTER(shell_step_stats)]),
        "shell_batch_state_layout": (C.c_int, [P, P, P]),
        "shell_batch_set_wait_limit": (C.c_int, [P, C.c_int64]),
        "shell_set_newton": (C.c_int, [P, C.c_int32]),
        "shell_solve_static": (C.c_int, [P, C.c_double, C.c_double, C.c_int32, P]),
        "shell_batch_destroy": (C.c_int, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load_library().shell_strerror(code).decode()
    except LibraryNotBuilt:
        return ERRORS.get(code, str(code))


def _check(code: int, what: str):
    if code != SHELL_OK:
        raise ShellError(code, what)


# ------------------------------------------------------------------------------------------ allocator
_torch_hooks = None


def _torch_allocator():
    """(alloc, free) ctypes callbacks into PyTorch's CUDA caching allocator, or None."""
    global _torch_hooks
    if _torch_hooks is not None:
        return _torch_hooks
    try:
        import torch
        if not torch.cuda.is_available():
            return None
    except Exception:
        return None

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    return _torch_hooks


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def make_options(dt=1e-2, precision="fp64", pcg_rtol=0.0, refine_rtol=0.0, pcg_max_it=20000, refine_max=20,
                 stream: Optional[int] = None, use_torch_allocator: bool = True,
                 preconditioner="auto", no_staging: bool = False) -> shell_options:
    lib = load_library()
    o = shell_options()
    lib.shell_default_options(C.byref(o))
    o.dt = float(dt)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.pcg_rtol = float(pcg_rtol)
    o.refine_rtol = float(refine_rtol)
    o.pcg_max_it = int(pcg_max_it)
    o.refine_max = int(refine_max)
    o.preconditioner = PRECONDITIONERS[preconditioner] if isinstance(preconditioner, str) else int(preconditioner)
    o.no_staging = 1 if no_staging else 0
    o.cuda_stream = _current_stream() if stream is None else int(stream)
    hooks = _torch_allocator() if use_torch_allocator else None
    if hooks:
        o.alloc, o.free = hooks
    return o


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _arr(a, dtype, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ------------------------------------------------------------------------------------------ handle API
class Handle:
    """Owning wrapper of a ``shell_handle*``."""

    def __init__(self, ptr, n_verts, opts, keep):
        self.ptr = ptr
        self.n_verts = n_verts
        self._opts = opts
        self._keep = keep

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                load_library().shell_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def shell_create(tris, rest, model, E, nu, thickness, density, *, init_xyz=None, init_vel=None, pinned=None,
                 clamped_edges=None, gravity=(0.0, 0.0, 0.0), load_vtx=None, load_f=None, fixed_dofs=None, dt=1e-2,
                 precision="fp64", pcg_rtol=0.0, refine_rtol=0.0, pcg_max_it=20000, refine_max=20,
                 stream=None, use_torch_allocator=True, preconditioner="auto", no_staging=False) -> Handle:
    """shell_create: rest-state precompute and constant-matrix assembly on the GPU (see include/shell.h)."""
    lib = load_library()
    tris = _arr(tris, np.int32, (-1, 3))
    rest = _arr(rest, np.float64, (-1, 3))
    V = rest.shape[0]
    x0 = _arr(init_xyz, np.float64, (V, 3))
    v0 = _arr(init_vel, np.float64, (V, 3))
    pin = _arr(pinned, np.uint8, (V,))
    fd = _arr(fixed_dofs, np.uint8, (V,))
    ce = _arr(clamped_edges, np.int32, (-1, 2)) if clamped_edges is not None else np.zeros((0, 2), np.int32)
    lv = _arr(load_vtx, np.int32, (-1,)) if load_vtx is not None else np.zeros((0,), np.int32)
    lf = _arr(load_f, np.float64, (-1, 3)) if load_f is not None else np.zeros((0, 3), np.float64)
    mesh = shell_mesh(V, tris.shape[0], _ptr(tris), _ptr(rest), _ptr(x0), _ptr(v0))
    mat = shell_material(E, nu, thickness, density)
    bc = shell_bc()
    bc.pinned = _ptr(pin)
    bc.n_clamped = ce.shape[0]
    bc.clamped_edges = _ptr(ce) if ce.shape[0] else None
    bc.gravity = (C.c_double * 3)(*[float(g) for g in gravity])
    bc.n_loads = lv.shape[0]
    bc.load_vtx = _ptr(lv) if lv.shape[0] else None
    bc.load_f = _ptr(lf) if lv.shape[0] else None
    bc.fixed_dofs = _ptr(fd)
    opts = make_options(dt, precision, pcg_rtol, refine_rtol, pcg_max_it, refine_max, stream, use_torch_allocator,
                        preconditioner, no_staging)
    out = C.c_void_p()
    m = MODELS[model] if isinstance(model, str) else int(model)
    _check(lib.shell_create(C.byref(mesh), C.byref(mat), m, C.byref(bc), C.byref(opts), C.byref(out)), "shell_create")
    return Handle(out.value, V, opts, None)


def create_from_scenario(sc, precision="fp64", **kw) -> Handle:
    """shell_create from any object with the fields of a generated scenario (tris, rest, x0, v0, model, E, nu,
    thickness, density, pinned, clamped_edges, gravity, load_vtx, load_f, dt; fixed_dofs if present)."""
    return shell_create(sc.tris, sc.rest, sc.model, sc.E, sc.nu, sc.thickness, sc.density, init_xyz=sc.x0,
                        init_vel=sc.v0, pinned=sc.pinned, clamped_edges=sc.clamped_edges, gravity=sc.gravity,
                        load_vtx=sc.load_vtx, load_f=sc.load_f, fixed_dofs=getattr(sc, "fixed_dofs", None),
                        dt=sc.dt, precision=precision, **kw)


def shell_step(h: Handle, n_steps: int = 1, check: bool = True) -> dict:
    st = shell_step_stats()
    rc = load_library().shell_step(h.ptr, int(n_steps), C.byref(st))
    if check:
        _check(rc, "shell_step")
    d = st.as_dict()
    d["rc"] = rc
    return d


def shell_set_nonlinear(h: Handle, max_iters: int, rtol: float = 1e-8):
    """Exact backward Euler by chord iteration: up to max_iters solves per step (<= 1: linearised step)."""
    _check(load_library().shell_set_nonlinear(h.ptr, int(max_iters), float(rtol)), "shell_set_nonlinear")


def shell_set_newton(h: Handle, on: bool = True):
    """Newton iterations (tangent of the corotated membrane) for the handle's exact backward-Euler steps."""
    _check(load_library().shell_set_newton(h.ptr, 1 if on else 0), "shell_set_newton")


def shell_solve_static(h: Handle, eps_f: float = 1e-3, eps_u: float = 0.1, max_iters: int = 1000,
                       check: bool = True) -> dict:
    """Quasi-static equilibrium (Eq. 64) by Newton-Raphson with the displacement limit eps_u."""
    st = shell_step_stats()
    rc = load_library().shell_solve_static(h.ptr, float(eps_f), float(eps_u), int(max_iters), C.byref(st))
    if check:
        _check(rc, "shell_solve_static")
    d = st.as_dict()
    d["rc"] = rc
    return d


def shell_step_noalloc(h: Handle, n_steps: int = 1, check: bool = True) -> dict:
    """shell_step that allocates no device memory (static launch scratch; see include/shell.h)."""
    st = shell_step_stats()
    rc = load_library().shell_step_noalloc(h.ptr, int(n_steps), C.byref(st))
    if check:
        _check(rc, "shell_step_noalloc")
    d = st.as_dict()
    d["rc"] = rc
    return d


def shell_energy(h: Handle) -> np.ndarray:
    out = np.zeros(4, np.float64)
    _check(load_library().shell_energy(h.ptr, out.ctypes.data), "shell_energy")
    return out


def shell_forces(h: Handle) -> np.ndarray:
    out = np.zeros((h.n_verts, 3), np.float64)
    _check(load_library().shell_forces(h.ptr, out.ctypes.data), "shell_forces")
    return out


def shell_apply_matrix(h: Handle, vec) -> np.ndarray:
    """out = A vec with the constant step matrix A = M + dt^2 K (FP64, host buffers)."""
    a = _arr(vec, np.float64, (h.n_verts, 3))
    out = np.zeros((h.n_verts, 3), np.float64)
    _check(load_library().shell_apply_matrix(h.ptr, a.ctypes.data, out.ctypes.data), "shell_apply_matrix")
    return out


def shell_get_state(h: Handle):
    x = np.zeros((h.n_verts, 3), np.float64)
    v = np.zeros((h.n_verts, 3), np.float64)
    _check(load_library().shell_get_state(h.ptr, x.ctypes.data, v.ctypes.data), "shell_get_state")
    return x, v


def shell_set_state(h: Handle, x=None, v=None):
    xa = _arr(x, np.float64, (h.n_verts, 3))
    va = _arr(v, np.float64, (h.n_verts, 3))
    _check(load_library().shell_set_state(h.ptr, _ptr(xa), _ptr(va)), "shell_set_state")


def shell_get_state_device(h: Handle, x_dev=None, v_dev=None):
    """Copy the state into caller-owned device buffers ([V][3] float64 torch tensors), stream ordered."""
    px = None if x_dev is None else x_dev.data_ptr()
    pv = None if v_dev is None else v_dev.data_ptr()
    _check(load_library().shell_get_state_device(h.ptr, px, pv), "shell_get_state_device")


def shell_set_state_device(h: Handle, x_dev=None, v_dev=None):
    px = None if x_dev is None else x_dev.data_ptr()
    pv = None if v_dev is None else v_dev.data_ptr()
    _check(load_library().shell_set_state_device(h.ptr, px, pv), "shell_set_state_device")


def shell_info(h: Handle) -> dict:
    out = np.zeros(9, np.int64)
    _check(load_library().shell_info(h.ptr, out.ctypes.data), "shell_info")
    return {"n_verts": int(out[0]), "n_tris": int(out[1]), "n_stencils": int(out[2]), "device_bytes": int(out[3]),
            "nnz": int(out[4]), "nnz_stored": int(out[5]), "n_slots": int(out[6]), "amg_levels": int(out[7]),
            "vcycle_bytes": int(out[8])}


def shell_destroy(h: Handle):
    if h.ptr:
        _check(load_library().shell_destroy(h.ptr), "shell_destroy")
        h.ptr = None


def shell_topology_summary(tris, n_verts, model, clamped_edges=None) -> dict:
    """Host-only stencil / matrix-structure check (no GPU needed)."""
    tris = _arr(tris, np.int32, (-1, 3))
    ce = _arr(clamped_edges, np.int32, (-1, 2)) if clamped_edges is not None else np.zeros((0, 2), np.int32)
    out = np.zeros(8, np.int64)
    m = MODELS[model] if isinstance(model, str) else int(model)
    _check(load_library().shell_topology_summary(int(n_verts), tris.shape[0], tris.ctypes.data, ce.shape[0],
                                                 ce.ctypes.data if ce.shape[0] else None, m, out.ctypes.data),
           "shell_topology_summary")
    keys = ("edge_stencils", "clamped_edge_stencils", "virtual_tri_stencils", "nnz", "nnz_stored", "n_slots",
            "n_assembled", "bad_indices")
    return {k: int(v) for k, v in zip(keys, out)}


def shell_strerror(code: int) -> str:
    return _strerror(code)


# ------------------------------------------------------------------------------------------ batch API
class Batch:
    def __init__(self, ptr, opts):
        self.ptr = ptr
        self._opts = opts
        self.members = {}
        self._layout = None    # (slots, row offsets) of the packed state layout, until the next admit / retire
        self._slots = None     # resident slots in increasing order and as a set, likewise

    def _changed(self):
        self._layout = None
        self._slots = None

    def resident_slots(self) -> tuple:
        if self._slots is None:
            keys = tuple(sorted(self.members))
            self._slots = (keys, frozenset(keys))
        return self._slots[0]

    def _resident(self):
        self.resident_slots()
        return self._slots

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                load_library().shell_batch_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


class BatchStats(Mapping):
    """Statistics of one batch call: slot -> dict of the shell_step_stats fields, for the resident slots.
    Each slot's dict is built when first read, so a call whose statistics are not read pays nothing for
    them."""
    __slots__ = ("_arr", "_keys", "_set", "_cache")

    def __init__(self, arr, keys, key_set=None):
        self._arr = arr
        self._keys = tuple(keys)
        self._set = frozenset(self._keys) if key_set is None else key_set
        self._cache = {}

    def __getitem__(self, slot):
        d = self._cache.get(slot)
        if d is None:
            if slot not in self._set:
                raise KeyError(slot)
            d = self._cache[slot] = self._arr[slot].as_dict()
        return d

    def __contains__(self, slot):
        return slot in self._set

    def raw(self, slot):
        """The slot's shell_step_stats record itself (fields as attributes), or None if not resident."""
        return self._arr[slot] if slot in self._set else None

    def __iter__(self):
        return iter(self._keys)

    def __len__(self):
        return len(self._keys)


def shell_batch_create(budget_bytes: int, stream=None, use_torch_allocator=True) -> Batch:
    opts = make_options(stream=stream, use_torch_allocator=use_torch_allocator)
    out = C.c_void_p()
    _check(load_library().shell_batch_create(C.byref(opts), int(budget_bytes), C.byref(out)), "shell_batch_create")
    return Batch(out.value, opts)


def shell_batch_admit(b: Batch, h: Handle, check: bool = True) -> int:
    slot = C.c_int32(-1)
    rc = load_library().shell_batch_admit(b.ptr, h.ptr, C.byref(slot))
    if check:
        _check(rc, "shell_batch_admit")
    elif rc != SHELL_OK:
        return rc
    b.members[slot.value] = h
    b._changed()
    return slot.value


def shell_batch_retire(b: Batch, slot: int):
    _check(load_library().shell_batch_retire(b.ptr, int(slot)), "shell_batch_retire")
    b.members.pop(slot, None)
    b._changed()


def shell_batch_step(b: Batch, n_steps: int = 1, check: bool = True):
    """Step every resident instance n_steps times: (rc, BatchStats: slot -> statistics of the call)."""
    lib = load_library()
    cap = lib.shell_batch_capacity(b.ptr)
    stats = (shell_step_stats * max(1, cap))()
    rc = lib.shell_batch_step(b.ptr, int(n_steps), stats)
    if check:
        _check(rc, "shell_batch_step")
    return rc, BatchStats(stats, *b._resident())


def shell_batch_step_times(b: Batch, n: int) -> np.ndarray:
    out = np.zeros(max(1, n), np.float32)
    k = load_library().shell_batch_step_times(b.ptr, out.ctypes.data, int(n))
    return out[:max(0, k)]


def shell_batch_set_profiling(b: Batch, on: bool = True):
    _check(load_library().shell_batch_set_profiling(b.ptr, 1 if on else 0), "shell_batch_set_profiling")


def shell_batch_kernel_times(b: Batch) -> np.ndarray:
    out = np.zeros(2, np.float64)
    _check(load_library().shell_batch_kernel_times(b.ptr, out.ctypes.data), "shell_batch_kernel_times")
    return out


def shell_batch_set_wait_limit(b: Batch, ns: int = 0):
    """Bound of a team-barrier wait of the batch's solve launches in ns (<= 0: the default, 4 s)."""
    _check(load_library().shell_batch_set_wait_limit(b.ptr, int(ns)), "shell_batch_set_wait_limit")


def shell_batch_autotune(b: Batch, steps_per_trial: int = 2) -> dict:
    """Pick the fastest launch shape of the batch's solve kernel on real steps (see include/shell.h)."""
    ms = np.zeros(12, np.float64)
    choice = np.zeros(3, np.int32)
    _check(load_library().shell_batch_autotune(b.ptr, int(steps_per_trial), ms.ctypes.data, choice.ctypes.data),
           "shell_batch_autotune")
    ran = int(np.sum(ms != -1.0))     # -1: skipped; -2: ran, cluster launch refused
    settle = 3                        # calls with the chosen shape after the trials
    return {"trial_ms": ms.tolist(), "ctas_per_sm": int(choice[0]), "share_scale": choice[1] / 100.0,
            "clusters": bool(choice[2]), "steps": (ran + settle) * int(steps_per_trial)}


def shell_batch_set_launch(b: Batch, ctas_per_sm: int, share_scale: float = 1.0, clusters: bool = False):
    """Apply a solve-launch shape without tuning (the fields shell_batch_autotune reports)."""
    _check(load_library().shell_batch_set_launch(b.ptr, int(ctas_per_sm), int(round(share_scale * 100)),
                                                 1 if clusters else 0), "shell_batch_set_launch")


def shell_batch_state_layout(b: Batch):
    """(slots, row_offsets) of the packed state layout: resident slots in increasing order (read once per
    admit / retire; the arrays are read-only)."""
    if b._layout is None:
        lib = load_library()
        n = lib.shell_batch_state_layout(b.ptr, None, None)
        slots = np.zeros(max(1, n), np.int32)
        offs = np.zeros(n + 1, np.int64)
        lib.shell_batch_state_layout(b.ptr, slots.ctypes.data, offs.ctypes.data)
        slots, offs = slots[:n], offs
        slots.flags.writeable = False
        offs.flags.writeable = False
        b._layout = (slots, offs)
    return b._layout


def shell_batch_get_states(b: Batch, x_out=None, v_out=None):
    """Packed [rows][3] FP64 positions and velocities of every resident instance (one copy each way)."""
    _, offs = shell_batch_state_layout(b)
    rows = int(offs[-1])
    x = np.empty((rows, 3), np.float64) if x_out is None else x_out
    v = np.empty((rows, 3), np.float64) if v_out is None else v_out
    assert x.flags.c_contiguous and v.flags.c_contiguous and x.shape == (rows, 3) and v.shape == (rows, 3)
    _check(load_library().shell_batch_get_states(b.ptr, x.ctypes.data, v.ctypes.data), "shell_batch_get_states")
    return x, v


def shell_batch_set_states(b: Batch, x, v):
    _, offs = shell_batch_state_layout(b)
    rows = int(offs[-1])
    xa = _arr(x, np.float64, (rows, 3))
    va = _arr(v, np.float64, (rows, 3))
    _check(load_library().shell_batch_set_states(b.ptr, xa.ctypes.data, va.ctypes.data), "shell_batch_set_states")


def shell_batch_step_states(b: Batch, n_steps: int, x_in=None, v_in=None, x_out=None, v_out=None,
                            check: bool = True):
    """shell_batch_set_states + shell_batch_step + shell_batch_get_states in one call with one wait (packed
    [rows][3] FP64 host buffers; None keeps the device states / copies nothing out)."""
    lib = load_library()
    _, offs = shell_batch_state_layout(b)
    rows = int(offs[-1])
    for a in (x_in, v_in, x_out, v_out):
        assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (rows, 3))
    ptr = lambda a: None if a is None else a.ctypes.data
    cap = lib.shell_batch_capacity(b.ptr)
    stats = (shell_step_stats * max(1, cap))()
    rc = lib.shell_batch_step_states(b.ptr, int(n_steps), ptr(x_in), ptr(v_in), ptr(x_out), ptr(v_out), stats)
    if check:
        _check(rc, "shell_batch_step_states")
    return rc, BatchStats(stats, *b._resident())


def shell_batch_destroy(b: Batch):
    if b.ptr:
        _check(load_library().shell_batch_destroy(b.ptr), "shell_batch_destroy")
        b.ptr = None
        b.members.clear()
        b._changed()
