"""Global system of the oracle: stencil sets, lumped mass, constant matrix, linearised backward Euler.

Reading of the time step (Section 5, Eq. 62-63). The paper minimises the incremental potential
E(x) = 1/2 |x - x_hat|_M^2 + dt^2 Psi(x) with a Newton-type solver. The step computed here is one
linearised backward-Euler solve with the constant matrix:

    (M + dt^2 K) v' = M v + dt (f(x) + f_ext),    x' = x + dt v',

where f = -grad(Psi_m + Psi_b) is the exact gradient, K = K_b + K_m is constant (the bending Hessian
of Eq. 21 / 41 / 53 assembled once from the rest state, plus the isotropic membrane block of
:func:`oracle.energies.membrane_stiffness_blocks`), and M is the lumped mass m_i = sum over incident
triangles of density * thickness * area / 3 (the paper does not give M). For plates without membrane
this is exactly backward Euler, since the plate force is linear. Pinned vertices get an identity row
and column and a zero right-hand side, so their velocity is zero.

Per-component constraints (the symmetry conditions of Section 6.1's hemisphere: one or two displacement
components of a vertex fixed, the others free) do not fit the scalar matrix: with them the step is solved on
the 3V unknowns (vertex-major x, y, z), the matrix A (x) I_3 keeping the rows and columns of the free
components and getting identity rows and columns, with zero right-hand sides, at the fixed ones.

The linear system is solved directly (scipy SuperLU factorisation, computed once), so the oracle gives
the exact solution of each step's system up to rounding.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as op
from .energies import (FIXED, PLATE, SHELL, StencilSet, frame_normal, membrane_energy_force, membrane_rest,
                       membrane_stiffness_blocks, stencil_energy, stencil_forces, stencil_hessian_blocks)
from .topology import CLAMPED, build_stencils, stencil_positions

MODELS = ("EP", "ES", "FP", "FS", "SP", "SS")


@dataclasses.dataclass
class Model:
    model: str
    tris: np.ndarray
    rest: np.ndarray
    E: float
    nu: float
    thickness: float
    density: float
    dt: float
    pinned: np.ndarray          # [V] bool
    f_ext: np.ndarray           # [V,3]
    mass: np.ndarray            # [V]
    stencils: List[StencilSet]
    Dm_inv: np.ndarray          # [T,2,2]
    tri_area: np.ndarray        # [T]
    membrane: bool
    fixed: Optional[np.ndarray] = None    # [V,3] bool: fixed components (all three at pinned vertices)
    A: Optional[sp.csc_matrix] = None
    _lu: object = None
    _lu3: object = None

    @property
    def partial(self) -> bool:
        """True when some vertex has fixed and free components (the step needs the 3V matrix)."""
        return bool(np.any(self.fixed.any(axis=1) & ~self.fixed.all(axis=1)))

    @property
    def n_verts(self):
        return self.rest.shape[0]


def _edge_stencils(rest, topo, model, kb):
    sets = []
    e = topo["edge"]
    if len(e):
        X = rest[e]
        L, area = op.edge_operator(X)
        L = L[:, None, :]
        W = (kb * area)[:, None, None]
        if model == "ES":
            n0, _ = frame_normal(X, "edge")
            d = X - X[:, 1:2]
            kappa0 = np.einsum("srk,skc,sc->sr", L, d, n0)
            mode = np.full(len(e), SHELL)
        else:
            kappa0 = np.zeros((len(e), 1))
            mode = np.full(len(e), PLATE)
        sets.append(StencilSet("edge", e.copy(), L, W, kappa0, mode, np.zeros((len(e), 3)), X))
    c = topo["edge_clamped"]
    if len(c):
        X3 = rest[c]
        L, area = op.edge_clamped_operator(X3)
        L = L[:, None, :]
        W = (kb * area)[:, None, None]
        X4 = np.concatenate([X3, (X3[:, 1] + X3[:, 2] - X3[:, 0])[:, None]], axis=1)
        nfix = np.cross(X3[:, 1] - X3[:, 0], X3[:, 2] - X3[:, 0])
        nfix /= op.norm(nfix)[:, None]
        kappa0 = np.einsum("srk,skc,sc->sr", L, X4 - X4[:, 1:2], nfix)
        idx = np.concatenate([c, -np.ones((len(c), 1), np.int64)], axis=1)
        sets.append(StencilSet("edge", idx, L, W, kappa0, np.full(len(c), FIXED), nfix, X4))
    return sets


def _triangle_stencils(rest, topo, model, D_b):
    t = topo["tri"]
    bc = topo["tri_bc"]
    X = stencil_positions(rest, t, bc)
    L, Dmat, area = op.triangle_stencil_operators(X, bc, model[0], D_b)
    W = area[:, None, None] * Dmat
    n0 = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    n0 /= op.norm(n0)[:, None]
    d = X - X[:, :1]
    clamped = np.any(bc == CLAMPED, axis=1)
    mode = np.full(len(t), SHELL if model[1] == "S" else PLATE)
    mode[clamped] = FIXED
    kappa0 = np.einsum("srk,skc,sc->sr", L, d, n0)
    kappa0[mode == PLATE] = 0.0
    nfix = np.where(clamped[:, None], n0, 0.0)
    return [StencilSet("tri", t.copy(), L, W, kappa0, mode, nfix, X)]


def build_model(tris, rest, model, E, nu, thickness, density, dt, pinned=None, clamped_edges=(),
                gravity=(0.0, 0.0, 0.0), load_vtx=(), load_f=(), membrane=True, factor=True,
                fixed_dofs=None) -> Model:
    """Rest-state precompute and constant matrix for one mesh (the 'create' step). ``fixed_dofs``: per-vertex
    bit mask of fixed components (bit 0 x, bit 1 y, bit 2 z) or None; all three bits pin the vertex."""
    if model not in MODELS:
        raise ValueError(model)
    tris = np.asarray(tris, np.int64)
    rest = np.asarray(rest, np.float64)
    V = rest.shape[0]
    topo = build_stencils(tris, V, clamped_edges)
    D_b = op.bending_D(E, nu, thickness)
    kb = op.bending_rigidity(E, nu, thickness)
    if model[0] == "E":
        sets = _edge_stencils(rest, topo, model, kb)
    else:
        sets = _triangle_stencils(rest, topo, model, D_b)
    Dm_inv, area = membrane_rest(rest[tris])
    mass = np.zeros(V)
    np.add.at(mass, tris.ravel(), np.repeat(density * thickness * area / 3.0, 3))
    pin = np.zeros(V, bool) if pinned is None else np.asarray(pinned).astype(bool)
    if len(np.asarray(clamped_edges).ravel()):
        pin[np.asarray(clamped_edges).ravel()] = True
    fixed = np.repeat(pin[:, None], 3, axis=1)
    if fixed_dofs is not None:
        bits = np.asarray(fixed_dofs).astype(np.int64)
        fixed |= ((bits[:, None] >> np.arange(3)[None, :]) & 1).astype(bool)
        pin |= fixed.all(axis=1)
    f_ext = mass[:, None] * np.asarray(gravity, np.float64)[None, :]
    lv = np.asarray(load_vtx, np.int64).ravel()
    if len(lv):
        np.add.at(f_ext, lv, np.asarray(load_f, np.float64).reshape(-1, 3))
    m = Model(model, tris, rest, E, nu, thickness, density, dt, pin, f_ext, mass, sets, Dm_inv, area, membrane,
              fixed)
    if factor:
        m.A = system_matrix(m)
        if m.partial:
            m._lu3 = spla.splu(system_matrix3(m))
        else:
            m._lu = spla.splu(m.A)
    return m


def from_scenario(sc, membrane=True, factor=True) -> Model:
    """Build the oracle model of a :class:`shellgen.Scenario`."""
    return build_model(sc.tris, sc.rest, sc.model, sc.E, sc.nu, sc.thickness, sc.density, sc.dt, sc.pinned,
                       sc.clamped_edges, sc.gravity, sc.load_vtx, sc.load_f, membrane=membrane, factor=factor,
                       fixed_dofs=getattr(sc, "fixed_dofs", None))


# ------------------------------------------------------------------ matrices
def _scatter(blocks, idx, V):
    S, k = idx.shape
    rows = np.repeat(idx, k, axis=1).ravel()
    cols = np.tile(idx, (1, k)).ravel()
    vals = blocks.reshape(S, k * k).ravel()
    keep = (rows >= 0) & (cols >= 0)
    return sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(V, V)).tocsr()


def stiffness_matrices(m: Model):
    """Scalar (per vertex pair) constant bending and membrane stiffness K_b, K_m; the 3V x 3V matrices are
    these (x) I_3."""
    V = m.n_verts
    Kb = sp.csr_matrix((V, V))
    for st in m.stencils:
        Kb = Kb + _scatter(stencil_hessian_blocks(st), st.idx, V)
    if m.membrane:
        Km = _scatter(membrane_stiffness_blocks(m.Dm_inv, m.tri_area, m.E, m.nu, m.thickness), m.tris, V)
    else:
        Km = sp.csr_matrix((V, V))
    return Kb, Km


def system_matrix(m: Model) -> sp.csc_matrix:
    """A = M + dt^2 (K_b + K_m) with identity rows/columns at pinned vertices (scalar, V x V)."""
    Kb, Km = stiffness_matrices(m)
    A = sp.diags(m.mass) + (m.dt ** 2) * (Kb + Km)
    keep = sp.diags((~m.pinned).astype(np.float64))
    A = keep @ A @ keep + sp.diags(m.pinned.astype(np.float64))
    return A.tocsc()


def system_matrix3(m: Model) -> sp.csc_matrix:
    """The step matrix on the 3V unknowns (vertex-major x, y, z): (M + dt^2 (K_b + K_m)) (x) I_3 with identity
    rows and columns at every fixed component."""
    Kb, Km = stiffness_matrices(m)
    A3 = sp.kron(sp.diags(m.mass) + (m.dt ** 2) * (Kb + Km), sp.identity(3), format="csr")
    free = (~m.fixed).ravel().astype(np.float64)
    return (sp.diags(free) @ A3 @ sp.diags(free) + sp.diags(1.0 - free)).tocsc()


def solve_step_matrix(m: Model, b):
    """A^-1 b for b [V,3] (direct SuperLU solve, factorised once): the scalar matrix on the three components
    alike, or the 3V matrix when some vertex has fixed and free components."""
    if m.partial:
        if m._lu3 is None:
            m._lu3 = spla.splu(system_matrix3(m))
        return m._lu3.solve(np.ascontiguousarray(b).ravel()).reshape(-1, 3)
    if m._lu is None:
        m.A = system_matrix(m)
        m._lu = spla.splu(m.A)
    return m._lu.solve(b)


# ------------------------------------------------------------------ forces / energy / step
def forces(m: Model, x):
    """f = -grad(Psi_m + Psi_b) at positions x [V,3] (exact gradient, not the constant Hessian)."""
    V = m.n_verts
    f = np.zeros((V, 3))
    for st in m.stencils:
        F = stencil_forces(x, st)
        real = st.idx >= 0
        np.add.at(f, st.idx[real], F[real])
    if m.membrane:
        _, Fm = membrane_energy_force(x[m.tris], m.Dm_inv, m.tri_area, m.E, m.nu, m.thickness)
        np.add.at(f, m.tris.ravel(), Fm.reshape(-1, 3))
    return f


def bending_energy(m: Model, x):
    return float(sum(np.sum(stencil_energy(x, st)) for st in m.stencils))


def membrane_energy(m: Model, x):
    if not m.membrane:
        return 0.0
    e, _ = membrane_energy_force(x[m.tris], m.Dm_inv, m.tri_area, m.E, m.nu, m.thickness)
    return float(np.sum(e))


def energy(m: Model, x, v):
    """(membrane, bending, kinetic, external potential) with the external potential -sum f_ext.(x - X)."""
    kin = 0.5 * float(np.sum(m.mass[:, None] * v * v))
    ext = -float(np.sum(m.f_ext * (x - m.rest)))
    return membrane_energy(m, x), bending_energy(m, x), kin, ext


def rhs(m: Model, x, v):
    """b = M v + dt (f(x) + f_ext), zero at fixed components."""
    b = m.mass[:, None] * v + m.dt * (forces(m, x) + m.f_ext)
    b[m.fixed] = 0.0
    return b


def step(m: Model, x, v, n_steps=1):
    """n_steps linearised backward-Euler steps; returns (x, v)."""
    x = np.array(x, np.float64, copy=True)
    v = np.array(v, np.float64, copy=True)
    for _ in range(n_steps):
        v = solve_step_matrix(m, rhs(m, x, v))
        x = x + m.dt * v
    return x, v


# ------------------------------------------------------------------ exact backward Euler (chord iteration)
def residual_nonlinear(m: Model, x, v, vn):
    """Backward-Euler residual of a candidate new velocity vn (Section 5, Eq. 62-63 without the
    linearisation): R = M (vn - v) - dt (f(x + dt vn) + f_ext) at free components, R = vn at fixed ones.
    R = 0 is the stationarity condition of the incremental potential in the velocity unknown."""
    R = m.mass[:, None] * (vn - v) - m.dt * (forces(m, x + m.dt * vn) + m.f_ext)
    R[m.fixed] = vn[m.fixed]
    return R


def step_nonlinear(m: Model, x, v, n_steps=1, max_iters=50, rtol=1e-8):
    """n_steps backward-Euler steps solved to the nonlinear residual: chord iteration with the constant
    matrix A = M + dt^2 K, v_0 = 0, v_{k+1} = v_k - A^-1 R(v_k), stopping at the first iterate with
    ||R(v_k)|| <= rtol ||R(0)|| (or after max_iters solves). The first iterate is the linearised step.
    Returns (x, v, iterations of each step)."""
    x = np.array(x, np.float64, copy=True)
    v = np.array(v, np.float64, copy=True)
    iters = []
    for _ in range(n_steps):
        vk = np.zeros_like(v)
        R = residual_nonlinear(m, x, v, vk)
        n0 = np.linalg.norm(R)
        k = 0
        while k < max_iters:
            vk = vk - solve_step_matrix(m, R)
            k += 1
            R = residual_nonlinear(m, x, v, vk)
            if np.linalg.norm(R) <= rtol * n0:
                break
        iters.append(k)
        x = x + m.dt * vk
        v = vk
    return x, v, iters


def incremental_potential(m: Model, x, v, vn):
    """Incremental potential of the step in the velocity unknown (fixed components of it are zero):
    E(vn) = 1/2 (vn - v)^T M (vn - v) + Psi(x + dt vn) - f_ext . (x + dt vn); its gradient in vn is
    M (vn - v) - dt (f(x + dt vn) + f_ext) = R(vn) at free components, so backward Euler is its minimiser."""
    d = vn - v
    xn = x + m.dt * vn
    return (0.5 * float(np.sum(m.mass[:, None] * d * d)) + membrane_energy(m, xn) + bending_energy(m, xn)
            - float(np.sum(m.f_ext * xn)))
