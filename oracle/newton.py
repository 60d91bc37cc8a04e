"""Newton iterations with the corotated membrane tangent (oracle; test infrastructure only).

Section 5 solves the dynamic step (Eq. 62-63) by minimising the incremental potential with a Newton-type
solver, and the quasi-static benchmarks (Eq. 64) by Newton-Raphson in one load step with a residual-force
tolerance eps_f and an incremental-displacement limit eps_u (a step whose largest nodal displacement exceeds
eps_u is scaled down to it). The models' bending Hessian is constant (Eq. 21, 41, 53); the membrane's is
not. The tangent used here is

    K_T(x) = K_b (x) I_3 + sum_t H_t(x),

K_b the constant bending Hessian and H_t the Hessian of the corotated constant-strain membrane energy of
triangle t (:func:`membrane_hessian_blocks`, exact, with its two rotation terms clamped at zero so that each
block is positive semi-definite). The frozen-rotation part of it (:func:`membrane_tangent_blocks`; the
rotation R = F S^-1 held at its value at x) is, for vertices a, b with hat-function gradients g_a, g_b and
r_a = R g_a,

    H_ab = A t [ mu (g_a . g_b) R R^T + mu r_b r_a^T + lam r_a r_b^T ],

the linear constant-strain stiffness at the rest state, bounded by the constant isotropic block
2 (mu + lam) A t (g_a . g_b) I_3 that the linearised step uses. Alone it lets the Newton iteration of a
bending-dominated plate stall near equilibrium (the full step raises the energy); with the rotation terms it
converges. Readings: the projected exact membrane Hessian (the paper's membrane Hessian is that of its own
membrane model and is not given), and for the shell models the constant bending Hessian (as the paper uses it)
also inside Newton, so their Newton iteration converges to the exact solution at a linear rate.

* :func:`step_newton` -- exact backward Euler: v_0 = 0, v_{k+1} = v_k - J(v_k)^-1 R(v_k),
  J(v) = M + dt^2 K_T(x + dt v), R(v) the backward-Euler residual; stops at ||R(v_k)|| <= rtol ||R(0)||.
* :func:`solve_static` -- Eq. 64: x_{k+1} = x_k + alpha dx, K_T(x_k) dx = f(x_k) + f_ext,
  alpha = min(1, eps_u / |dx|_inf); stops once |f(x_k) + f_ext| < eps_f (2-norm over free degrees of
  freedom). Fixed components (every component of a pinned vertex) stay put.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .energies import lame
from .system import Model, forces, residual_nonlinear, stiffness_matrices


def membrane_rotation(x3, Dm_inv):
    """Polar rotation R = F S^-1 [T,3,2] of the deformation gradient F = [x2-x1, x3-x1] Dm^-1."""
    Ds = np.stack([x3[:, 1] - x3[:, 0], x3[:, 2] - x3[:, 0]], axis=-1)
    F = Ds @ Dm_inv
    w, Q = np.linalg.eigh(np.swapaxes(F, 1, 2) @ F)
    Sinv = Q @ ((1.0 / np.sqrt(w))[:, :, None] * np.swapaxes(Q, 1, 2))
    return F @ Sinv


def hat_gradients(Dm_inv):
    """g_a [T,3,2]: gradients of the three hat functions in the triangle's rest 2D frame."""
    g2, g3 = Dm_inv[:, 0, :], Dm_inv[:, 1, :]
    return np.stack([-g2 - g3, g2, g3], axis=1)


def membrane_tangent_blocks(x3, Dm_inv, area, E, nu, t):
    """Frozen-rotation membrane Hessian blocks H [T,3,3,3,3]: H[t,a,b] is the 3x3 block of vertices a, b."""
    mu, lam = lame(E, nu)
    R = membrane_rotation(x3, Dm_inv)
    g = hat_gradients(Dm_inv)
    r = np.einsum("tij,taj->tai", R, g)                       # r_a = R g_a
    P = R @ np.swapaxes(R, 1, 2)                              # R R^T
    gg = np.einsum("tai,tbi->tab", g, g)
    H = (mu * gg[:, :, :, None, None] * P[:, None, None]
         + mu * np.einsum("tbi,taj->tabij", r, r)
         + lam * np.einsum("tai,tbj->tabij", r, r))
    return (area * t)[:, None, None, None, None] * H


def membrane_hessian_blocks(x3, Dm_inv, area, E, nu, t, project=True):
    """Exact Hessian blocks [T,3,3,3,3] of the corotated membrane energy, optionally with its two rotation
    terms clamped so that each triangle's block is positive semi-definite.

    With F = R S (R 3x2 with orthonormal columns, S the 2x2 stretch, n = r_0 x r_1), a variation dF splits
    into A = R^T dF (2x2) and b = dF^T n (2-vector). The second variation of A t (mu |S - I|^2 +
    lam/2 tr(S - I)^2) is

        A t [ 2 mu |sym A|^2 + lam tr(A)^2 + kappa (A_10 - A_01)^2 + b^T Q b ],
        kappa = mu - c / tr(S),   Q = 2 mu I - c S^-1,   c = 2 mu - lam tr(S - I),

    from dP = 2 mu dF - c dR + lam tr(A) R (P the first Piola stress) and the variation of the polar factor,
    dR = R J (A_10 - A_01) / tr(S) + n b^T S^-1 (J the 2D quarter turn). The first two terms are the
    frozen-rotation tangent; kappa and Q vanish at the rest state. project=True clamps kappa and the
    eigenvalues of Q at zero (they turn negative under compression)."""
    mu, lam = lame(E, nu)
    Ds = np.stack([x3[:, 1] - x3[:, 0], x3[:, 2] - x3[:, 0]], axis=-1)
    F = Ds @ Dm_inv
    w, Vq = np.linalg.eigh(np.swapaxes(F, 1, 2) @ F)
    sv = np.sqrt(w)                                            # singular values = eigenvalues of S
    Sinv = Vq @ ((1.0 / sv)[:, :, None] * np.swapaxes(Vq, 1, 2))
    R = F @ Sinv
    n = np.cross(R[:, :, 0], R[:, :, 1])
    c = 2.0 * mu - lam * (sv.sum(axis=1) - 2.0)
    kappa = mu - c / sv.sum(axis=1)
    qe = 2.0 * mu - c[:, None] / sv                            # eigenvalues of Q (eigenvectors Vq)
    if project:
        kappa = np.maximum(kappa, 0.0)
        qe = np.maximum(qe, 0.0)
    Q = Vq @ (qe[:, :, None] * np.swapaxes(Vq, 1, 2))
    T = F.shape[0]
    z = np.zeros((T, 3))
    r0, r1 = R[:, :, 0], R[:, :, 1]
    # each term as a row vector on vec(dF) = (dF[:, 0], dF[:, 1])
    s00 = np.concatenate([r0, z], 1)
    s11 = np.concatenate([z, r1], 1)
    s01 = 0.5 * np.concatenate([r1, r0], 1)
    tr = np.concatenate([r0, r1], 1)
    rot = np.concatenate([r1, -r0], 1)
    b0 = np.concatenate([n, z], 1)
    b1 = np.concatenate([z, n], 1)
    outer = lambda a, b: np.einsum("ti,tj->tij", a, b)
    C = (2.0 * mu * (outer(s00, s00) + outer(s11, s11) + 2.0 * outer(s01, s01)) + lam * outer(tr, tr)
         + kappa[:, None, None] * outer(rot, rot)
         + Q[:, 0, 0, None, None] * outer(b0, b0) + Q[:, 1, 1, None, None] * outer(b1, b1)
         + Q[:, 0, 1, None, None] * (outer(b0, b1) + outer(b1, b0)))
    C = (area * t)[:, None, None] * C
    g = hat_gradients(Dm_inv)
    G = np.zeros((T, 3, 6, 3))                                  # vec(dF) = sum_a G_a u_a
    for a in range(3):
        for k in range(2):
            G[:, a, 3 * k:3 * k + 3, :] = g[:, a, k, None, None] * np.eye(3)
    return np.einsum("taki,tkl,tblj->tabij", G, C, G)


def _scatter_blocks(H, tris, V):
    """Sparse 3V x 3V matrix from per-triangle vertex-pair blocks H [T,3,3,3,3]."""
    T = tris.shape[0]
    a_idx = np.repeat(np.arange(3), 3)
    b_idx = np.tile(np.arange(3), 3)
    rows, cols, vals = [], [], []
    for a, b in zip(a_idx, b_idx):
        for i in range(3):
            for j in range(3):
                rows.append(3 * tris[:, a] + i)
                cols.append(3 * tris[:, b] + j)
                vals.append(H[:, a, b, i, j])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * V, 3 * V)).tocsr()


def tangent_matrix(m: Model, x, frozen=False) -> sp.csr_matrix:
    """K_T(x) = K_b (x) I_3 + sum_t H_t(x) as a 3V x 3V matrix (unknowns ordered vertex-major, x y z); H_t the
    projected exact membrane Hessian, or (frozen=True) the frozen-rotation one."""
    V = m.n_verts
    Kb, _ = stiffness_matrices(m)
    K = sp.kron(Kb, sp.identity(3), format="csr")
    if m.membrane:
        fn = membrane_tangent_blocks if frozen else membrane_hessian_blocks
        H = fn(x[m.tris], m.Dm_inv, m.tri_area, m.E, m.nu, m.thickness)
        K = K + _scatter_blocks(H, m.tris, V)
    return K


def _pin_rows(m: Model, K):
    """Identity rows and columns at the fixed components (every component of a pinned vertex)."""
    free = (~m.fixed).ravel().astype(np.float64)
    D = sp.diags(free)
    return (D @ K @ D + sp.diags(1.0 - free)).tocsc()


def step_newton(m: Model, x, v, n_steps=1, max_iters=30, rtol=1e-10):
    """n_steps exact backward-Euler steps by Newton on the incremental potential (see module docstring).
    Returns (x, v, iterations of each step)."""
    x = np.array(x, np.float64, copy=True)
    v = np.array(v, np.float64, copy=True)
    Mv = np.repeat(m.mass, 3)
    iters = []
    for _ in range(n_steps):
        vk = np.zeros_like(v)
        R = residual_nonlinear(m, x, v, vk)
        n0 = np.linalg.norm(R)
        k = 0
        while k < max_iters and np.linalg.norm(R) > rtol * n0:
            J = sp.diags(Mv) + m.dt ** 2 * tangent_matrix(m, x + m.dt * vk)
            dv = spla.spsolve(_pin_rows(m, J), R.ravel()).reshape(-1, 3)
            vk = vk - dv
            k += 1
            R = residual_nonlinear(m, x, v, vk)
        iters.append(k)
        x = x + m.dt * vk
        v = vk
    return x, v, iters


def static_residual(m: Model, x):
    """f(x) + f_ext at free components (zero at fixed ones): the residual of Eq. 64."""
    r = forces(m, x) + m.f_ext
    r[m.fixed] = 0.0
    return r


def solve_static(m: Model, x0, eps_f=1e-3, eps_u=0.1, max_iters=1000, shift=False):
    """Eq. 64 by Newton-Raphson in one load step with the displacement limit eps_u (module docstring).
    shift=True adds M / dt^2 to the tangent (a damped Newton step with the same fixed point; the GPU's linear
    systems carry this shift). Returns (x, iterations, final residual norm)."""
    x = np.array(x0, np.float64, copy=True)
    Ms = sp.diags(np.repeat(m.mass, 3) / m.dt ** 2) if shift else None
    for k in range(max_iters + 1):
        r = static_residual(m, x)
        nr = np.linalg.norm(r)
        if nr < eps_f or k == max_iters:
            return x, k, nr
        K = tangent_matrix(m, x)
        if shift:
            K = K + Ms
        dx = spla.spsolve(_pin_rows(m, K), r.ravel()).reshape(-1, 3)
        dx[m.fixed] = 0.0
        big = np.abs(dx).max()
        alpha = min(1.0, eps_u / big) if big > 0 else 1.0
        x = x + alpha * dx
    return x, max_iters, nr
