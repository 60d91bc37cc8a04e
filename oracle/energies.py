"""Per-stencil bending energies and exact gradients, and the corotated membrane (oracle; test only).

A stencil set holds, per stencil s: vertex indices idx [S,k], folded operator L [S,r,k] (r = 1 for the
edge hinge, 3 for triangle stencils), weighted material matrix W [S,r,r] (k_b A_E for the edge hinge,
A D_b or A R^T D_b R for triangle stencils), rest curvature kappa0 [S,r] and a mode:

* PLATE (EP, FP, SP; Eq. 20, Eq. 41, Eq. 53): the energy is the full ``(x) I_3`` quadratic form
  Psi = 1/2 sum_c (L x_c)^T W (L x_c), summed over the three world coordinates c, so the gradient is
  exactly the constant Hessian times x (Eq. 21-22).
* SHELL (ES, FS, SS; Eq. 23-26, Eq. 42-45, Eq. 54-57): eps = L N^T x - kappa0 with N = I (x) n, n the
  unit normal of the current corotational frame; Psi = 1/2 eps^T W eps and the gradient carries the
  derivative of n (App. B).
* FIXED: stencils that touch a clamped edge measure the transverse displacement from rest along the
  fixed rest normal n_cl: eps = L (n_cl . (x_j - X_j))_j (reading of Eq. 30-31 and Eq. 59: in the
  current frame of a boundary stencil the one real triangle's own plane gives w = 0 at all its nodes,
  so the clamp would measure nothing; the fixed normal keeps the zero-slope condition).

Every stencil subtracts its frame origin before applying L (x_2 for edge stencils, x_1 for triangle
stencils, App. A); this changes nothing because every folded row of L sums to zero.

Reading (edge-hinge normal, Eq. 8): we use n = (n_123 + n_432)/|n_123 + n_432|, the normalised sum of
the two triangles' unit normals. It is parallel to p/|p| + q/|q| of Eq. 8 (both lie in the plane normal
to the hinge and bisect the two faces) but keeps a sign, so curvature is signed, and stays well
conditioned when the two triangles are coplanar (then |p/|p| + q/|q|| -> 0). If |n_123 + n_432| < 1e-8
(folded past 180 degrees, the failure mode noted in Section 7) n_123 is used.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .operators import dot, norm

PLATE, SHELL, FIXED = 0, 1, 2


@dataclasses.dataclass
class StencilSet:
    kind: str            # 'edge' or 'tri'
    idx: np.ndarray      # [S,k] int64, -1 = virtual (its column of L is zero)
    L: np.ndarray        # [S,r,k]
    W: np.ndarray        # [S,r,r]
    kappa0: np.ndarray   # [S,r]
    mode: np.ndarray     # [S] PLATE / SHELL / FIXED
    nfix: np.ndarray     # [S,3] fixed normal (FIXED mode), else 0
    rest: np.ndarray     # [S,k,3] rest positions (virtual nodes included)

    @property
    def origin(self):
        return 1 if self.kind == "edge" else 0

    def __len__(self):
        return self.idx.shape[0]


def gather(x, idx):
    """Stencil positions [S,k,3]; virtual slots read vertex 0 (their operator column is zero)."""
    return x[np.where(idx < 0, 0, idx)]


def skew(v):
    """Cross-product matrix v^x of Eq. 74, batched: [...,3] -> [...,3,3]."""
    z = np.zeros(v.shape[:-1])
    x, y, w = v[..., 0], v[..., 1], v[..., 2]
    return np.stack([np.stack([z, -w, y], -1), np.stack([w, z, -x], -1), np.stack([-y, x, z], -1)], -2)


def unit_and_jacobian(c):
    """n = c/|c| and dn/dc = (I - n n^T)/|c| (App. B Eq. 67)."""
    l = norm(c)
    n = c / l[..., None]
    P = np.eye(3) - n[..., :, None] * n[..., None, :]
    return n, P / l[..., None, None]


def triangle_normal_jacobian(x1, x2, x3):
    """Unit normal of triangle (x1,x2,x3) and its Jacobians d n / d x_j (App. B Eq. 72-73)."""
    c = np.cross(x2 - x1, x3 - x1)
    n, dn_dc = unit_and_jacobian(c)
    dc = [skew(x3 - x2), skew(x1 - x3), skew(x2 - x1)]   # d c / d x1, d x2, d x3 (Eq. 73)
    return n, [dn_dc @ d for d in dc]


def frame_normal(xs, kind):
    """Current corotational frame normal n [S,3] and Jacobians J [S,k,3,3] (J[:,j] = dn/dx_j)."""
    S, k = xs.shape[:2]
    J = np.zeros((S, k, 3, 3))
    if kind == "tri":
        n, Jt = triangle_normal_jacobian(xs[:, 0], xs[:, 1], xs[:, 2])
        for j in range(3):
            J[:, j] = Jt[j]
        return n, J
    # edge hinge: oriented mean normal of T123 and T432 (reading of Eq. 8, see module docstring)
    n1, J1 = triangle_normal_jacobian(xs[:, 0], xs[:, 1], xs[:, 2])
    n2, J2 = triangle_normal_jacobian(xs[:, 3], xs[:, 2], xs[:, 1])
    m = n1 + n2
    n, dn_dm = unit_and_jacobian(m)
    Jm = np.zeros((S, k, 3, 3))
    for j, Jj in zip((0, 1, 2), J1):
        Jm[:, j] += Jj
    for j, Jj in zip((3, 2, 1), J2):
        Jm[:, j] += Jj
    J = np.einsum("sab,skbc->skac", dn_dm, Jm)
    folded = norm(m) < 1e-8
    if np.any(folded):
        n[folded] = n1[folded]
        J[folded] = 0.0
        for j in range(3):
            J[folded, j] = J1[j][folded]
    return n, J


def curvature_vectors(x, st):
    """G_i = sum_j L_ij (x_j - x_origin): [S,r,3], plus stencil positions [S,k,3]."""
    xs = gather(x, st.idx)
    d = xs - xs[:, st.origin][:, None, :]
    return np.einsum("srk,skc->src", st.L, d), xs


def stencil_energy(x, st):
    """Bending energy per stencil [S] (Eq. 16, 23, 39, 42, 52, 54 with the readings above)."""
    G, xs = curvature_vectors(x, st)
    E = np.zeros(len(st))
    p = st.mode == PLATE
    if np.any(p):
        E[p] = 0.5 * np.einsum("sic,sil,slc->s", G[p], st.W[p], G[p])
    s = st.mode == SHELL
    if np.any(s):
        n, _ = frame_normal(xs[s], st.kind)
        eps = np.einsum("sic,sc->si", G[s], n) - st.kappa0[s]
        E[s] = 0.5 * np.einsum("si,sil,sl->s", eps, st.W[s], eps)
    f = st.mode == FIXED
    if np.any(f):
        eps = np.einsum("sic,sc->si", G[f], st.nfix[f]) - st.kappa0[f]
        E[f] = 0.5 * np.einsum("si,sil,sl->s", eps, st.W[f], eps)
    return E


def stencil_forces(x, st):
    """Per-stencil nodal forces -dPsi/dx_j: [S,k,3] (Eq. 22, 25-26, 44-45, 56-57, App. B)."""
    G, xs = curvature_vectors(x, st)
    F = np.zeros(xs.shape)
    p = st.mode == PLATE
    if np.any(p):
        sig = np.einsum("sil,slc->sic", st.W[p], G[p])          # W L x_c per coordinate
        F[p] = -np.einsum("sij,sic->sjc", st.L[p], sig)
    s = st.mode == SHELL
    if np.any(s):
        n, J = frame_normal(xs[s], st.kind)
        eps = np.einsum("sic,sc->si", G[s], n) - st.kappa0[s]
        sig = np.einsum("sil,sl->si", st.W[s], eps)
        g = np.einsum("si,sic->sc", sig, G[s])                    # sum_i sigma_i G_i
        term1 = np.einsum("si,sij,sc->sjc", sig, st.L[s], n)     # N L^T sigma
        term2 = np.einsum("sjab,sa->sjb", J, g)                   # (dn/dx_j)^T g
        F[s] = -(term1 + term2)
    f = st.mode == FIXED
    if np.any(f):
        eps = np.einsum("sic,sc->si", G[f], st.nfix[f]) - st.kappa0[f]
        sig = np.einsum("sil,sl->si", st.W[f], eps)
        F[f] = -np.einsum("si,sij,sc->sjc", sig, st.L[f], st.nfix[f])
    return F


def stencil_hessian_blocks(st):
    """Constant scalar Hessian blocks L^T W L [S,k,k]; the matrix is this (x) I_3 (Eq. 21, 41, 53)."""
    return np.einsum("sik,sil,slm->skm", st.L, st.W, st.L)


# ------------------------------------------------------------------ membrane
def membrane_rest(X):
    """Rest data of the constant-strain triangles. X [T,3,3] -> (Dm^-1 [T,2,2], area [T]).

    Dm holds the rest edge vectors X_12, X_13 in the triangle's own 2D frame (x along X_12)."""
    e12 = X[:, 1] - X[:, 0]
    e13 = X[:, 2] - X[:, 0]
    ex = e12 / norm(e12)[:, None]
    nz = np.cross(e12, e13)
    area = 0.5 * norm(nz)
    nz = nz / norm(nz)[:, None]
    ey = np.cross(nz, ex)
    Dm = np.stack([np.stack([dot(ex, e12), dot(ex, e13)], -1), np.stack([dot(ey, e12), dot(ey, e13)], -1)], -2)
    return np.linalg.inv(Dm), area


def lame(E, nu):
    """mu and the plane-stress lambda: mu = E/(2(1+nu)), lam = E nu/(1 - nu^2)."""
    return E / (2.0 * (1.0 + nu)), E * nu / (1.0 - nu * nu)


def membrane_energy_force(x3, Dm_inv, area, E, nu, t):
    """Corotated linear constant-strain membrane (the paper adopts the constant strain triangle for the
    membrane, Section 3; reading: the corotated small-strain form, so the energy is rotation invariant).

    F = [x2-x1, x3-x1] Dm^-1 (3x2), S = sqrt(F^T F) (by eigen-decomposition), e = S - I,
    Psi = A t (mu |e|^2 + lam/2 tr(e)^2), dPsi/dF = A t R (2 mu e + lam tr(e) I) with R = F S^-1.
    Returns (energy [T], forces [T,3,3]).
    """
    mu, lam = lame(E, nu)
    Ds = np.stack([x3[:, 1] - x3[:, 0], x3[:, 2] - x3[:, 0]], axis=-1)      # [T,3,2]
    F = Ds @ Dm_inv
    C = np.swapaxes(F, 1, 2) @ F
    w, Q = np.linalg.eigh(C)
    sq = np.sqrt(w)
    S = Q @ (sq[:, :, None] * np.swapaxes(Q, 1, 2))
    Sinv = Q @ ((1.0 / sq)[:, :, None] * np.swapaxes(Q, 1, 2))
    e = S - np.eye(2)
    tr = e[:, 0, 0] + e[:, 1, 1]
    energy = area * t * (mu * np.sum(e * e, axis=(1, 2)) + 0.5 * lam * tr * tr)
    P = (F @ Sinv) @ (2.0 * mu * e + lam * tr[:, None, None] * np.eye(2))
    H = (area * t)[:, None, None] * (P @ np.swapaxes(Dm_inv, 1, 2))          # dPsi/dDs [T,3,2]
    forces = np.stack([H[:, :, 0] + H[:, :, 1], -H[:, :, 0], -H[:, :, 1]], axis=1)
    return energy, forces


def membrane_stiffness_blocks(Dm_inv, area, E, nu, t):
    """Constant isotropic membrane blocks k_ab = 2 (mu + lam) A t grad(phi_a).grad(phi_b) [T,3,3]; the
    matrix is this (x) I_3 (reading: the smallest isotropic weight that bounds the frozen-rotation
    membrane Hessian, because (tr e)^2 <= 2 |e|^2 in 2D)."""
    mu, lam = lame(E, nu)
    g2 = Dm_inv[:, 0, :]          # grad phi_2 = first row of Dm^-1
    g3 = Dm_inv[:, 1, :]
    g1 = -g2 - g3
    G = np.stack([g1, g2, g3], axis=1)   # [T,3,2]
    return (2.0 * (mu + lam) * area * t)[:, None, None] * (G @ np.swapaxes(G, 1, 2))
