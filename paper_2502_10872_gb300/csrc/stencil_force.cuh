// stencil_force.cuh -- per-stencil elastic forces (and energies) of one triangle or edge stencil, shared by
// the standalone force kernel (kernels_force.cu) and the force phase of the persistent step kernel
// (kernels_solve.cu).
//
// One thread per stencil. Each stencil fits its current corotational frame, applies its curvature
// operator and writes its nodal forces to its own contribution slots; the right-hand side (and
// shell_forces) later sums each vertex's slots in a fixed order, so results are deterministic.
//
//   plate  (EP, FP, SP; Eq. 20-22, 41, 53): f_j = -sum_i L_ij (W G)_i with G_i = sum_j L_ij (x_j - x_o)
//   shell  (ES, FS, SS; Eq. 25-26, 44-45, 56-57): eps = n.G - kappa0, sigma = W eps,
//          f_j = -(sum_i sigma_i L_ij) n - (dn/dx_j)^T sum_i sigma_i G_i   (App. B)
//   fixed  (stencils on clamped edges): as the shell with n the fixed rest normal and no dn/dx term.
// The frame normal of a triangle stencil is the central triangle's unit normal (Eq. 15); the edge hinge
// uses the normalised sum of its two faces' unit normals (parallel to the bisector of Eq. 8, signed and
// well conditioned when the faces are coplanar). Origins: x_1 for triangle stencils, x_2 for edge
// stencils (App. A); every row of L sums to zero, so subtracting the origin changes nothing.
//
// Membrane (every triangle, fused into the triangle pass): corotated linear constant-strain triangle,
// Psi = A t (mu |S - I|^2 + lam/2 tr(S - I)^2), S = sqrt(F^T F), force from P = R (2 mu e + lam tr e I),
// R = F S^-1. The Green strain F^T F - I is formed from FP64 differences of edge Gram matrices and S - I
// from a cancellation-free closed form of the 2x2 square root, so the FP32 path keeps the strain's
// relative accuracy.
//
// Position differences x_j - x_o are always formed in FP64 and then rounded to the kernel precision.
#pragma once
#include <cmath>

#include "internal.h"

namespace shl {
namespace {

template <typename R>
struct v3 {
  R x, y, z;
};
template <typename R>
__device__ inline v3<R> operator+(v3<R> a, v3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename R>
__device__ inline v3<R> operator-(v3<R> a, v3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename R>
__device__ inline v3<R> operator*(R s, v3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename R>
__device__ inline R dot(v3<R> a, v3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R>
__device__ inline v3<R> cross(v3<R> a, v3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ inline v3<R> zero3() { return {R(0), R(0), R(0)}; }
template <typename R>
__device__ inline R rsqrt_(R a);
template <>
__device__ inline float rsqrt_<float>(float a) { return 1.0f / sqrtf(a); }
template <>
__device__ inline double rsqrt_<double>(double a) { return 1.0 / sqrt(a); }

// precision-specific views of the stencil data
template <typename R>
struct Data;
// X: the positions the forces are evaluated at (x, or the chord iterate xk)
template <>
struct Data<double> {
  const double *tL, *tW, *tk0, *tn, *mD, *mAt, *eL, *ew, *ek0, *en;
  const double *X;
  __device__ Data(const Inst &I, const double *pos)
      : tL(I.t_L64), tW(I.t_W64), tk0(I.t_k064), tn(I.t_n64), mD(I.m_D64), mAt(I.m_At64), eL(I.e_L64),
        ew(I.e_w64), ek0(I.e_k064), en(I.e_n64), X(pos) {}
};
template <>
struct Data<float> {
  const float *tL, *tW, *tk0, *tn, *mD, *mAt, *eL, *ew, *ek0, *en;
  const double *X;
  __device__ Data(const Inst &I, const double *pos)
      : tL(I.t_L32), tW(I.t_W32), tk0(I.t_k032), tn(I.t_n32), mD(I.m_D32), mAt(I.m_At32), eL(I.e_L32),
        ew(I.e_w32), ek0(I.e_k032), en(I.e_n32), X(pos) {}
};

struct dpos {
  double x, y, z;
};
__device__ inline dpos loadx(const double *x, int nv, int i) { return {x[i], x[nv + i], x[2 * nv + i]}; }
template <typename R>
__device__ inline v3<R> diff(dpos a, dpos o) {
  return {R(a.x - o.x), R(a.y - o.y), R(a.z - o.z)};
}

template <typename R>
__device__ inline void store_slot(void *contrib, int slot, v3<R> f) {
  R *c = reinterpret_cast<R *>(contrib) + 3 * (size_t)slot;
  c[0] = f.x;
  c[1] = f.y;
  c[2] = f.z;
}

// Newton tangent data of triangle t (exact backward Euler and the quasi-static solve by Newton): the membrane
// Hessian at the current positions, projected to positive semi-definite, is determined by the polar rotation
// R = [R0 R1] (3x2), kappa = max(0, mu - c / tr S) and Q = sum_i max(0, 2 mu - c / s_i) v_i v_i^T over the
// eigenpairs (s_i, v_i) of the stretch S = I + e (2x2, the triangle's rest frame), c = 2 mu - lam tr(S - I).
// Stored as m_T[k * nt + t], k = 0..9: R0, R1, kappa, Q00, Q01, Q11.
template <typename R>
__device__ __noinline__ void store_tangent(const Inst &I, int t, R e00, R e01, R e11, v3<R> R0, v3<R> R1) {
  const int nt = I.nt;
  const R mu = R(I.mu), lam = R(I.lam);
  const R s00 = R(1) + e00, s11 = R(1) + e11, s01 = e01;
  const R tr = s00 + s11;
  const R c = R(2) * mu - lam * (e00 + e11);
  const R kap = fmax(R(0), mu - c / tr);
  const R d = s00 - s11, rr = sqrt(d * d + R(4) * s01 * s01);
  const R sp = R(0.5) * (tr + rr), sm = R(0.5) * (tr - rr);
  R vx = R(1), vy = R(0);   // unit eigenvector of the larger eigenvalue sp
  if (rr > R(0)) {
    if (d >= R(0)) {
      vx = d + rr;
      vy = R(2) * s01;
    } else {
      vx = R(2) * s01;
      vy = rr - d;
    }
    const R il = R(1) / sqrt(vx * vx + vy * vy);
    vx *= il;
    vy *= il;
  }
  const R qp = fmax(R(0), R(2) * mu - c / sp), qm = fmax(R(0), R(2) * mu - c / sm);
  double *T = I.m_T;
  T[t] = R0.x;
  T[nt + t] = R0.y;
  T[2 * nt + t] = R0.z;
  T[3 * nt + t] = R1.x;
  T[4 * nt + t] = R1.y;
  T[5 * nt + t] = R1.z;
  T[6 * nt + t] = kap;
  T[7 * nt + t] = qp * vx * vx + qm * vy * vy;
  T[8 * nt + t] = (qp - qm) * vx * vy;
  T[9 * nt + t] = qp * vy * vy + qm * vx * vx;
}

// ------------------------------------------------------------------ triangle pass (membrane + bending)
// TAN: the tangent data of Newton instances is written (a kernel without Newton support passes false)
template <typename R, bool TAN = true>
__device__ void tri_stencil(const Inst &I, const Data<R> &D, int t, bool want_energy) {
  const int nt = I.nt, nv = I.nv;
  const bool bend = I.t_mode[t] != MODE_NONE;
  const int nloc = bend ? 6 : 3;
  int idx[6];
  for (int j = 0; j < nloc; ++j) idx[j] = I.t_idx[j * nt + t];
  const dpos o = loadx(D.X, nv, idx[0]);
  dpos xd[3];
  v3<R> d[6];
  d[0] = zero3<R>();
  for (int j = 1; j < nloc; ++j) {
    if (idx[j] >= 0) {
      dpos xj = loadx(D.X, nv, idx[j]);
      if (j < 3) xd[j] = {xj.x - o.x, xj.y - o.y, xj.z - o.z};
      d[j] = diff<R>(xj, o);
    } else {
      d[j] = zero3<R>();
    }
  }
  v3<R> f[6];
  for (int j = 0; j < 6; ++j) f[j] = zero3<R>();
  double e_bend = 0.0, e_mem = 0.0;

  // ---- membrane
  {
    const R p = D.mD[t], q = D.mD[nt + t], r = D.mD[2 * nt + t];
    const R At = D.mAt[t];
    const R mu = R(I.mu), lam = R(I.lam);
    // FP64 Gram differences of the current and rest edge vectors a = x2 - x1, b = x3 - x1
    const double aa = xd[1].x * xd[1].x + xd[1].y * xd[1].y + xd[1].z * xd[1].z;
    const double ab = xd[1].x * xd[2].x + xd[1].y * xd[2].y + xd[1].z * xd[2].z;
    const double bb = xd[2].x * xd[2].x + xd[2].y * xd[2].y + xd[2].z * xd[2].z;
    const R g00 = R(aa - I.m_G64[t]), g01 = R(ab - I.m_G64[nt + t]), g11 = R(bb - I.m_G64[2 * nt + t]);
    // Green strain E = 1/2 Dm^-T (Ds^T Ds - Dm^T Dm) Dm^-1 with Dm^-1 = [[p, q], [0, r]]
    const R E00 = R(0.5) * p * p * g00;
    const R E01 = R(0.5) * p * (q * g00 + r * g01);
    const R E11 = R(0.5) * (q * q * g00 + R(2) * q * r * g01 + r * r * g11);
    // S = sqrt(I + 2E) = (C + sqrt(det C) I) / sqrt(tr C + 2 sqrt(det C)), written without cancellation
    const R trE = E00 + E11, detE = E00 * E11 - E01 * E01;
    const R sd = sqrt(R(1) + R(2) * trE + R(4) * detE);
    const R sdm1 = (R(2) * trE + R(4) * detE) / (sd + R(1));
    const R den = sqrt(R(4) + R(2) * trE + R(2) * sdm1);
    const R denm2 = (R(2) * trE + R(2) * sdm1) / (den + R(2));
    const R kq = sdm1 - denm2;
    const R e00 = (R(2) * E00 + kq) / den, e01 = (R(2) * E01) / den, e11 = (R(2) * E11 + kq) / den;
    const R tre = e00 + e11;
    if (want_energy) e_mem = double(At) * double(mu * (e00 * e00 + R(2) * e01 * e01 + e11 * e11) + R(0.5) * lam * tre * tre);
    // F = [a b] Dm^-1, R = F S^-1 (det S = sd)
    const v3<R> F0 = p * d[1];
    const v3<R> F1 = q * d[1] + r * d[2];
    const R S00 = R(1) + e00, S01 = e01, S11 = R(1) + e11;
    const R isd = R(1) / sd;
    const v3<R> R0 = isd * (S11 * F0 - S01 * F1);
    const v3<R> R1 = isd * (S00 * F1 - S01 * F0);
    if constexpr (TAN) {
      if (I.nl_newton) store_tangent<R>(I, t, e00, e01, e11, R0, R1);
    }
    const R s00 = R(2) * mu * e00 + lam * tre, s01 = R(2) * mu * e01, s11 = R(2) * mu * e11 + lam * tre;
    const v3<R> P0 = s00 * R0 + s01 * R1;
    const v3<R> P1 = s01 * R0 + s11 * R1;
    const v3<R> H0 = At * (p * P0 + q * P1);
    const v3<R> H1 = (At * r) * P1;
    f[0] = f[0] + H0 + H1;
    f[1] = f[1] - H0;
    f[2] = f[2] - H1;
  }

  // ---- bending (triangle-centred stencil)
  if (bend) {
    const uint8_t mode = I.t_mode[t];
    R L[3][6];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 6; ++j) L[i][j] = D.tL[(i * 6 + j) * nt + t];
    const R W00 = D.tW[t], W01 = D.tW[nt + t], W02 = D.tW[2 * nt + t], W11 = D.tW[3 * nt + t],
            W12 = D.tW[4 * nt + t], W22 = D.tW[5 * nt + t];
    v3<R> G[3];
    for (int i = 0; i < 3; ++i) {
      G[i] = zero3<R>();
      for (int j = 1; j < 6; ++j) G[i] = G[i] + L[i][j] * d[j];
    }
    if (mode == MODE_PLATE) {
      v3<R> S[3];
      S[0] = W00 * G[0] + W01 * G[1] + W02 * G[2];
      S[1] = W01 * G[0] + W11 * G[1] + W12 * G[2];
      S[2] = W02 * G[0] + W12 * G[1] + W22 * G[2];
      for (int j = 0; j < 6; ++j) f[j] = f[j] - (L[0][j] * S[0] + L[1][j] * S[1] + L[2][j] * S[2]);
      if (want_energy) e_bend = 0.5 * double(dot(G[0], S[0]) + dot(G[1], S[1]) + dot(G[2], S[2]));
    } else {
      v3<R> n;
      v3<R> c = cross(d[1], d[2]);
      R ic = R(0);
      if (mode == MODE_SHELL) {
        ic = rsqrt_<R>(dot(c, c));
        n = ic * c;
      } else {
        n = {D.tn[t], D.tn[nt + t], D.tn[2 * nt + t]};
      }
      R eps[3];
      for (int i = 0; i < 3; ++i) eps[i] = dot(n, G[i]) - D.tk0[i * nt + t];
      R sg[3];
      sg[0] = W00 * eps[0] + W01 * eps[1] + W02 * eps[2];
      sg[1] = W01 * eps[0] + W11 * eps[1] + W12 * eps[2];
      sg[2] = W02 * eps[0] + W12 * eps[1] + W22 * eps[2];
      for (int j = 0; j < 6; ++j) {
        R cj = sg[0] * L[0][j] + sg[1] * L[1][j] + sg[2] * L[2][j];
        f[j] = f[j] - cj * n;
      }
      if (mode == MODE_SHELL) {
        v3<R> g = sg[0] * G[0] + sg[1] * G[1] + sg[2] * G[2];
        v3<R> gc = ic * (g - dot(n, g) * n);
        v3<R> da = cross(d[2], gc);   // d Psi / d(x2 - x1) through the normal
        v3<R> db = cross(gc, d[1]);   // d Psi / d(x3 - x1)
        f[1] = f[1] - da;
        f[2] = f[2] - db;
        f[0] = f[0] + da + db;
      }
      if (want_energy) e_bend = 0.5 * double(eps[0] * sg[0] + eps[1] * sg[1] + eps[2] * sg[2]);
    }
  }
  const int base = t * I.kt;
  for (int j = 0; j < I.kt; ++j) store_slot<R>(I.contrib, base + j, f[j]);
  if (want_energy) {
    I.ebuf[2 * t] = e_bend;
    I.ebuf[2 * t + 1] = e_mem;
  }
}

// ------------------------------------------------------------------ edge-hinge stencils
template <typename R>
__device__ void edge_stencil(const Inst &I, const Data<R> &D, int e, bool want_energy) {
  const int ne = I.ne, nv = I.nv;
  int idx[4];
  for (int j = 0; j < 4; ++j) idx[j] = I.e_idx[j * ne + e];
  const dpos o = loadx(D.X, nv, idx[1]);
  v3<R> d[4];
  d[1] = zero3<R>();
  d[0] = diff<R>(loadx(D.X, nv, idx[0]), o);
  d[2] = diff<R>(loadx(D.X, nv, idx[2]), o);
  d[3] = idx[3] >= 0 ? diff<R>(loadx(D.X, nv, idx[3]), o) : zero3<R>();
  R L[4];
  for (int j = 0; j < 4; ++j) L[j] = D.eL[j * ne + e];
  const R w = D.ew[e];
  const v3<R> G = L[0] * d[0] + L[2] * d[2] + L[3] * d[3];
  v3<R> f[4];
  double en = 0.0;
  const uint8_t mode = I.e_mode[e];
  if (mode == MODE_PLATE) {
    const v3<R> S = w * G;
    for (int j = 0; j < 4; ++j) f[j] = (-L[j]) * S;
    if (want_energy) en = 0.5 * double(dot(G, S));
  } else {
    v3<R> n, a1, b1, a2, b2, n1, n2;
    R ic1 = R(0), ic2 = R(0), im = R(0);
    bool folded = false;
    if (mode == MODE_SHELL) {
      a1 = zero3<R>() - d[0];          // x2 - x1
      b1 = d[2] - d[0];                // x3 - x1
      a2 = d[2] - d[3];                // x3 - x4
      b2 = zero3<R>() - d[3];          // x2 - x4
      v3<R> c1 = cross(a1, b1), c2 = cross(a2, b2);
      ic1 = rsqrt_<R>(dot(c1, c1));
      ic2 = rsqrt_<R>(dot(c2, c2));
      n1 = ic1 * c1;
      n2 = ic2 * c2;
      v3<R> m = n1 + n2;
      R ml2 = dot(m, m);
      folded = ml2 < R(1e-16);
      if (folded) {
        n = n1;
      } else {
        im = rsqrt_<R>(ml2);
        n = im * m;
      }
    } else {
      n = {D.en[e], D.en[ne + e], D.en[2 * ne + e]};
    }
    const R eps = dot(n, G) - D.ek0[e];
    const R sg = w * eps;
    for (int j = 0; j < 4; ++j) f[j] = (-(sg * L[j])) * n;
    if (mode == MODE_SHELL) {
      v3<R> g = sg * G;
      v3<R> g1, g2;
      if (folded) {
        g1 = ic1 * (g - dot(n1, g) * n1);
        g2 = zero3<R>();
      } else {
        v3<R> gm = im * (g - dot(n, g) * n);
        g1 = ic1 * (gm - dot(n1, gm) * n1);
        g2 = ic2 * (gm - dot(n2, gm) * n2);
      }
      // T123 = (x1, x2, x3): c1 = (x2 - x1) x (x3 - x1)
      v3<R> da = cross(b1, g1), db = cross(g1, a1);
      f[1] = f[1] - da;
      f[2] = f[2] - db;
      f[0] = f[0] + da + db;
      // T432 = (x4, x3, x2): c2 = (x3 - x4) x (x2 - x4)
      v3<R> da2 = cross(b2, g2), db2 = cross(g2, a2);
      f[2] = f[2] - da2;
      f[1] = f[1] - db2;
      f[3] = f[3] + da2 + db2;
    }
    if (want_energy) en = 0.5 * double(eps * sg);
  }
  const int base = I.nt * I.kt + 4 * e;
  for (int j = 0; j < 4; ++j) store_slot<R>(I.contrib, base + j, f[j]);
  if (want_energy) {
    I.ebuf[2 * (I.nt + e)] = en;
    I.ebuf[2 * (I.nt + e) + 1] = 0.0;
  }
}


}  // namespace
}  // namespace shl
