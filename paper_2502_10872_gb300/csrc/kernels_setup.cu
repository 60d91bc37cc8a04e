// kernels_setup.cu -- rest-state precompute (FP64) and constant matrix assembly, once per mesh.
//
// Triangle-centred stencils (FVM hinge, Section 4.4 / App. C; smoothed hinge, Section 4.5):
//   L_p row i = (2 / (h_i + h_{i+3})) * (w_i / h_i + w_{i+3} / h_{i+3}
//               - ((1 - s_i)/h_i + (1 - s_{i+3})/h_{i+3}) w_a - (s_i/h_i + s_{i+3}/h_{i+3}) w_b)
//   for the hinge across central edge a -> b opposite vertex i (App. C Eq. 76-78), with signed feet
//   s = (X_v - X_a).(X_b - X_a) / |X_b - X_a|^2 (the s_p of App. B) in place of the unsigned ratios, so
//   the operator kills every affine field even when a foot falls outside its edge (obtuse triangles).
//   FVM hinge: W = A R^T D_b R (Eq. 38-41), R from the outward edge normals in the rest frame of App. A;
//   the twist row of R is dropped on stencils with a free edge (Section 4.4, boundary conditions).
//   Smoothed hinge: L_g = (L_p C_p)^-1 L_p (Eq. 49-50), W = A D_b (Eq. 52-53).
//   Virtual neighbours sit at M + N - L and are folded: clamped w_L' = w_L (Eq. 59), free
//   w_L' = w_M + w_N - w_L (Eq. 60-61). Stencils touching a clamped edge measure along their fixed rest
//   normal; rest-curved shells store kappa0 = L N0^T X (Eq. 43, Eq. 51, Eq. 55).
// Edge-based stencils (Section 4.3): L_m = 2 L_theta / (h1 + h4) (Eq. 9-10), weight k_b (A_123 + A_432)
//   (Eq. 16), rest normal the normalised sum of the two faces' unit normals (kappa0 of Eq. 14 for ES),
//   clamped boundary edges use L'_m of Eq. 31 and the real triangle's area and normal.
#include <cmath>

#include "internal.h"

namespace shl {
namespace {

struct d3 {
  double x, y, z;
};
__device__ inline d3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ inline d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline d3 cross(d3 a, d3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ inline double len(d3 a) { return sqrt(dot(a, a)); }

__device__ inline d3 load3(const double *soa, int n, int i) { return mk(soa[i], soa[n + i], soa[2 * n + i]); }

// distance of v from the line a-b and the signed foot coordinate
__device__ inline void foot(d3 v, d3 a, d3 b, double *h, double *s) {
  d3 e = b - a;
  double t = dot(v - a, e) / dot(e, e);
  *s = t;
  *h = len(v - a - t * e);
}

__constant__ int kHingeA[3] = {1, 2, 0};
__constant__ int kHingeB[3] = {2, 0, 1};

__global__ void k_pre_tri(const Inst *__restrict__ pI, double E, double nu, double th) {
  const Inst &I = *pI;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= I.nt) return;
  const int nt = I.nt, nv = I.nv;
  int idx[6];
  for (int j = 0; j < 6; ++j) idx[j] = I.t_idx[j * nt + t];
  uint8_t bc[3];
  for (int i = 0; i < 3; ++i) bc[i] = I.t_bc[i * nt + t];
  d3 X[6];
  for (int j = 0; j < 3; ++j) X[j] = load3(I.rest, nv, idx[j]);
  for (int i = 0; i < 3; ++i) {
    int a = kHingeA[i], b = kHingeB[i];
    X[3 + i] = idx[3 + i] >= 0 ? load3(I.rest, nv, idx[3 + i]) : X[a] + X[b] - X[i];
  }
  // ---- membrane rest data (constant-strain triangle in its own 2D frame)
  d3 e1 = X[1] - X[0], e2 = X[2] - X[0];
  d3 c = cross(e1, e2);
  double area2 = len(c);
  double l1 = len(e1);
  double scale = fmax(l1, len(e2));
  if (!(area2 > 1e-12 * scale * scale)) {
    atomicOr(I.err_flags, 1);
    return;
  }
  d3 ex = (1.0 / l1) * e1, ez = (1.0 / area2) * c;
  d3 ey = cross(ez, ex);
  double ma = l1, mb = dot(ex, e2), mc = dot(ey, e2);
  I.m_D64[t] = 1.0 / ma;
  I.m_D64[nt + t] = -mb / (ma * mc);
  I.m_D64[2 * nt + t] = 1.0 / mc;
  for (int k = 0; k < 3; ++k) I.m_D32[k * nt + t] = (float)I.m_D64[k * nt + t];
  I.m_G64[t] = dot(e1, e1);
  I.m_G64[nt + t] = dot(e1, e2);
  I.m_G64[2 * nt + t] = dot(e2, e2);
  const double area = 0.5 * area2;
  I.m_At64[t] = area * th;
  I.m_At32[t] = (float)(area * th);

  const int model = I.model;
  if (model == SHELL_EP || model == SHELL_ES) {
    I.t_mode[t] = MODE_NONE;
    return;
  }
  // ---- directional operator L_p (App. C)
  double L[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int i = 0; i < 3; ++i) {
    int a = kHingeA[i], b = kHingeB[i];
    double hi, si, hn, sn;
    foot(X[i], X[a], X[b], &hi, &si);
    foot(X[3 + i], X[a], X[b], &hn, &sn);
    if (!(hi > 1e-9 * scale) || !(hn > 1e-9 * scale)) {
      atomicOr(I.err_flags, 1);
      return;
    }
    double kk = 2.0 / (hi + hn);
    L[i][i] = kk / hi;
    L[i][3 + i] = kk / hn;
    L[i][a] = -kk * ((1.0 - si) / hi + (1.0 - sn) / hn);
    L[i][b] = -kk * (si / hi + sn / hn);
  }
  // rest corotational frame (App. A): 2D coordinates of the six nodes
  double P[6][2];
  for (int j = 0; j < 6; ++j) {
    d3 d = X[j] - X[0];
    P[j][0] = dot(d, ex);
    P[j][1] = dot(d, ey);
  }
  const double kb = E * th * th * th / (12.0 * (1.0 - nu * nu));
  const double Db[3][3] = {{kb, kb * nu, 0.0}, {kb * nu, kb, 0.0}, {0.0, 0.0, kb * 0.5 * (1.0 - nu)}};
  double D[3][3];
  const bool fvm = (model == SHELL_FP || model == SHELL_FS);
  if (fvm) {
    double R[3][3];
    bool has_free = false;
    for (int i = 0; i < 3; ++i) {
      int a = kHingeA[i], b = kHingeB[i];
      double tx = P[b][0] - P[a][0], ty = P[b][1] - P[a][1];
      double tl = sqrt(tx * tx + ty * ty);
      double mx = ty / tl, my = -tx / tl;       // outward normal of a counter-clockwise triangle
      R[0][i] = mx * mx;
      R[1][i] = my * my;
      R[2][i] = 2.0 * mx * my;
      has_free |= (bc[i] == BC_FREE);
    }
    if (has_free)
      for (int i = 0; i < 3; ++i) R[2][i] = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int l = 0; l < 3; ++l) {
        double acc = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) acc += R[p][i] * Db[p][q] * R[q][l];
        D[i][l] = acc;
      }
  } else {
    // smoothed hinge: M = L_p C_p with C_p rows (x^2/2, y^2/2, xy/2)
    double M[3][3];
    for (int i = 0; i < 3; ++i) {
      M[i][0] = M[i][1] = M[i][2] = 0.0;
      for (int j = 0; j < 6; ++j) {
        M[i][0] += L[i][j] * 0.5 * P[j][0] * P[j][0];
        M[i][1] += L[i][j] * 0.5 * P[j][1] * P[j][1];
        M[i][2] += L[i][j] * 0.5 * P[j][0] * P[j][1];
      }
    }
    double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
    double fro = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) fro += M[i][j] * M[i][j];
    fro = sqrt(fro);
    if (!(fabs(det) > 1e-12 * fro * fro * fro)) {
      atomicOr(I.err_flags, 2);
      return;
    }
    double Mi[3][3];
    Mi[0][0] = c00 / det;
    Mi[1][0] = c01 / det;
    Mi[2][0] = c02 / det;
    Mi[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
    Mi[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
    Mi[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
    Mi[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
    Mi[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
    Mi[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
    double G[3][6];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 6; ++j) G[i][j] = Mi[i][0] * L[0][j] + Mi[i][1] * L[1][j] + Mi[i][2] * L[2][j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 6; ++j) L[i][j] = G[i][j];
    for (int i = 0; i < 3; ++i)
      for (int l = 0; l < 3; ++l) D[i][l] = Db[i][l];
  }
  // ---- boundary folds of the virtual columns
  for (int i = 0; i < 3; ++i) {
    if (bc[i] == BC_INTERIOR) continue;
    int a = kHingeA[i], b = kHingeB[i];
    for (int r = 0; r < 3; ++r) {
      double cv = L[r][3 + i];
      if (bc[i] == BC_CLAMPED) {
        L[r][i] += cv;
      } else {
        L[r][a] += cv;
        L[r][b] += cv;
        L[r][i] -= cv;
      }
      L[r][3 + i] = 0.0;
    }
  }
  const bool clamped = (bc[0] == BC_CLAMPED) || (bc[1] == BC_CLAMPED) || (bc[2] == BC_CLAMPED);
  const bool shell = (model == SHELL_FS || model == SHELL_SS);
  uint8_t mode = clamped ? MODE_FIXED : (shell ? MODE_SHELL : MODE_PLATE);
  double k0[3] = {0.0, 0.0, 0.0};
  if (mode != MODE_PLATE) {
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int j = 1; j < 6; ++j) acc += L[i][j] * dot(ez, X[j] - X[0]);
      k0[i] = acc;
    }
  }
  I.t_mode[t] = mode;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 6; ++j) {
      I.t_L64[(i * 6 + j) * nt + t] = L[i][j];
      I.t_L32[(i * 6 + j) * nt + t] = (float)L[i][j];
    }
  const double Wv[6] = {area * D[0][0], area * D[0][1], area * D[0][2], area * D[1][1], area * D[1][2], area * D[2][2]};
  for (int k = 0; k < 6; ++k) {
    I.t_W64[k * nt + t] = Wv[k];
    I.t_W32[k * nt + t] = (float)Wv[k];
  }
  for (int i = 0; i < 3; ++i) {
    I.t_k064[i * nt + t] = k0[i];
    I.t_k032[i * nt + t] = (float)k0[i];
  }
  const double nf[3] = {ez.x, ez.y, ez.z};
  for (int k = 0; k < 3; ++k) {
    I.t_n64[k * nt + t] = clamped ? nf[k] : 0.0;
    I.t_n32[k * nt + t] = clamped ? (float)nf[k] : 0.0f;
  }
}

__global__ void k_pre_edge(const Inst *__restrict__ pI, double kb) {
  const Inst &I = *pI;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I.ne) return;
  const int ne = I.ne, nv = I.nv;
  int idx[4];
  for (int j = 0; j < 4; ++j) idx[j] = I.e_idx[j * ne + e];
  const bool clamped = idx[3] < 0;
  d3 X[4];
  for (int j = 0; j < 3; ++j) X[j] = load3(I.rest, nv, idx[j]);
  X[3] = clamped ? X[1] + X[2] - X[0] : load3(I.rest, nv, idx[3]);
  double h1, sp, h4, sq;
  foot(X[0], X[1], X[2], &h1, &sp);
  foot(X[3], X[1], X[2], &h4, &sq);
  double scale = len(X[2] - X[1]);
  if (!(h1 > 1e-9 * scale) || !(h4 > 1e-9 * scale)) {
    atomicOr(I.err_flags, 1);
    return;
  }
  double kk = 2.0 / (h1 + h4);
  double L[4] = {kk / h1, -kk * ((1.0 - sp) / h1 + (1.0 - sq) / h4), -kk * (sp / h1 + sq / h4), kk / h4};
  d3 c1 = cross(X[1] - X[0], X[2] - X[0]);
  double A1 = 0.5 * len(c1);
  d3 n1 = (1.0 / len(c1)) * c1;
  uint8_t mode;
  double w, k0 = 0.0;
  d3 nf = mk(0.0, 0.0, 0.0);
  if (clamped) {
    L[0] += L[3];
    L[3] = 0.0;
    w = kb * A1;
    mode = MODE_FIXED;
    nf = n1;
    for (int j = 0; j < 3; ++j) k0 += L[j] * dot(nf, X[j] - X[1]);
  } else {
    d3 c2 = cross(X[2] - X[3], X[1] - X[3]);
    double A4 = 0.5 * len(c2);
    w = kb * (A1 + A4);
    if (I.model == SHELL_ES) {
      d3 m = n1 + (1.0 / len(c2)) * c2;
      double ml = len(m);
      d3 n0 = ml < 1e-8 ? n1 : (1.0 / ml) * m;
      for (int j = 0; j < 4; ++j) k0 += L[j] * dot(n0, X[j] - X[1]);
      mode = MODE_SHELL;
    } else {
      mode = MODE_PLATE;
    }
  }
  I.e_mode[e] = mode;
  for (int j = 0; j < 4; ++j) {
    I.e_L64[j * ne + e] = L[j];
    I.e_L32[j * ne + e] = (float)L[j];
  }
  I.e_w64[e] = w;
  I.e_w32[e] = (float)w;
  I.e_k064[e] = k0;
  I.e_k032[e] = (float)k0;
  const double nfa[3] = {nf.x, nf.y, nf.z};
  for (int k = 0; k < 3; ++k) {
    I.e_n64[k * ne + e] = nfa[k];
    I.e_n32[k * ne + e] = (float)nfa[k];
  }
}

// lumped mass m_i = rho * sum over incident triangles of (A t) / 3; f_ext = m_i g (point loads added after)
__global__ void k_mass(const Inst *__restrict__ pI, double rho, double gx, double gy, double gz) {
  const Inst &I = *pI;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.nv) return;
  const int tri_slots = I.nt * I.kt;
  double m = 0.0;
  for (int q = I.vtx_ptr[i]; q < I.vtx_ptr[i + 1]; ++q) {
    int s = I.vtx_slot[q];
    if (s < tri_slots && (s % I.kt) < 3) m += I.m_At64[s / I.kt];
  }
  m *= rho / 3.0;
  I.mass[i] = m;
  I.fext[i] = m * gx;
  I.fext[I.nv + i] = m * gy;
  I.fext[2 * I.nv + i] = m * gz;
}

__global__ void k_point_loads(const Inst *__restrict__ pI, int n, const int32_t *vtx, const double *f) {
  const Inst &I = *pI;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int k = 0; k < n; ++k) {  // serial: repeated vertices accumulate in a fixed order
    int i = vtx[k];
    for (int c = 0; c < 3; ++c) I.fext[c * I.nv + i] += f[3 * k + c];
  }
}

// local constant matrices: triangle bending L^T W L (6x6), membrane 2 (mu + lam) A t grad phi grad phi
// (3x3), edge bending w L L^T (4x4)
__global__ void k_local_tri(const Inst *__restrict__ pI) {
  const Inst &I = *pI;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= I.nt) return;
  const int nt = I.nt;
  const bool edge_model = (I.model == SHELL_EP || I.model == SHELL_ES);
  const int mem_off = edge_model ? 0 : nt * 36;
  if (!edge_model) {
    double L[3][6], W[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 6; ++j) L[i][j] = I.t_L64[(i * 6 + j) * nt + t];
    const double *Wp = I.t_W64;
    W[0][0] = Wp[t];
    W[0][1] = W[1][0] = Wp[nt + t];
    W[0][2] = W[2][0] = Wp[2 * nt + t];
    W[1][1] = Wp[3 * nt + t];
    W[1][2] = W[2][1] = Wp[4 * nt + t];
    W[2][2] = Wp[5 * nt + t];
    for (int j = 0; j < 6; ++j) {
      double WL[3];
      for (int i = 0; i < 3; ++i) WL[i] = W[i][0] * L[0][j] + W[i][1] * L[1][j] + W[i][2] * L[2][j];
      for (int k = 0; k < 6; ++k) I.local[t * 36 + k * 6 + j] = L[0][k] * WL[0] + L[1][k] * WL[1] + L[2][k] * WL[2];
    }
  }
  const double d0 = I.m_D64[t], d1 = I.m_D64[nt + t], d2 = I.m_D64[2 * nt + t];
  const double g[3][2] = {{-d0, -d1 - d2}, {d0, d1}, {0.0, d2}};
  const double c = 2.0 * (I.mu + I.lam) * I.m_At64[t];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) I.local[mem_off + t * 9 + a * 3 + b] = c * (g[a][0] * g[b][0] + g[a][1] * g[b][1]);
}

__global__ void k_local_edge(const Inst *__restrict__ pI) {
  const Inst &I = *pI;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I.ne) return;
  const int off = I.nt * 9;
  double L[4];
  for (int j = 0; j < 4; ++j) L[j] = I.e_L64[j * I.ne + e];
  const double w = I.e_w64[e];
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 4; ++k) I.local[off + e * 16 + j * 4 + k] = w * L[j] * L[k];
}

// A = M + dt^2 (K_b + K_m), identity rows / columns at pinned vertices; also the Jacobi inverse diagonal
__global__ void k_assemble(const Inst *__restrict__ pI) {
  const Inst &I = *pI;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.nv) return;
  const int s = i >> 5, lane = i & 31;
  const int base = I.sl_ptr[s];
  const int width = (I.sl_ptr[s + 1] - base) >> 5;
  const double dt2 = I.dt * I.dt;
  const int dp = I.diag_pos[i];
  const bool pin_i = I.pinned[i] != 0;
  double rowsum = 0.0;
  for (int k = 0; k < width; ++k) {
    const int p = base + 32 * k + lane;
    const int c = I.sl_col[p];
    double v = 0.0;
    for (int q = I.asm_ptr[p]; q < I.asm_ptr[p + 1]; ++q) v += I.local[I.asm_src[q]];
    v *= dt2;
    if (p == dp) v += I.mass[i];
    if (pin_i || I.pinned[c]) v = (p == dp) ? 1.0 : 0.0;
    I.val64[p] = v;
    I.val32[p] = (float)v;
    rowsum += v;
  }
  I.rs32[i] = (float)rowsum;
  const double dinv = 1.0 / I.val64[dp];
  I.dinv64[i] = dinv;
  I.dinv32[i] = (float)dinv;
}

}  // namespace

cudaError_t launch_precompute(const Inst *d, const Inst &h, double E, double nu, double th, double rho,
                              cudaStream_t st) {
  const int B = 128;
  if (h.nt > 0) k_pre_tri<<<(h.nt + B - 1) / B, B, 0, st>>>(d, E, nu, th);
  if (h.ne > 0) k_pre_edge<<<(h.ne + B - 1) / B, B, 0, st>>>(d, E * th * th * th / (12.0 * (1.0 - nu * nu)));
  return cudaGetLastError();
}

cudaError_t launch_mass(const Inst *d, const Inst &h, double rho, const double g[3], int n_loads,
                        const int32_t *d_lv, const double *d_lf, cudaStream_t st) {
  const int B = 256;
  k_mass<<<(h.nv + B - 1) / B, B, 0, st>>>(d, rho, g[0], g[1], g[2]);
  if (n_loads > 0) k_point_loads<<<1, 32, 0, st>>>(d, n_loads, d_lv, d_lf);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const Inst *d, const Inst &h, cudaStream_t st) {
  const int B = 128;
  if (h.nt > 0) k_local_tri<<<(h.nt + B - 1) / B, B, 0, st>>>(d);
  if (h.ne > 0) k_local_edge<<<(h.ne + B - 1) / B, B, 0, st>>>(d);
  k_assemble<<<(h.nv + B - 1) / B, B, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace shl
