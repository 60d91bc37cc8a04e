// Host check of the multigrid set-up used by the solve kernel (built and run by test_host_multigrid.py; no
// GPU). Reads a scalar CSR matrix (int32 n, nnz; int32 ptr[n+1], col[nnz]; double val[nnz]), builds the
// hierarchy with the library's own set-up code, checks that the hierarchy is bitwise the same when its
// row-parallel parts run on 1 or 3 threads, and checks on every level with a next one:
//   1. Ps is exactly Rs^T (structure and values);
//   2. Rs equals R (I - omega A D^-1) formed by an explicit sparse product;
// and, for three right-hand sides, that the cycle the kernel runs (per level one down step r = b - A x,
// bc = Rs b with x = omega D^-1 b, one up step y = x + omega D^-1 r + Ps yc; the dense coarse operator or the
// coarsest solve below) equals the plain V(1,1) cycle of vcycle_host (pre-smoothing, residual, restriction,
// correction, post-smoothing). Prints "OK <worst relative difference>" or "FAIL <what>".
#include "../paper_2502_10872_gb300/csrc/amg_setup.cpp"

#include <cstdio>
#include <random>

using namespace shl;

namespace {

void folded_cycle(const HostAmg &H, int l, int top, const std::vector<double> &b, std::vector<double> &y) {
  const HostAmgLevel &V = H.levels[l];
  const int n = V.A.n;
  if (l == top) {
    if (H.dense_level == top) {
      y.assign(n, 0.0);
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) y[i] += H.dense[(size_t)j * n + i] * b[j];
    } else {
      vcycle_host(H, l, b, y);   // the coarsest level: same solve on both sides
    }
    return;
  }
  std::vector<double> x(n), r(n), t, bc, yc, py;
  for (int i = 0; i < n; ++i) x[i] = V.omega * V.dinv[i] * b[i];
  csr_apply(V.A, x, t);
  for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
  csr_apply(V.Rs, b, bc);
  folded_cycle(H, l + 1, top, bc, yc);
  csr_apply(V.Ps, yc, py);
  y.resize(n);
  for (int i = 0; i < n; ++i) y[i] = x[i] + V.omega * V.dinv[i] * r[i] + py[i];
}

double max_abs(const std::vector<double> &v) {
  double m = 0.0;
  for (double a : v) m = std::max(m, std::fabs(a));
  return m;
}

}  // namespace

int main(int argc, char **argv) {
  if (argc < 2) return 2;
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 2;
  int hdr[2];
  if (fread(hdr, 4, 2, f) != 2) return 2;
  HostCsr A;
  A.n = A.m = hdr[0];
  A.ptr.resize(A.n + 1);
  A.col.resize(hdr[1]);
  A.val.resize(hdr[1]);
  const size_t got = fread(A.ptr.data(), 4, A.n + 1, f) + fread(A.col.data(), 4, hdr[1], f) +
                     fread(A.val.data(), 8, hdr[1], f);
  fclose(f);
  if (got != (size_t)A.n + 1 + 2 * (size_t)hdr[1]) return 2;
  HostAmg H;
  build_amg(A, &H);
  // the same hierarchy, bit for bit, whatever the number of set-up threads (the row-parallel parts are
  // forced onto 1 and onto 3 threads, for any matrix size)
  {
    const int cap = setup_threads_cap, min_rows = setup_threads_min_rows;
    setup_threads_min_rows = 1;
    HostAmg H1, H3;
    setup_threads_cap = 1;
    build_amg(A, &H1);
    setup_threads_cap = 3;
    build_amg(A, &H3);
    setup_threads_cap = cap;
    setup_threads_min_rows = min_rows;
    auto same_csr = [](const HostCsr &a, const HostCsr &b) {
      return a.n == b.n && a.m == b.m && a.ptr == b.ptr && a.col == b.col && a.val == b.val;
    };
    const HostAmg *hs[3] = {&H, &H1, &H3};
    for (int k = 1; k < 3; ++k) {
      const HostAmg &X = *hs[k];
      bool same = X.levels.size() == H.levels.size() && X.coarse_inv == H.coarse_inv &&
                  X.coarse_sweeps == H.coarse_sweeps && X.dense_level == H.dense_level && X.dense == H.dense;
      for (size_t l = 0; same && l < H.levels.size(); ++l) {
        const HostAmgLevel &a = H.levels[l], &b = X.levels[l];
        same = same_csr(a.A, b.A) && same_csr(a.P, b.P) && same_csr(a.R, b.R) && same_csr(a.Rs, b.Rs) &&
               same_csr(a.Ps, b.Ps) && a.dinv == b.dinv && a.rowsum == b.rowsum && a.omega == b.omega;
      }
      if (!same) {
        printf("FAIL the hierarchy depends on the number of set-up threads (%d)\n", k == 1 ? 1 : 3);
        return 1;
      }
    }
  }
  const int L = (int)H.levels.size();
  if (L < 2) {
    printf("FAIL no hierarchy (%d level)\n", L);
    return 1;
  }
  for (int l = 0; l + 1 < L; ++l) {
    const HostAmgLevel &V = H.levels[l];
    const HostCsr T = transpose(V.Rs);
    if (T.ptr != V.Ps.ptr || T.col != V.Ps.col || T.val != V.Ps.val) {
      printf("FAIL level %d: Ps is not Rs^T\n", l);
      return 1;
    }
    HostCsr S = V.A;   // I - omega A D^-1
    for (int i = 0; i < S.n; ++i)
      for (int q = S.ptr[i]; q < S.ptr[i + 1]; ++q)
        S.val[q] = (S.col[q] == i ? 1.0 : 0.0) - V.omega * V.A.val[q] * V.dinv[S.col[q]];
    const HostCsr E = multiply(V.R, S);
    // compare as dense rows (structural zeros may differ)
    double worst = 0.0, scale = max_abs(V.Rs.val);
    std::vector<double> row(V.Rs.m, 0.0);
    for (int i = 0; i < V.Rs.n; ++i) {
      for (int q = V.Rs.ptr[i]; q < V.Rs.ptr[i + 1]; ++q) row[V.Rs.col[q]] += V.Rs.val[q];
      for (int q = E.ptr[i]; q < E.ptr[i + 1]; ++q) row[E.col[q]] -= E.val[q];
      for (int q = V.Rs.ptr[i]; q < V.Rs.ptr[i + 1]; ++q) worst = std::max(worst, std::fabs(row[V.Rs.col[q]]));
      for (int q = E.ptr[i]; q < E.ptr[i + 1]; ++q) worst = std::max(worst, std::fabs(row[E.col[q]]));
      for (int q = V.Rs.ptr[i]; q < V.Rs.ptr[i + 1]; ++q) row[V.Rs.col[q]] = 0.0;
      for (int q = E.ptr[i]; q < E.ptr[i + 1]; ++q) row[E.col[q]] = 0.0;
    }
    if (!(worst <= 1e-12 * scale)) {
      printf("FAIL level %d: Rs differs from R (I - omega A D^-1) by %.3e (scale %.3e)\n", l, worst, scale);
      return 1;
    }
  }
  const int top = H.dense_level > 0 ? H.dense_level : L - 1;
  std::mt19937 g(11);
  std::normal_distribution<double> N;
  double worst = 0.0;
  for (int t = 0; t < 3; ++t) {
    std::vector<double> b(A.n), y0, y1;
    for (double &v : b) v = N(g);
    if (t == 2)
      for (int i = 0; i < A.n; ++i) b[i] = 1.0 + 1e-3 * i;   // smooth: the coarse correction dominates
    vcycle_host(H, 0, b, y0);
    folded_cycle(H, 0, top, b, y1);
    double d = 0.0, s = 0.0;
    for (int i = 0; i < A.n; ++i) {
      d += (y0[i] - y1[i]) * (y0[i] - y1[i]);
      s += y0[i] * y0[i];
    }
    worst = std::max(worst, std::sqrt(d / s));
  }
  if (!(worst <= 1e-12)) {
    printf("FAIL folded cycle differs from the plain V(1,1) cycle by %.3e\n", worst);
    return 1;
  }
  printf("OK %.3e levels %d top %d\n", worst, L, top);
  return 0;
}
