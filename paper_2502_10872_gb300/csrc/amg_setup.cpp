// amg_setup.cpp -- smoothed-aggregation algebraic multigrid (Vanek, Mandel, Brezina 1996) for the
// constant step matrix A = M + dt^2 K. The matrix never changes, so the hierarchy is built once per mesh;
// the V-cycle runs inside the persistent solve kernel as the PCG preconditioner.
//
//   strength    |a_ij| >= theta sqrt(a_ii a_jj)
//   aggregates  greedy: a node whose strong neighbours are all free roots an aggregate with them; leftover
//               nodes join a neighbouring aggregate; the rest form their own
//   P           (I - omega D^-1 A) P0, P0 the aggregate indicator (near-null space: constants), omega = 4/(3 rho)
//   Rs, Ps      R (I - omega A D^-1) and its transpose: the damped-Jacobi sweeps of a V(1,1) cycle folded
//               into the transfers, so that a level's down step (residual and restriction) and its up step
//               (correction and post-smoothing) each read only vectors the previous step wrote
//   A_c         P^T A P (Galerkin), repeated until the level is small; the coarsest is inverted densely
//   dense end   from the first level of at most dense_max rows down, the cycle (started from zero) is a fixed
//               linear map of that level's right-hand side: stored as a dense matrix, built by applying the
//               same steps to the unit vectors
#include "amg_setup.h"

#include <algorithm>
#include <cmath>
#include <system_error>
#include <thread>

namespace shl {

namespace {

// Host threads for the row-parallel parts of the set-up (sparse products, the smoothed prolongation, the
// power iteration): up to setup_threads_cap, and only for matrices of at least setup_threads_min_rows rows,
// large enough to repay starting them. (Variables, so that the host check can compare thread counts.)
int setup_threads_cap = 4;
int setup_threads_min_rows = 16384;
int setup_threads(int n) {
  if (n < setup_threads_min_rows) return 1;
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min((unsigned)std::max(1, setup_threads_cap), hw));
}

// Runs fn(t, lo, hi) for the T contiguous chunks [lo, hi) of [0, n), chunk 0 on the calling thread. A chunk
// whose thread cannot be started runs on the calling thread instead (each chunk writes only its own outputs,
// so the result is the same).
template <typename F>
void parallel_chunks(int n, int T, F &&fn) {
  auto run = [&](int t) { fn(t, (int)((long long)n * t / T), (int)((long long)n * (t + 1) / T)); };
  if (T <= 1) {
    run(0);
    return;
  }
  std::vector<std::thread> th;
  int started = 1;
  try {
    for (; started < T; ++started) th.emplace_back(run, started);
  } catch (const std::system_error &) {
  }
  run(0);
  for (int t = started; t < T; ++t) run(t);
  for (std::thread &x : th) x.join();
}

// Per-thread scratch of a row computation: a dense marker and accumulator over the columns, the row's columns.
struct RowWork {
  std::vector<int32_t> mark;
  std::vector<double> acc;
  std::vector<int32_t> cols;
};

// CSR matrix of n rows and m columns whose row i row_fn(i, work, cols, vals) appends. Rows are computed by
// contiguous chunks on setup_threads(n) threads, each row exactly as a serial loop computes it, so the
// matrix does not depend on the number of threads.
template <typename F>
HostCsr build_rows(int n, int m, F &&row_fn) {
  const int T = setup_threads(n);
  std::vector<std::vector<int32_t>> cols(T);
  std::vector<std::vector<double>> vals(T);
  std::vector<int32_t> len(n);
  parallel_chunks(n, T, [&](int t, int lo, int hi) {
    RowWork w;
    w.mark.assign(m, -1);
    w.acc.assign(m, 0.0);
    for (int i = lo; i < hi; ++i) {
      const size_t before = cols[t].size();
      row_fn(i, w, cols[t], vals[t]);
      len[i] = (int32_t)(cols[t].size() - before);
    }
  });
  HostCsr C;
  C.n = n;
  C.m = m;
  C.ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) C.ptr[i + 1] = C.ptr[i] + len[i];
  C.col.reserve(C.ptr[n]);
  C.val.reserve(C.ptr[n]);
  for (int t = 0; t < T; ++t) {
    C.col.insert(C.col.end(), cols[t].begin(), cols[t].end());
    C.val.insert(C.val.end(), vals[t].begin(), vals[t].end());
  }
  return C;
}

HostCsr transpose(const HostCsr &M) {
  HostCsr T;
  T.n = M.m;
  T.m = M.n;
  T.ptr.assign(T.n + 1, 0);
  for (int32_t c : M.col) T.ptr[c + 1]++;
  for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(M.col.size());
  T.val.resize(M.val.size());
  std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < M.n; ++i)
    for (int q = M.ptr[i]; q < M.ptr[i + 1]; ++q) {
      int k = fill[M.col[q]]++;
      T.col[k] = i;
      T.val[k] = M.val[q];
    }
  return T;
}

// C = A * B (sparse, rows accumulated with a dense marker)
HostCsr multiply(const HostCsr &A, const HostCsr &B) {
  return build_rows(A.n, B.m, [&](int i, RowWork &w, std::vector<int32_t> &oc, std::vector<double> &ov) {
    w.cols.clear();
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      const int k = A.col[q];
      const double a = A.val[q];
      for (int r = B.ptr[k]; r < B.ptr[k + 1]; ++r) {
        const int j = B.col[r];
        if (w.mark[j] != i) {
          w.mark[j] = i;
          w.acc[j] = 0.0;
          w.cols.push_back(j);
        }
        w.acc[j] += a * B.val[r];
      }
    }
    std::sort(w.cols.begin(), w.cols.end());
    for (int j : w.cols) {
      oc.push_back(j);
      ov.push_back(w.acc[j]);
    }
  });
}

double diag_of(const HostCsr &A, int i) {
  for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
    if (A.col[q] == i) return A.val[q];
  return 0.0;
}

// spectral radius of D^-1 A by power iteration (an upper estimate is fine for the weights)
double rho_dinv_a(const HostCsr &A, const std::vector<double> &dinv) {
  const int n = A.n;
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3);
  double lam = 1.0;
  const int T = setup_threads(n);
  for (int it = 0; it < 20; ++it) {
    parallel_chunks(n, T, [&](int, int lo, int hi) {
      for (int i = lo; i < hi; ++i) {
        double s = 0.0;
        for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += A.val[q] * x[A.col[q]];
        y[i] = dinv[i] * s;
      }
    });
    double nrm = 0.0;   // summed in row order, as the rows were before
    for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
    nrm = std::sqrt(nrm);
    double xn = 0.0;
    for (int i = 0; i < n; ++i) xn += x[i] * x[i];
    lam = nrm / std::sqrt(xn);
    if (!(nrm > 0)) break;
    for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
  }
  return lam * 1.05;   // safety margin for the unconverged power iteration
}

// returns the number of aggregates; agg[i] = -1 for rows left out (isolated)
int aggregate(const HostCsr &A, double theta, std::vector<int32_t> &agg) {
  const int n = A.n;
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = std::fabs(diag_of(A, i));
  auto strong = [&](int i, int q) {
    const int j = A.col[q];
    return j != i && std::fabs(A.val[q]) >= theta * std::sqrt(d[i] * d[j]);
  };
  agg.assign(n, -2);   // -2 = free
  int na = 0;
  std::vector<char> isolated(n, 0);
  for (int i = 0; i < n; ++i) {
    bool any = false;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) any |= strong(i, q);
    if (!any) {
      isolated[i] = 1;
      agg[i] = -1;
    }
  }
  // pass 1: roots whose strong neighbourhood is entirely free
  for (int i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    bool free_nb = true;
    for (int q = A.ptr[i]; q < A.ptr[i + 1] && free_nb; ++q)
      if (strong(i, q) && agg[A.col[q]] != -2) free_nb = false;
    if (!free_nb) continue;
    agg[i] = na;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q)) agg[A.col[q]] = na;
    ++na;
  }
  // pass 2: join the strongest aggregated neighbour
  std::vector<int32_t> agg1 = agg;
  for (int i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    double best = -1.0;
    int ba = -2;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q) && agg[A.col[q]] >= 0 && std::fabs(A.val[q]) > best) {
        best = std::fabs(A.val[q]);
        ba = agg[A.col[q]];
      }
    agg1[i] = ba;
  }
  agg = agg1;
  // pass 3: what is left forms aggregates with its free strong neighbours
  for (int i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    agg[i] = na;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q) && agg[A.col[q]] == -2) agg[A.col[q]] = na;
    ++na;
  }
  return na;
}

bool dense_inverse(const HostCsr &A, std::vector<double> &inv) {
  const int n = A.n;
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) L[(size_t)i * n + A.col[q]] = A.val[q];
  // Cholesky (lower), in place
  for (int j = 0; j < n; ++j) {
    double s = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(s > 0)) return false;
    const double ljj = std::sqrt(s);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = L[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> e(n), y(n);
  for (int c = 0; c < n; ++c) {
    std::fill(e.begin(), e.end(), 0.0);
    e[c] = 1.0;
    for (int i = 0; i < n; ++i) {
      double t = e[i];
      for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * y[k];
      y[i] = t / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * e[k];
      e[i] = t / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = e[i];
  }
  return true;
}

void csr_apply(const HostCsr &M, const std::vector<double> &x, std::vector<double> &y) {
  y.assign(M.n, 0.0);
  for (int i = 0; i < M.n; ++i) {
    double s = 0.0;
    for (int q = M.ptr[i]; q < M.ptr[i + 1]; ++q) s += M.val[q] * x[M.col[q]];
    y[i] = s;
  }
}

// y = V-cycle of levels >= l applied to b from a zero guess, with the steps of the GPU cycle: pre-smoothing
// x = omega D^-1 b, residual, restriction, the coarser cycle, correction x += P y_c, post-smoothing
// y = x + omega D^-1 (b - A x); the coarsest level is solved with its dense inverse or damped-Jacobi sweeps.
void vcycle_host(const HostAmg &H, int l, const std::vector<double> &b, std::vector<double> &y) {
  const HostAmgLevel &V = H.levels[l];
  const int n = V.A.n;
  std::vector<double> t;
  if (l == (int)H.levels.size() - 1) {
    if (H.coarse_sweeps == 0) {
      y.assign(n, 0.0);
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += H.coarse_inv[(size_t)i * n + j] * b[j];
        y[i] = s;
      }
    } else {
      y.resize(n);
      for (int i = 0; i < n; ++i) y[i] = V.omega * V.dinv[i] * b[i];
      for (int sw = 1; sw < H.coarse_sweeps; ++sw) {
        csr_apply(V.A, y, t);
        for (int i = 0; i < n; ++i) y[i] += V.omega * V.dinv[i] * (b[i] - t[i]);
      }
    }
    return;
  }
  std::vector<double> x(n), r(n), bc, yc, px;
  for (int i = 0; i < n; ++i) x[i] = V.omega * V.dinv[i] * b[i];
  csr_apply(V.A, x, t);
  for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
  csr_apply(V.R, r, bc);
  vcycle_host(H, l + 1, bc, yc);
  csr_apply(V.P, yc, px);
  for (int i = 0; i < n; ++i) x[i] += px[i];
  csr_apply(V.A, x, t);
  y.resize(n);
  for (int i = 0; i < n; ++i) y[i] = x[i] + V.omega * V.dinv[i] * (b[i] - t[i]);
}

void finish_level(HostAmgLevel &L) {
  const int n = L.A.n;
  L.dinv.resize(n);
  L.rowsum.resize(n);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int q = L.A.ptr[i]; q < L.A.ptr[i + 1]; ++q) s += L.A.val[q];
    L.rowsum[i] = s;
    L.dinv[i] = 1.0 / diag_of(L.A, i);
  }
  L.omega = 4.0 / (3.0 * rho_dinv_a(L.A, L.dinv));
}

}  // namespace

void build_amg(const HostCsr &A0, HostAmg *out, int max_levels, int coarse_max, double theta, int dense_max) {
  HostAmg &H = *out;
  H = HostAmg();
  H.levels.emplace_back();
  H.levels[0].A = A0;
  finish_level(H.levels[0]);
  while ((int)H.levels.size() < max_levels) {
    HostAmgLevel &F = H.levels.back();
    const int n = F.A.n;
    if (n <= coarse_max) break;
    std::vector<int32_t> agg;
    const int na = aggregate(F.A, theta, agg);
    if (na == 0 || na > (int)(0.8 * n)) break;   // coarsening stalled
    // P = (I - omega D^-1 A) P0
    const HostCsr P = build_rows(n, na, [&](int i, RowWork &w, std::vector<int32_t> &oc, std::vector<double> &ov) {
      w.cols.clear();
      auto add = [&](int c, double v) {
        if (w.mark[c] != i) {
          w.mark[c] = i;
          w.acc[c] = 0.0;
          w.cols.push_back(c);
        }
        w.acc[c] += v;
      };
      if (agg[i] >= 0) add(agg[i], 1.0);
      if (agg[i] != -1) {   // rows left out (isolated) get no prolongation
        for (int q = F.A.ptr[i]; q < F.A.ptr[i + 1]; ++q) {
          const int j = F.A.col[q];
          if (agg[j] >= 0) add(agg[j], -F.omega * F.dinv[i] * F.A.val[q]);
        }
      }
      std::sort(w.cols.begin(), w.cols.end());
      for (int c : w.cols)
        if (w.acc[c] != 0.0) {
          oc.push_back(c);
          ov.push_back(w.acc[c]);
        }
    });
    F.P = P;
    F.R = transpose(P);
    const HostCsr AP = multiply(F.A, P);
    // Ps = P - omega D^-1 (A P), merged row by row (both rows sorted by column), and Rs = Ps^T
    F.Ps = build_rows(n, na, [&](int i, RowWork &, std::vector<int32_t> &oc, std::vector<double> &ov) {
      int q = P.ptr[i];
      const int q1 = P.ptr[i + 1];
      const double s = -F.omega * F.dinv[i];
      for (int k = AP.ptr[i]; k < AP.ptr[i + 1]; ++k) {
        for (; q < q1 && P.col[q] < AP.col[k]; ++q) {
          oc.push_back(P.col[q]);
          ov.push_back(P.val[q]);
        }
        double v = s * AP.val[k];
        if (q < q1 && P.col[q] == AP.col[k]) v += P.val[q++];
        oc.push_back(AP.col[k]);
        ov.push_back(v);
      }
      for (; q < q1; ++q) {
        oc.push_back(P.col[q]);
        ov.push_back(P.val[q]);
      }
    });
    const HostCsr &Ps = F.Ps;
    F.Rs = transpose(Ps);
    HostCsr Ac = multiply(F.R, AP);
    H.levels.emplace_back();
    H.levels.back().A = Ac;
    finish_level(H.levels.back());
  }
  HostAmgLevel &C = H.levels.back();
  if (C.A.n <= coarse_max && dense_inverse(C.A, H.coarse_inv)) {
    H.coarse_sweeps = 0;
  } else {
    H.coarse_inv.clear();
    H.coarse_sweeps = 8;
  }
  // dense operator of the cycle below the first small level: column j = cycle applied to e_j
  const int L = (int)H.levels.size();
  for (int l = 1; l < L; ++l) {
    const int n = H.levels[l].A.n;
    if (n > dense_max) continue;
    H.dense_level = l;
    H.dense_n = n;
    H.dense.assign((size_t)n * n, 0.0);
    std::vector<double> e(n, 0.0), y;
    for (int j = 0; j < n; ++j) {
      e[j] = 1.0;
      vcycle_host(H, l, e, y);
      e[j] = 0.0;
      for (int i = 0; i < n; ++i) H.dense[(size_t)j * n + i] = y[i];
    }
    break;
  }
}

HostSell to_sell4(const HostCsr &M) {
  HostSell S;
  S.n = M.n;
  S.n_slices = (M.n + 7) / 8;
  S.sl_ptr.assign(S.n_slices + 1, 0);
  for (int s = 0; s < S.n_slices; ++s) {
    int w = 0;
    for (int i = 0; i < 8; ++i) {
      const int r = s * 8 + i;
      if (r < M.n) w = std::max(w, (M.ptr[r + 1] - M.ptr[r] + 3) / 4);
    }
    S.sl_ptr[s + 1] = S.sl_ptr[s] + 32 * w;
  }
  const int nnz = S.sl_ptr[S.n_slices];
  S.sl_col.assign(nnz, 0);
  S.val.assign(nnz, 0.0);
  for (int r = 0; r < M.n; ++r) {
    const int s = r / 8, i = r % 8;
    for (int k = 0; k < M.ptr[r + 1] - M.ptr[r]; ++k) {
      const int pos = S.sl_ptr[s] + 32 * (k / 4) + 4 * i + k % 4;
      S.sl_col[pos] = M.col[M.ptr[r] + k];
      S.val[pos] = M.val[M.ptr[r] + k];
    }
  }
  return S;
}

HostSell to_sell(const HostCsr &M) {
  HostSell S;
  S.n = M.n;
  S.n_slices = (M.n + 31) / 32;
  S.sl_ptr.assign(S.n_slices + 1, 0);
  for (int s = 0; s < S.n_slices; ++s) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      const int r = s * 32 + l;
      if (r < M.n) w = std::max(w, M.ptr[r + 1] - M.ptr[r]);
    }
    S.sl_ptr[s + 1] = S.sl_ptr[s] + 32 * w;
  }
  const int nnz = S.sl_ptr[S.n_slices];
  S.sl_col.assign(nnz, 0);
  S.val.assign(nnz, 0.0);
  for (int s = 0; s < S.n_slices; ++s) {
    const int w = (S.sl_ptr[s + 1] - S.sl_ptr[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int r = s * 32 + l;
      for (int k = 0; k < w; ++k) {
        const int pos = S.sl_ptr[s] + 32 * k + l;
        if (r < M.n && k < M.ptr[r + 1] - M.ptr[r]) {
          S.sl_col[pos] = M.col[M.ptr[r] + k];
          S.val[pos] = M.val[M.ptr[r] + k];
        } else {
          S.sl_col[pos] = 0;
          S.val[pos] = 0.0;
        }
      }
    }
  }
  return S;
}

}  // namespace shl
