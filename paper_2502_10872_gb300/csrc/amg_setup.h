// amg_setup.h -- smoothed-aggregation multigrid hierarchy of the constant step matrix (host, once per mesh).
#pragma once
#include <cstdint>
#include <vector>

namespace shl {

struct HostCsr {
  int n = 0, m = 0;                 // rows, columns
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
};

// SELL-32 image of a CSR matrix (padding: own row / column 0 with value 0)
struct HostSell {
  int n = 0, n_slices = 0;
  std::vector<int32_t> sl_ptr, sl_col;
  std::vector<double> val;
};

struct HostAmgLevel {
  HostCsr A;                        // level operator (level 0: the step matrix)
  HostCsr P;                        // prolongation: rows of this level -> columns of the next
  HostCsr R;                        // restriction P^T
  // The smoother folded into the transfers (what the GPU cycle applies): Rs = R (I - omega A D^-1) maps the
  // level's right-hand side b to the restricted residual of its pre-smoothing from zero, R (b - A omega
  // D^-1 b); Ps = Rs^T = (I - omega D^-1 A) P maps the coarse solution to the coarse correction plus the
  // post-smoothing sweep's response to it.
  HostCsr Rs, Ps;
  std::vector<double> dinv;         // 1 / diag(A)
  std::vector<double> rowsum;       // sum_j A_ij (FP64)
  double omega = 0.0;               // damped-Jacobi weight 4 / (3 rho(D^-1 A))
};

struct HostAmg {
  std::vector<HostAmgLevel> levels; // levels[L-1] is the coarsest
  std::vector<double> coarse_inv;   // dense inverse of the coarsest operator (row-major), empty if none
  int coarse_sweeps = 0;            // Jacobi sweeps on the coarsest level when it is too large to invert
  // The V-cycle restricted to levels >= dense_level (started from zero) is a fixed linear map of that level's
  // right-hand side: dense holds it as a dense n x n matrix, column-major (dense_level = -1: none).
  int dense_level = -1;
  int dense_n = 0;
  std::vector<double> dense;
};

// Builds the hierarchy of the SPD matrix A (CSR, diagonal present). Rows whose only entry is the diagonal
// (pinned vertices) are left out of the coarse spaces: the smoother solves them exactly.
// dense_max: the first level l >= 1 of at most dense_max rows gets the dense operator of the cycle below it.
void build_amg(const HostCsr &A, HostAmg *out, int max_levels = 12, int coarse_max = 48, double theta = 0.08,
               int dense_max = 400);

HostSell to_sell(const HostCsr &M);

// SELL with 4 lanes per row (for the long rows of the restriction): slices of 8 rows; entry k of the slice's
// row i (i = 0..7) sits at sl_ptr[s] + 32 (k / 4) + 4 i + k % 4, padding column 0 with value 0.
HostSell to_sell4(const HostCsr &M);

}  // namespace shl
