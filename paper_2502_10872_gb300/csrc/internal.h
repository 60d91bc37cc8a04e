// internal.h -- device-side data layout of the thin plate / shell library (not part of the public ABI).
//
// One simulation ("instance") owns one device block holding everything below. All per-vertex vectors are
// structure-of-arrays [3][nv] (coalesced per-row access) except the vector the SpMV gathers, which is
// array-of-structures [nv][4] so one gather is one 16-byte (FP32) or two 16-byte (FP64) loads.
// The matrix is the scalar constant matrix A = M + dt^2 (K_b + K_m) (every 3x3 block of the bending and
// membrane Hessians is a multiple of I_3, Eq. 21 / 41 / 53), stored as SELL-32: slices of 32 rows,
// column-major inside a slice, width = the longest row of the slice.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/shell.h"

namespace shl {

constexpr int kSlice = 32;          // SELL slice height (one warp)
constexpr int kBlock = 256;         // threads of every CTA of the persistent solve kernel
constexpr int kForceBlock = 128;    // threads of a force tile
constexpr int kMaxTeamWaitMs = 4000;  // default bound of a team-barrier wait (Sched::wait_ns)
constexpr int kBarWords = 64;       // barrier words per team (256 bytes): a 64-bit arrival counter at [0, 2),
                                    // the rest unused (one team's words do not share a cache line with
                                    // another team's)

// stencil modes
enum : uint8_t { MODE_PLATE = 0, MODE_SHELL = 1, MODE_FIXED = 2, MODE_NONE = 3 };
// boundary code of a triangle-stencil hinge
enum : uint8_t { BC_INTERIOR = 0, BC_FREE = 1, BC_CLAMPED = 2 };

struct InstStatus {
  int32_t err;          // SHELL_OK or the code that stopped this instance
  int32_t steps_done;   // committed steps (cumulative; the host takes differences)
  int32_t last_iters;   // PCG iterations of the last committed step
  int32_t last_rounds;  // refinement rounds of the last committed step
  long long total_iters;
  double rel_res;       // relative residual of the last committed step
  int32_t fail_step;    // steps_done when the failure happened
  int32_t team_size;    // CTAs that solved this instance in the last step
  long long total_rounds;
  long long last_ns;    // device time of the last step's solve of this instance (right-hand side to commit)
  long long max_ns;     // longest solve time since the status was last gathered (the gather resets it)
  int32_t nl_flags;     // bit 0: a step's chord iteration is in progress; bit 1: last step stopped at nl_max
  int32_t nl_iters;     // chord iterations of the step in progress / of the last committed step
  double nl_r0;         // ||R(0)||^2 of the step in progress (= ||b||^2 of its first solve)
  long long nl_step_pcg;  // PCG iterations summed over the chord iterations of the step in progress
};

// Per-block gather lists of a SELL matrix (device pointers): block b (256 rows, or 64 rows for matrices with 4
// lanes per row) stages the vector entries col[b * max .. b * max + max) in shared memory (lists padded to
// the longest, max); c16 is each stored entry's index into its block's list; own[b] is the local index of
// the block's first row (square matrices). max = 0: no lists.
struct HaloDev {
  int32_t *col, *own;
  uint16_t *c16;
  int32_t max, pad;
};

// One level of the smoothed-aggregation multigrid preconditioner (device pointers). P (rows of this level ->
// columns of the next) and the level-0 operator are SELL-32; R = P^T (rows of the next level -> columns of
// this one) and the coarse operators A (levels >= 1), whose rows are long, are SELL with 4 lanes per row
// (slices of 8 rows, entry k of slice row i at ptr[s] + 32 (k / 4) + 4 i + k % 4), with gather lists over
// 64-row blocks. Level vectors are array-of-structures [n][4] in the solve precision.
struct AmgDev {
  int32_t n, n_next;
  int32_t *a_ptr, *a_col;
  float *a_val32;
  double *a_val64;
  float *rs32;                   // row sums (FP64 sum, rounded) for the FP32 difference-form SpMV
  float *dinv32;
  double *dinv64;
  int32_t *p_ptr, *p_col;        // Ps = (I - omega D^-1 A) P, SELL-32 (fine rows -> next level's columns)
  float *p_val32;
  double *p_val64;
  int32_t *r_ptr, *r_col;        // Rs = R (I - omega A D^-1) = Ps^T, 4 lanes per row
  float *r_val32;
  double *r_val64;
  double omega;                  // damped-Jacobi weight
  void *b, *x, *r, *y;           // right-hand side, pre-smoothed x, its residual, cycle output (AoS)
  HaloDev ha, hp, hr;            // gather lists of A, Ps and Rs (FP32 products)
};

// Per-instance device descriptor (lives in device memory; every pointer is a device pointer).
struct Inst {
  // sizes and parameters
  int32_t nv, nt, ne;            // vertices, triangles, edge stencils (interior + clamped)
  int32_t model;                 // shell_model
  int32_t precision;             // shell_precision
  int32_t kt;                    // contribution slots per triangle: 6 (triangle stencils) or 3 (membrane only)
  int32_t n_slices;              // SELL slices
  int32_t rows_per_thread;       // rows per thread of a reduction chunk (chunk = kBlock * rows_per_thread)
  int32_t n_chunks;
  int32_t pcg_max_it, refine_max;
  int32_t nl_max;                // chord iterations per step of the exact backward Euler (<= 1: linearised step)
  int32_t nl_newton;             // 1: the iterations use the Newton tangent (projected membrane Hessian at x_k)
  int32_t nl_static;             // 1: quasi-static solve (Eq. 64): no inertia in the residual, eps_u limiter
  double dt, pcg_rtol, refine_rtol;
  double nl_rtol;                // chord stop: ||R(v_k)|| <= nl_rtol ||R(0)||
  double nl_atol;                // or ||R(v_k)|| / dt <= nl_atol (static: ||f + f_ext|| <= nl_atol)
  double nl_eps_u;               // static: largest nodal displacement of one iteration (0: no limit)
  double mu, lam;                // membrane Lame parameters (plane stress)

  // state (FP64, SoA [3][nv])
  double *x, *v, *rest, *fext;
  double *vprev;                 // velocity before the last committed step (warm-start extrapolation)
  double *vprev2, *vprev3;       // the two velocities before that (cubic extrapolation)
  double *xk;                    // [3][nv] chord iterate x + dt v_k, where the next forces are evaluated
  double *vk;                    // [3][nv] the iterate v_k itself (quasi-static limiter)
  double *mass;                  // [nv]
  uint8_t *pinned;               // [nv]
  uint8_t *fix;                  // [nv] fixed-component bits (1 x, 2 y, 4 z) when some vertex has fixed and free
                                 // components (projected solves, Newton-capable variant only), else null

  // triangle data (membrane for every model; bending stencil for FVM / smoothed hinges)
  int32_t *t_idx;                // [6][nt] (relabelled; -1 = virtual neighbour)
  uint8_t *t_bc;                 // [3][nt]
  uint8_t *t_mode;               // [nt]
  double *t_L64;  float *t_L32;  // [18][nt] 3x6 operator, row-major index i*6+j
  double *t_W64;  float *t_W32;  // [6][nt] symmetric 3x3 (00,01,02,11,12,22), area included
  double *t_k064; float *t_k032; // [3][nt]
  double *t_n64;  float *t_n32;  // [3][nt] fixed rest normal (FIXED mode)
  double *m_D64;  float *m_D32;  // [3][nt] Dm^-1 = [[d0, d1], [0, d2]]
  double *m_G64;                 // [3][nt] rest Gram |A|^2, A.B, |B|^2 of edges A = X2-X1, B = X3-X1
  double *m_At64; float *m_At32; // [nt] area * thickness
  double *m_T;                   // [10][nt] Newton tangent data (R0, R1, kappa, Q00, Q01, Q11), see store_tangent

  // edge stencils (edge hinge models)
  int32_t *e_idx;                // [4][ne] (x1, x2, x3, x4); x4 = -1 on clamped stencils
  uint8_t *e_mode;               // [ne]
  double *e_L64;  float *e_L32;  // [4][ne]
  double *e_w64;  float *e_w32;  // [ne] k_b A_E
  double *e_k064; float *e_k032; // [ne]
  double *e_n64;  float *e_n32;  // [3][ne]

  // force contributions: slot s holds 3 components at contrib[3*s+c]; vertex i sums slots
  // vtx_slot[vtx_ptr[i] .. vtx_ptr[i+1]) in that order
  int32_t *vtx_ptr, *vtx_slot;
  void *contrib;                 // float or double [n_slots][3]
  int32_t n_slots;
  int32_t n_local;               // local matrix entries (assembly)

  // matrix (SELL-32)
  int32_t *sl_ptr;               // [n_slices+1] element offset of each slice
  int32_t *sl_col;               // [nnz_pad]
  double *val64;  float *val32;  // [nnz_pad]
  double *dinv64; float *dinv32; // [nv] inverse diagonal (Jacobi)
  float *rs32;                   // [nv] row sums of A (FP64 sum, rounded): FP32 SpMV in difference form
  int32_t *diag_pos;             // [nv]
  HaloDev h0;                    // gather lists of the matrix (FP32 products)
  int32_t *asm_ptr, *asm_src;    // assembly sources of each SELL position
  double *local;                 // [n_local] per-stencil local matrix entries

  // solver scratch
  double *b;                     // [3][nv] right-hand side
  double *sol;                   // [3][nv] FP64 solution (velocity v')
  double *r64;                   // [3][nv] FP64 residual (refinement)
  double *g64;                   // [nv][4] FP64 gathered vector
  void *r, *p, *s, *w;           // [3][nv] PCG vectors in the solve precision
  void *xs;                      // [3][nv] FP64 inner solution (the FP32 refinement round's correction)
  void *g;                       // [nv][4] gathered vector in the solve precision
  double *part;                  // [n_chunks][4] reduction partials
  double *ebuf;                  // [nt + ne][2] per-stencil energies (bending, membrane)

  InstStatus *status;            // one per instance
  int32_t *err_flags;            // precompute error flags (degenerate / singular)

  // multigrid preconditioner (amg_levels == 0: Jacobi)
  int32_t amg_levels;
  int32_t amg_coarse_n;          // rows of the coarsest level
  int32_t amg_coarse_sweeps;     // 0: dense inverse on the coarsest level, else Jacobi sweeps
  int32_t amg_dense_level;       // level whose cycle is applied as one dense operator (-1: none)
  AmgDev *amg;                   // [amg_levels]
  double *amg_cinv64;            // dense inverse of the coarsest operator [n][n]
  float *amg_cinv32;
  int32_t amg_dense_n, pad2;     // rows of that level
  double *amg_dense64;           // the cycle of levels >= amg_dense_level as a dense matrix, column-major
  float *amg_dense32;
};

// A force tile: kForceBlock consecutive stencils of one instance.
struct Tile {
  int32_t inst;
  int32_t kind;    // 0 = triangles, 1 = edge stencils
  int32_t first;
  int32_t count;
};

// Persistent-solve schedule: CTA b belongs to team cta_team[b] with rank cta_rank[b]; team t has
// team_size[t] CTAs and processes instances team_list[team_ptr[t] .. team_ptr[t+1]) in order.
// With cluster > 0 the launch uses thread-block clusters of that many CTAs; a team whose size is a multiple
// of the cluster size starts on a cluster boundary and synchronises with the hardware cluster barrier
// (one cluster), or hierarchically (cluster barrier, then a bounded global barrier between the clusters'
// leader CTAs, then the cluster barrier again). Every other multi-CTA team uses the global barrier.
struct Sched {
  int32_t *cta_team, *cta_rank;
  int32_t *team_size, *team_ptr, *team_list;
  unsigned int *bar;     // [n_teams][kBarWords] barrier words
  int32_t *abort_flag;   // set when a bounded wait gives up
  int32_t *cluster_ok;   // [n_ctas / cluster] per-cluster barrier verdict (hierarchical teams)
  int32_t n_ctas;
  int32_t cluster;       // CTAs per cluster of the launch, 0 = no clusters
  int32_t halo_cap;      // vector entries the launch's dynamic shared memory stages (set by launch_solve)
  int32_t chord_k;       // chord iteration of the step this launch performs (0: the first, or the only one)
  unsigned long long wait_ns;  // bound of a team-barrier wait (ns); past it the CTA raises the abort flag
  // instances solved by one CTA each, taken in this order by whichever CTA is free: the single-CTA teams, and
  // the CTAs of multi-CTA teams once their own list is done (queue_ctr is zeroed before every launch)
  int32_t *queue;
  unsigned int *queue_ctr;
  int32_t n_queue;
};

// ---------------------------------------------------------------- launchers (defined in .cu files)
cudaError_t launch_precompute(const Inst *d_inst, const Inst &h_inst, double E, double nu, double thickness,
                              double density, cudaStream_t st);
cudaError_t launch_assemble(const Inst *d_inst, const Inst &h_inst, cudaStream_t st);
// chord_k > 0: only instances in a chord iteration, at their iterate positions xk
cudaError_t launch_forces(const Inst *d_insts, const Tile *d_tiles, int n_tiles, int want_energy, int fp32,
                          cudaStream_t st, int chord_k = 0);
cudaError_t launch_gather_forces(const Inst *d_inst, const Inst &h_inst, double *d_out, cudaStream_t st);
cudaError_t launch_energy_reduce(const Inst *d_inst, const Inst &h_inst, double *d_out4, cudaStream_t st);
cudaError_t launch_solve(const Inst *d_insts, const Sched &sched, int grid, int prec, int occ, cudaStream_t st);
cudaError_t launch_aos_to_soa(const double *src, double *dst, int nv, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *src, double *dst, int nv, cudaStream_t st);
cudaError_t launch_mass(const Inst *d_inst, const Inst &h_inst, double rho, const double g[3], int n_loads,
                        const int32_t *d_lv, const double *d_lf, cudaStream_t st);
cudaError_t launch_gather_status(const Inst *d_insts, int n, InstStatus *d_out, const int32_t *d_abort,
                                 int32_t *d_out_abort, cudaStream_t st);
cudaError_t launch_matvec64(const Inst *d_inst, const Inst &h_inst, const double *d_in, double *d_out,
                           cudaStream_t st);
cudaError_t launch_pack_states(const Inst *d_insts, int n, const long long *d_offs, long long rows, double *d_x,
                               double *d_v, int unpack, cudaStream_t st);
int solve_blocks_per_sm(int prec, int occ);   // prec: 0 mixed, 1 FP64 only, 2 FP32-refinement only, 3 Newton
int solve_max_clusters(int prec, int cluster);   // co-resident clusters of the solve kernel, 0 if unsupported
constexpr int kCluster = 8;                      // cluster size of the batched solve launch (portable)
int static_max_ctas();
cudaError_t launch_step_static(const Inst *d_inst, const Tile *d_tiles, int n_tiles, int fp32, int newton,
                               int team_ctas, int n_steps, int chord_launches, InstStatus *h_status,
                               int32_t *h_aborted, cudaStream_t st);

}  // namespace shl
