// kernels_solve.cu -- persistent step kernel: per-stencil forces, right-hand side, preconditioned conjugate
// gradients on the constant matrix (Jacobi, or a smoothed-aggregation multigrid V-cycle with its damped-Jacobi
// sweeps folded into the transfers and one dense operator for its coarse end), state update. One launch per
// step serves every instance of a batch; each team evaluates its own FP32 instance's stencils before its solve
// (FP64 instances take their forces from the standalone force launch just before).
//
// Step (Section 5, Eq. 62-63, linearised): (M + dt^2 K) v' = M v + dt (f + f_ext); x' = x + dt v'.
// Exact backward Euler (optional, per instance): the same launch repeated as a chord iteration, each with
// the forces at the previous iterate (phase_rhs, finish_step, phase_chord).
// FP32 products stage each block's gathered vector entries in shared memory (per-block gather lists).
//
// Work split. The grid is cut into teams of CTAs; a team processes a fixed list of instances one after the
// other, all of its CTAs working on the same instance. Rows are grouped in chunks of kBlock * rpt rows
// (rpt = rows per thread, fixed per instance); chunk c is owned by team rank c mod team_size. Teams of one
// CTA synchronise with __syncthreads; larger teams with a global-memory barrier whose spin is bounded in
// time (on timeout the kernel raises an abort flag and every CTA returns). The launch is cooperative, so
// all CTAs are co-resident and the barrier cannot wait for a CTA that is not running.
//
// Reductions are deterministic and independent of the team size: each chunk reduces its rows with a fixed
// tree into a per-chunk partial; every CTA then sums all partials of the instance in a fixed lane-strided
// order and tree. An instance therefore gets bit-identical results whether it runs alone or in a batch.
//
// Solver: Chronopoulos-Gear form of preconditioned CG (one fused reduction of (r,u), (w,u), (r,r) per
// iteration; two team barriers per iteration with the Jacobi preconditioner, and the multigrid cycle adds two
// per level above its dense end and one for that end):
//   p = u + beta p; s = w + beta s; x += alpha p; r -= alpha s; u = D^-1 r; w = A u;
//   gamma' = (r,u); delta' = (w,u); beta' = gamma'/gamma; alpha' = gamma'/(delta' - beta' gamma'/alpha).
// Warm start: the velocity extrapolated from the last four (cubic). FP64 mode: one CG in FP64 from it, until
// ||r|| <= rtol ||b||.
// FP32 refinement mode: r64 = b - A v in FP64 (FP64 matrix and vector); inner CG in FP32 on A d = r64 from
// d = 0 to a relative tolerance (or to a margin below the refinement target, if that is reached first);
// v += d; repeat until ||r64|| <= refine_rtol ||b||.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "internal.h"
#include "stencil_force.cuh"

namespace shl {
namespace {

struct alignas(16) D4 {
  double x, y, z, w;
};

__device__ inline unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ inline unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline int ld_volatile_i(const int *p) { return *((volatile const int *)p); }

struct Team {
  int team, rank, size;
  unsigned int *bar;
  int *abort_flag;
  int bank;     // partials are double-buffered: reduction k writes bank k % 2
  int mode;     // 0: one CTA; 1: global barrier; 2: one whole cluster; 3: several whole clusters
  int cluster;  // CTAs per cluster
  int *cluster_ok;
  unsigned long long t0;   // start of the current instance's solve (global timer, ns)
  int cap;      // vector entries the dynamic shared memory can stage (0: no staging)
  int chord_k;  // chord iteration of the step this launch performs
  unsigned long long wait_ns;   // bound of a barrier wait
};

__device__ inline void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ inline unsigned int cluster_ctarank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ inline double *part_of(const Inst &I, const Team &tm, int ch) {
  return I.part + 4 * ((size_t)tm.bank * I.n_chunks + ch);
}

__device__ inline unsigned long long ld_acquire64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Bounded global-memory barrier among `parties` arrivals on the team's words (thread 0 of the caller only).
// The team's 64-bit arrival counter only grows: it is zeroed when the team layout is built (and after an
// abandoned launch), and every CTA of a team passes the same barriers, so an episode starts at a multiple
// of `parties` and ends when the counter reaches the next one. The last arrival's own increment releases the
// others (no reset or generation word to write after it), and no word is read before arriving.
// Returns 0 if it gave up (timeout, or abort raised elsewhere).
__device__ int global_arrive_wait(const Team &tm, unsigned int parties) {
  unsigned long long *count = reinterpret_cast<unsigned long long *>(tm.bar);
  __threadfence();   // this CTA's writes of the phase are visible before its arrival
  const unsigned long long o = atomicAdd(count, 1ull);
  const unsigned long long target = (o / parties + 1ull) * parties;
  if (o + 1ull != target) {
    const unsigned long long t0 = gtimer();
    const unsigned long long limit = tm.wait_ns;
    while (ld_acquire64(count) < target) {
      if (ld_volatile_i(tm.abort_flag)) return 0;
      if (gtimer() - t0 > limit) {
        atomicExch(tm.abort_flag, 1);
        return 0;
      }
      __nanosleep(32);
    }
  }
  __threadfence();
  return 1;
}

// Team barrier. Returns false if the barrier was abandoned (timeout or abort raised by another CTA); every
// CTA of a team, and of a cluster, gets the same verdict.
__device__ bool team_sync(const Team &tm) {
  __shared__ int s_ok;
  __syncthreads();
  if (tm.mode == 0) return true;
  if (tm.mode == 2) {            // the team is one cluster: hardware barrier, cannot time out
    cluster_barrier();
    return true;
  }
  if (tm.mode == 3) {            // several clusters: cluster barrier, leaders meet globally, cluster barrier
    cluster_barrier();
    const unsigned int crank = cluster_ctarank();
    int *flag = tm.cluster_ok + (blockIdx.x / tm.cluster);
    if (crank == 0 && threadIdx.x == 0) {
      const int ok = global_arrive_wait(tm, (unsigned int)(tm.size / tm.cluster));
      *((volatile int *)flag) = ok;
    }
    cluster_barrier();
    if (threadIdx.x == 0) s_ok = *((volatile int *)flag);
    __syncthreads();
    return s_ok != 0;
  }
  if (threadIdx.x == 0) s_ok = global_arrive_wait(tm, (unsigned int)tm.size);
  __syncthreads();
  return s_ok != 0;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-chunk partials: each chunk's three values are reduced by a fixed tree (warp shuffles, then the warps
// in order). The warp sums of up to kStage chunks are staged in shared memory and written out together, so
// a CTA that owns several chunks of a phase pays two __syncthreads per kStage chunks instead of per chunk.
constexpr int kStage = 32;

struct ChunkStage {
  int n = 0;       // staged chunks
  int first = 0;   // chunk id of the first staged one
};

__device__ inline double (*stage_buf())[kBlock / 32][3] {
  __shared__ double sm[kStage][kBlock / 32][3];
  return sm;
}

__device__ void stage_flush(ChunkStage &cs, const Inst &I, const Team &tm) {
  double(*sm)[kBlock / 32][3] = stage_buf();
  __syncthreads();
  if ((int)threadIdx.x < cs.n) {
    const int k = threadIdx.x;
    double a0 = sm[k][0][0], a1 = sm[k][0][1], a2 = sm[k][0][2];
    for (int w = 1; w < kBlock / 32; ++w) {
      a0 += sm[k][w][0];
      a1 += sm[k][w][1];
      a2 += sm[k][w][2];
    }
    double *dst = part_of(I, tm, cs.first + k * tm.size);
    dst[0] = a0;
    dst[1] = a1;
    dst[2] = a2;
  }
  __syncthreads();
  cs.n = 0;
}

template <typename A>
__device__ void stage_chunk(ChunkStage &cs, const Inst &I, const Team &tm, int ch, A v0, A v1, A v2) {
  double(*sm)[kBlock / 32][3] = stage_buf();
  if (cs.n == 0) cs.first = ch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  v2 = warp_sum(v2);
  if (lane == 0) {
    sm[cs.n][warp][0] = double(v0);
    sm[cs.n][warp][1] = double(v1);
    sm[cs.n][warp][2] = double(v2);
  }
  if (++cs.n == kStage) stage_flush(cs, I, tm);
}

// sum all chunk partials of an instance in a fixed order; result broadcast to the CTA. Flips the bank, so
// the next phase may write partials while slower CTAs of the team still read these.
__device__ void team_reduce(const Inst &I, Team &tm, double out[3]) {
  __shared__ double res[3];
  const double *part = I.part + 4 * (size_t)tm.bank * I.n_chunks;
  const int n_chunks = I.n_chunks;
  tm.bank ^= 1;
  if (threadIdx.x < 32) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int c = threadIdx.x; c < n_chunks; c += 32) {
      a0 += __ldcg(part + 4 * c);
      a1 += __ldcg(part + 4 * c + 1);
      a2 += __ldcg(part + 4 * c + 2);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (threadIdx.x == 0) {
      res[0] = a0;
      res[1] = a1;
      res[2] = a2;
    }
  }
  __syncthreads();
  out[0] = res[0];
  out[1] = res[1];
  out[2] = res[2];
}

// ------------------------------------------------------------------ precision traits
template <typename R>
struct Vec;
template <>
struct Vec<double> {
  typedef D4 G;
  __device__ static const double *val(const Inst &I) { return I.val64; }
  __device__ static const double *dinv(const Inst &I) { return I.dinv64; }
  __device__ static G *g(const Inst &I) { return reinterpret_cast<D4 *>(I.g); }
  __device__ static G mk(double x, double y, double z) { return {x, y, z, 0.0}; }
};
template <>
struct Vec<float> {
  typedef float4 G;
  __device__ static const float *val(const Inst &I) { return I.val32; }
  __device__ static const float *dinv(const Inst &I) { return I.dinv32; }
  __device__ static G *g(const Inst &I) { return reinterpret_cast<float4 *>(I.g); }
  __device__ static G mk(float x, float y, float z) { return make_float4(x, y, z, 0.0f); }
};

__device__ inline D4 ldg4(const D4 *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 a = q[0], b = q[1];
  return {a.x, a.y, b.x, b.y};
}
__device__ inline float4 ldg4(const float4 *p) { return *p; }

// y = A g for one row (SELL-32)
// g is written by other CTAs during the launch: it must not be read through the non-coherent path, so it
// carries no __restrict__ / const-restrict qualification. Both forms issue the column, value and gather
// loads of several nonzeros before consuming them (memory-level parallelism per thread). Matrix data uses
// normal caching: the same constant matrix is read by every product of every iteration, so L2 reuse of it
// matters more than protecting the gathered vector (a streaming hint halved the L2 hit rate).
//
// FP64 (refinement residual, FP64 CG): y_i = sum_j a_ij g_j.
__device__ inline void spmv_row(const Inst &I, const double *__restrict__ val, const D4 *g, int row, double &ax,
                                double &ay, double &az) {
  constexpr int U = 4;
  const int s = row >> 5, lane = row & 31;
  const int b1 = I.sl_ptr[s + 1];
  ax = ay = az = 0.0;
  for (int p = I.sl_ptr[s] + lane; p < b1; p += 32 * U) {
    int c[U];
    double a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? I.sl_col[q] : row;
      a[j] = ok ? val[q] : 0.0;
    }
    D4 v[U];
#pragma unroll
    for (int j = 0; j < U; ++j) v[j] = ldg4(g + c[j]);
#pragma unroll
    for (int j = 0; j < U; ++j) {
      ax += a[j] * v[j].x;
      ay += a[j] * v[j].y;
      az += a[j] * v[j].z;
    }
  }
}

// FP32 (inner CG): difference form y_i = rs_i g_i + sum_{j != i} a_ij (g_j - g_i), rs_i = sum_j a_ij taken
// in FP64. When dt^2 K dominates M, A's smallest eigenvalues come from the mass while its entries come from
// the stiffness; rounding the entries to FP32 in the plain form would perturb those modes by more than
// their size. In this form the rounding of a_ij only scales differences, and the constant mode sees the
// accurately rounded row sum.
__device__ inline void spmv_row(const Inst &I, const float *__restrict__ val, const float4 *g, int row, float &ax,
                                float &ay, float &az) {
  constexpr int U = 8;
  const int s = row >> 5, lane = row & 31;
  const int b1 = I.sl_ptr[s + 1];
  const float4 ui = g[row];
  const float rs = I.rs32[row];
  ax = rs * ui.x;
  ay = rs * ui.y;
  az = rs * ui.z;
  for (int p = I.sl_ptr[s] + lane; p < b1; p += 32 * U) {
    int c[U];
    float a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? I.sl_col[q] : row;
      a[j] = ok ? val[q] : 0.0f;
    }
    float4 v[U];
#pragma unroll
    for (int j = 0; j < U; ++j) v[j] = g[c[j]];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      ax += a[j] * (v[j].x - ui.x);
      ay += a[j] * (v[j].y - ui.y);
      az += a[j] * (v[j].z - ui.z);
    }
  }
}

// ------------------------------------------------------------------ staged FP32 products
// A CTA processes 256 rows at a time. With gather lists (HaloDev), it first copies the vector entries its
// rows reference into shared memory (mostly contiguous runs, one coalesced pass), then every nonzero reads
// its gathered value from there through a 16-bit local index: one global request per distinct column of the
// block instead of one per nonzero, and 2 instead of 4 bytes of column index per nonzero.
extern __shared__ float4 sh_halo[];   // dynamic shared memory: Team::cap entries

__device__ inline bool halo_on(const HaloDev &H, int cap) { return H.max > 0 && H.max <= cap; }

// Copies block blk's list entries of vec into shared memory (all threads of the CTA; barriers on both sides).
// vec is written by other CTAs of the launch, so it is read with coherent loads.
__device__ __forceinline__ void stage_block(const HaloDev &H, int blk, const float4 *vec) {
  const int mx = H.max;
  const int32_t *hl = H.col + (size_t)blk * mx;
  __syncthreads();   // earlier readers of the buffer are done
  // four entries per thread and pass: the column loads, then the gathers, are in flight together
  for (int k = threadIdx.x; k < mx; k += 4 * kBlock) {
    const bool o1 = k + kBlock < mx, o2 = k + 2 * kBlock < mx, o3 = k + 3 * kBlock < mx;
    const int c0 = __ldg(hl + k);
    const int c1 = o1 ? __ldg(hl + k + kBlock) : c0;
    const int c2 = o2 ? __ldg(hl + k + 2 * kBlock) : c0;
    const int c3 = o3 ? __ldg(hl + k + 3 * kBlock) : c0;
    const float4 t0 = vec[c0];
    const float4 t1 = vec[c1];
    const float4 t2 = vec[c2];
    const float4 t3 = vec[c3];
    sh_halo[k] = t0;
    if (o1) sh_halo[k + kBlock] = t1;
    if (o2) sh_halo[k + 2 * kBlock] = t2;
    if (o3) sh_halo[k + 3 * kBlock] = t3;
  }
  __syncthreads();
}

// One row of a staged product, all threads of the CTA (valid: this thread's row exists). The loads that do
// not depend on the staged vector are issued before the staging barrier: the row's slice bounds, its row
// sum and its first U nonzeros (column indices and values); so they overlap the list -> vector -> shared-
// memory chain, which starts at once (lists sit at a fixed stride: no lookup of the block's list). vec is
// written by other CTAs of the launch, so it is read with coherent loads. DIFF: difference form
// y_i = rs_i u_i + sum_j a_ij (u_j - u_i) of a square matrix (ui returns u_i); else plain
// y_i = sum_j m_ij v_j. The arithmetic is that of the unstaged products.
template <bool DIFF>
__device__ __forceinline__ void staged_row(const HaloDev &H, int blk, const float4 *vec, const int32_t *sp,
                                           const float *__restrict__ val, const float *rs, int row, bool valid,
                                           float &ax, float &ay, float &az, float4 &ui) {
  constexpr int U = 8;
  const int own = DIFF ? __ldg(H.own + blk) + (int)threadIdx.x : 0;
  int p = 0, b1 = 0;
  float r = 0.0f;
  if (valid) {
    const int s = row >> 5;
    p = sp[s] + (row & 31);
    b1 = sp[s + 1];
    if (DIFF) r = rs[row];
  }
  int c[U];
  float a[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = p + 32 * j;
    const bool ok = q < b1;
    c[j] = ok ? (int)H.c16[q] : own;
    a[j] = ok ? val[q] : 0.0f;
  }
  stage_block(H, blk, vec);
  ax = ay = az = 0.0f;
  if (!valid) return;
  if (DIFF) {
    ui = sh_halo[own];
    ax = r * ui.x;
    ay = r * ui.y;
    az = r * ui.z;
  }
  for (;;) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const float4 t = sh_halo[c[j]];
      if (DIFF) {
        ax += a[j] * (t.x - ui.x);
        ay += a[j] * (t.y - ui.y);
        az += a[j] * (t.z - ui.z);
      } else {
        ax += a[j] * t.x;
        ay += a[j] * t.y;
        az += a[j] * t.z;
      }
    }
    p += 32 * U;
    if (p >= b1) break;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? (int)H.c16[q] : own;
      a[j] = ok ? val[q] : 0.0f;
    }
  }
}

// FP64 plain product of the level matrix from staged FP64 entries (the refinement residual of FP32
// instances, which carry the matrix's gather lists): the buffer holds D4 entries (two float4 slots each);
// the loads that do not depend on the staged vector go first; the arithmetic is that of spmv_row (FP64).
__device__ __forceinline__ void staged_row64(const HaloDev &H, int blk, const D4 *vec, const int32_t *sp,
                                             const double *__restrict__ val, int row, bool valid, double &ax,
                                             double &ay, double &az) {
  constexpr int U = 4;
  D4 *sh = reinterpret_cast<D4 *>(sh_halo);
  int p = 0, b1 = 0;
  if (valid) {
    const int s = row >> 5;
    p = sp[s] + (row & 31);
    b1 = sp[s + 1];
  }
  int c[U];
  double a[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = p + 32 * j;
    const bool ok = q < b1;
    c[j] = ok ? (int)H.c16[q] : 0;
    a[j] = ok ? val[q] : 0.0;
  }
  const int mx = H.max;
  const int32_t *hl = H.col + (size_t)blk * mx;
  __syncthreads();   // earlier readers of the buffer are done
  for (int k = threadIdx.x; k < mx; k += 2 * kBlock) {
    const bool o1 = k + kBlock < mx;
    const int c0 = __ldg(hl + k);
    const int c1 = o1 ? __ldg(hl + k + kBlock) : c0;
    const D4 t0 = ldg4(vec + c0);
    const D4 t1 = ldg4(vec + c1);
    sh[k] = t0;
    if (o1) sh[k + kBlock] = t1;
  }
  __syncthreads();
  ax = ay = az = 0.0;
  if (!valid) return;
  for (;;) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const D4 t = sh[c[j]];
      ax += a[j] * t.x;
      ay += a[j] * t.y;
      az += a[j] * t.z;
    }
    p += 32 * U;
    if (p >= b1) break;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? (int)H.c16[q] : 0;
      a[j] = ok ? val[q] : 0.0;
    }
  }
}

// ------------------------------------------------------------------ Newton tangent
// Row `row` of dt^2 (H - K_iso) u, summed over the triangles incident to the row's vertex: H_t is the membrane
// Hessian of triangle t at the positions of its last force evaluation, projected to positive semi-definite
// (tangent data m_T, see store_tangent), K_iso,t the constant isotropic block 2 (mu + lam) A t grad(phi_a) .
// grad(phi_b) (x) I_3 the step matrix holds. Added to the step matrix's product, it gives the Newton matrix
// M + dt^2 (K_b + sum_t H_t). With U = sum_b u_b g_b^T (3x2, g_b the hat gradients), A = R^T U, b = U^T n:
//   y_a = A t [R Sigma + n (Q b)^T - 2 (mu + lam) U] g_a,
//   Sigma = 2 mu sym(A) + lam tr(A) I + kappa (A_10 - A_01) [[0, -1], [1, 0]].
// Pinned vertices have identity rows and columns in the step matrix: their rows get no correction and their
// entries of u count as zero. u: gathered vector (AoS) of the product.
template <typename R, typename G>
__device__ __noinline__ void tangent_corr(const Inst &I, const G *u, int row, R &cx, R &cy, R &cz) {
  cx = cy = cz = R(0);
  if (I.pinned[row]) return;
  const int nt = I.nt, kt = I.kt;
  const R mu = R(I.mu), lam = R(I.lam), w2 = R(2) * (mu + lam);
  const double *T = I.m_T;
  v3<R> y = zero3<R>();
  for (int q = I.vtx_ptr[row]; q < I.vtx_ptr[row + 1]; ++q) {
    const int s = I.vtx_slot[q];
    if (s >= nt * kt) continue;            // an edge stencil's slot
    const int t = s / kt, j = s - t * kt;
    if (j >= 3) continue;                  // a bending neighbour's slot
    v3<R> uu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int v = I.t_idx[a * nt + t];
      const G g = ldg4(u + v);
      uu[a] = I.pinned[v] ? zero3<R>() : v3<R>{R(g.x), R(g.y), R(g.z)};
    }
    const R p = R(I.m_D64[t]), qd = R(I.m_D64[nt + t]), r = R(I.m_D64[2 * nt + t]), At = R(I.m_At64[t]);
    const v3<R> du = uu[1] - uu[0], dv = uu[2] - uu[0];
    const v3<R> U0 = p * du, U1 = qd * du + r * dv;
    const v3<R> R0 = {R(T[t]), R(T[nt + t]), R(T[2 * nt + t])};
    const v3<R> R1 = {R(T[3 * nt + t]), R(T[4 * nt + t]), R(T[5 * nt + t])};
    const R kap = R(T[6 * nt + t]), Q00 = R(T[7 * nt + t]), Q01 = R(T[8 * nt + t]), Q11 = R(T[9 * nt + t]);
    const v3<R> n = cross(R0, R1);
    const R A00 = dot(R0, U0), A01 = dot(R0, U1), A10 = dot(R1, U0), A11 = dot(R1, U1);
    const R b0 = dot(n, U0), b1 = dot(n, U1);
    const R trA = A00 + A11, wv = A10 - A01, sy = mu * (A01 + A10);
    const R S00 = R(2) * mu * A00 + lam * trA, S11 = R(2) * mu * A11 + lam * trA;
    const R S01 = sy - kap * wv, S10 = sy + kap * wv;
    const R Qb0 = Q00 * b0 + Q01 * b1, Qb1 = Q01 * b0 + Q11 * b1;
    const v3<R> P0 = S00 * R0 + S10 * R1 + Qb0 * n - w2 * U0;
    const v3<R> P1 = S01 * R0 + S11 * R1 + Qb1 * n - w2 * U1;
    const v3<R> H0 = At * (p * P0 + qd * P1);
    const v3<R> H1 = (At * r) * P1;
    if (j == 0)
      y = y - (H0 + H1);
    else if (j == 1)
      y = y + H0;
    else
      y = y + H1;
  }
  const R dt2 = R(I.dt * I.dt);
  cx = dt2 * y.x;
  cy = dt2 * y.y;
  cz = dt2 * y.z;
}

// ------------------------------------------------------------------ phases
// Per-stencil forces of the instance at the positions of this launch (x, or the chord iterate xk of exact
// backward Euler), in the instance's precision, written to its contribution slots (one writer per slot). The
// team's CTAs take 256-stencil chunks of the combined list (triangles, then edge stencils) round robin; the
// right-hand side reads the slots after the next team barrier.
template <typename R, bool NT>
__device__ void phase_forces(const Inst &I, const Team &tm) {
  const Data<R> D(I, tm.chord_k > 0 ? I.xk : I.x);
  const int ns = I.nt + I.ne;
  for (int c = tm.rank; c * kBlock < ns; c += tm.size) {
    const int s = c * kBlock + (int)threadIdx.x;
    if (s < I.nt)
      tri_stencil<R, NT>(I, D, s, false);
    else if (s < ns)
      edge_stencil<R>(I, D, s - I.nt, false);
  }
}

#define ROWS_BEGIN(I, tm)                                                                 \
  for (int ch = (tm).rank; ch < (I).n_chunks; ch += (tm).size) {                        \
    for (int rr = 0; rr < (I).rows_per_thread; ++rr) {                                  \
      const int row = (ch * (I).rows_per_thread + rr) * kBlock + (int)threadIdx.x;      \
      if (row < (I).nv) {
#define ROWS_END \
  }              \
  }              \
  }

// b = M v + dt (f + f_ext) (zero at pinned vertices and fixed components); warm start sol = 4 (v + v_prev2) - 6 v_prev - v_prev3;
// g64 = sol; partial ||b||^2
// Chord iteration k > 0 of the exact backward-Euler step (forces at x + dt v_k, v_k in sol and g64):
// b = M v + dt (f + f_ext) + (A - M) v_k, warm start v_k kept, so that the first residual b - A v_k is
// -R(v_k), the backward-Euler residual, and the solve gives v_{k+1} = v_k - A^-1 R(v_k).
template <typename RC, bool NT>
__device__ void phase_rhs(const Inst &I, const Team &tm) {
  const int nv = I.nv;
  const bool chord = tm.chord_k > 0;
  const RC *con = reinterpret_cast<const RC *>(I.contrib);
  ChunkStage cs;
  for (int ch = tm.rank; ch < I.n_chunks; ch += tm.size) {
    double bb = 0.0;
    for (int rr = 0; rr < I.rows_per_thread; ++rr) {
      const int row = (ch * I.rows_per_thread + rr) * kBlock + (int)threadIdx.x;
      if (row >= nv) continue;
      double f[3] = {0.0, 0.0, 0.0};
      // the vertex's slots in their fixed order, four per round: the slot indices, then their contributions
      // (written by the team's force phase: coherent loads), are in flight together
      const int q1 = I.vtx_ptr[row + 1];
      for (int q = I.vtx_ptr[row]; q < q1; q += 4) {
        size_t sl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) sl[j] = q + j < q1 ? (size_t)I.vtx_slot[q + j] : 0;
        RC cv[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int c = 0; c < 3; ++c) cv[j][c] = q + j < q1 ? __ldcg(con + 3 * sl[j] + c) : RC(0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (q + j < q1)
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] += double(cv[j][c]);
      }
      const bool pin = I.pinned[row] != 0;
      unsigned fx = 0u;   // fixed components of a vertex with fixed and free ones
      if constexpr (NT) fx = I.fix ? (unsigned)I.fix[row] : 0u;
      const double m = I.mass[row];
      double av[3] = {0.0, 0.0, 0.0};
      if (chord) {
        const D4 *vk = reinterpret_cast<const D4 *>(I.g64);
        spmv_row(I, I.val64, vk, row, av[0], av[1], av[2]);
        if constexpr (NT) {
          if (I.nl_newton) {
            double cx, cy, cz;
            tangent_corr<double, D4>(I, vk, row, cx, cy, cz);
            av[0] += cx;
            av[1] += cy;
            av[2] += cz;
          }
        }
      }
      double sv[3];
      for (int c = 0; c < 3; ++c) {
        const double v = I.v[c * nv + row];
        // quasi-static: b = dt (f + f_ext) + J v_k, so that b - J v_k = dt (f + f_ext), the residual of Eq. 64
        double b = (I.nl_static ? 0.0 : m * v) + I.dt * (f[c] + I.fext[c * nv + row]);
        if (chord) b += av[c] - (I.nl_static ? 0.0 : m * I.sol[c * nv + row]);
        const bool fixed = pin || ((fx >> c) & 1u);
        if (fixed) b = 0.0;
        I.b[c * nv + row] = b;
        bb += b * b;
        // initial guess: cubic extrapolation of the last four velocities, 4 (v + v_prev2) - 6 v_prev - v_prev3
        // (v_prev, v_prev2, v_prev3: the velocities before the last three committed steps; setting a state
        // leaves them, as they only shape the initial guess); zero for the quasi-static solve
        if (!chord) {
          const int k = c * nv + row;
          sv[c] = (fixed || I.nl_static) ? 0.0 : 4.0 * (v + I.vprev2[k]) - 6.0 * I.vprev[k] - I.vprev3[k];
          I.sol[c * nv + row] = sv[c];
        }
      }
      if (!chord) reinterpret_cast<D4 *>(I.g64)[row] = {sv[0], sv[1], sv[2], 0.0};
    }
    stage_chunk<double>(cs, I, tm, ch, bb, 0.0, 0.0);
  }
  if (cs.n) stage_flush(cs, I, tm);
}

// FP64 residual r64 = b - A64 sol; returns partial ||r64||^2. If R is float also prepares the inner CG:
// r32 = r64, xs = 0 (FP64), g32 = D32^-1 r32. If R is double: r = r64 (in place), sol unchanged, g = D^-1 r.
// Multigrid: also the first V-cycle's level-0 pre-smoothing from zero, b0 = r, x0 = omega D^-1 r (row-local).
template <typename R, bool NT>
__device__ void phase_resid(const Inst &I, const Team &tm) {
  const int nv = I.nv;
  const bool amg = I.amg_levels > 0;
  typename Vec<R>::G *b0 = amg ? reinterpret_cast<typename Vec<R>::G *>(I.amg[0].b) : nullptr;
  typename Vec<R>::G *x0 = amg ? reinterpret_cast<typename Vec<R>::G *>(I.amg[0].x) : nullptr;
  const R om0 = amg ? R(I.amg[0].omega) : R(0);
  const D4 *g64 = reinterpret_cast<const D4 *>(I.g64);
  R *r = reinterpret_cast<R *>(I.r);
  double *xs = reinterpret_cast<double *>(I.xs);
  typename Vec<R>::G *g = Vec<R>::g(I);
  const R *dinv = Vec<R>::dinv(I);
  const bool st = I.h0.max > 0 && 2 * I.h0.max <= tm.cap;   // FP64 entries take two buffer slots
  ChunkStage cs;
  for (int ch = tm.rank; ch < I.n_chunks; ch += tm.size) {
    double rr2 = 0.0;
    for (int rr = 0; rr < I.rows_per_thread; ++rr) {
      const int blk = ch * I.rows_per_thread + rr;
      if (blk * kBlock >= nv) break;
      const int row = blk * kBlock + (int)threadIdx.x;
      double ax, ay, az;
      if (st) {
        staged_row64(I.h0, blk, g64, I.sl_ptr, I.val64, row, row < nv, ax, ay, az);
        if (row >= nv) continue;
      } else {
        if (row >= nv) continue;
        spmv_row(I, I.val64, g64, row, ax, ay, az);
      }
      if constexpr (NT) {
        if (I.nl_newton) {
          double cx, cy, cz;
          tangent_corr<double, D4>(I, g64, row, cx, cy, cz);
          ax += cx;
          ay += cy;
          az += cz;
        }
      }
      double r0 = I.b[row] - ax, r1 = I.b[nv + row] - ay, r2 = I.b[2 * nv + row] - az;
      if constexpr (NT) {
        if (I.fix) {   // projected residual: zero at the fixed components
          const unsigned fx = I.fix[row];
          if (fx & 1u) r0 = 0.0;
          if (fx & 2u) r1 = 0.0;
          if (fx & 4u) r2 = 0.0;
        }
      }
      I.r64[row] = r0;
      I.r64[nv + row] = r1;
      I.r64[2 * nv + row] = r2;
      rr2 += r0 * r0 + r1 * r1 + r2 * r2;
      const R q0 = R(r0), q1 = R(r1), q2 = R(r2);
      r[row] = q0;
      r[nv + row] = q1;
      r[2 * nv + row] = q2;
      if (sizeof(R) == 4) {
        xs[row] = 0.0;
        xs[nv + row] = 0.0;
        xs[2 * nv + row] = 0.0;
      }
      const R di = dinv[row];
      g[row] = Vec<R>::mk(di * q0, di * q1, di * q2);
      if (amg) {
        b0[row] = Vec<R>::mk(q0, q1, q2);
        const R d = om0 * di;
        x0[row] = Vec<R>::mk(d * q0, d * q1, d * q2);
      }
    }
    stage_chunk<double>(cs, I, tm, ch, rr2, 0.0, 0.0);
  }
  if (cs.n) stage_flush(cs, I, tm);
}

// w = A u (u = g); partials (r,u), (w,u), (r,r)
template <typename R, bool NT>
__device__ void phase_spmv(const Inst &I, const Team &tm) {
  const int nv = I.nv;
  const R *val = Vec<R>::val(I);
  const typename Vec<R>::G *g = Vec<R>::g(I);
  const R *r = reinterpret_cast<const R *>(I.r);
  R *w = reinterpret_cast<R *>(I.w);
  bool st = false;
  if constexpr (sizeof(R) == 4) st = halo_on(I.h0, tm.cap);
  ChunkStage cs;
  for (int ch = tm.rank; ch < I.n_chunks; ch += tm.size) {
    R gu = R(0), wu = R(0), rr2 = R(0);
    for (int rr = 0; rr < I.rows_per_thread; ++rr) {
      const int blk = ch * I.rows_per_thread + rr;
      if (blk * kBlock >= nv) break;
      R ax, ay, az;
      typename Vec<R>::G u;
      const int row = blk * kBlock + (int)threadIdx.x;
      if constexpr (sizeof(R) == 4) {
        if (st) {
          staged_row<true>(I.h0, blk, g, I.sl_ptr, val, I.rs32, row, row < nv, ax, ay, az, u);
          if (row >= nv) continue;
        } else {
          if (row >= nv) continue;
          spmv_row(I, val, g, row, ax, ay, az);
          u = ldg4(g + row);
        }
      } else {
        if (row >= nv) continue;
        spmv_row(I, val, g, row, ax, ay, az);
        u = ldg4(g + row);
      }
      if constexpr (NT) {
        if (I.nl_newton) {
          R cx, cy, cz;
          tangent_corr<R, typename Vec<R>::G>(I, g, row, cx, cy, cz);
          ax += cx;
          ay += cy;
          az += cz;
        }
        if (I.fix) {   // projected product P A u (u is zero at the fixed components)
          const unsigned fx = I.fix[row];
          if (fx & 1u) ax = R(0);
          if (fx & 2u) ay = R(0);
          if (fx & 4u) az = R(0);
        }
      }
      w[row] = ax;
      w[nv + row] = ay;
      w[2 * nv + row] = az;
      const R r0 = r[row], r1 = r[nv + row], r2 = r[2 * nv + row];
      gu += r0 * R(u.x) + r1 * R(u.y) + r2 * R(u.z);
      wu += ax * R(u.x) + ay * R(u.y) + az * R(u.z);
      rr2 += r0 * r0 + r1 * r1 + r2 * r2;
    }
    stage_chunk<R>(cs, I, tm, ch, gu, wu, rr2);
  }
  if (cs.n) stage_flush(cs, I, tm);
}

// p = u + beta p; s = w + beta s; x += alpha p; r -= alpha s; then (Jacobi) u = D^-1 r -> g. With the
// multigrid preconditioner u is read from g and the new u = B r is computed by the V-cycle afterwards.
// The solution x is accumulated in FP64 in both precisions (alpha_x: alpha in FP64): the recurrences never
// read it, and in FP32 its rounding alone would leave the refinement's true residual above 1e-8 of ||b||.
// In FP32 the recurrence r -= alpha s takes alpha rounded to FP32 while x takes the FP64 alpha, so x and the
// recursive residual drift apart by about 2^-24 of each step; the FP64 residual of the next refinement round
// is formed from x itself, so the drift is measured there and corrected like any other inner error.
template <typename R>
__device__ void phase_update(const Inst &I, const Team &tm, R alpha, R beta, bool first, double *x,
                             double alpha_x) {
  const int nv = I.nv;
  const bool amg = I.amg_levels > 0;
  const R *dinv = Vec<R>::dinv(I);
  typename Vec<R>::G *g = Vec<R>::g(I);
  R *r = reinterpret_cast<R *>(I.r);
  R *p = reinterpret_cast<R *>(I.p);
  R *s = reinterpret_cast<R *>(I.s);
  const R *w = reinterpret_cast<const R *>(I.w);
  // multigrid: the level-0 pre-smoothing from zero (b0 = r, x0 = omega D^-1 r) of the next V-cycle is
  // row-local, so it is done here from the new r
  typename Vec<R>::G *b0 = amg ? reinterpret_cast<typename Vec<R>::G *>(I.amg[0].b) : nullptr;
  typename Vec<R>::G *x0 = amg ? reinterpret_cast<typename Vec<R>::G *>(I.amg[0].x) : nullptr;
  const R om0 = amg ? R(I.amg[0].omega) : R(0);
  ROWS_BEGIN(I, tm)
  const R di = dinv[row];
  R uo[3];
  if (amg) {
    const typename Vec<R>::G gu = ldg4(g + row);
    uo[0] = R(gu.x);
    uo[1] = R(gu.y);
    uo[2] = R(gu.z);
  }
  R rv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int k = c * nv + row;
    const R rc = r[k];
    const R u = amg ? uo[c] : di * rc;
    const R pc = first ? u : u + beta * p[k];
    const R sc = first ? w[k] : w[k] + beta * s[k];
    p[k] = pc;
    s[k] = sc;
    x[k] += alpha_x * double(pc);
    const R rn = rc - alpha * sc;
    r[k] = rn;
    rv[c] = rn;
  }
  if (!amg) {
    g[row] = Vec<R>::mk(di * rv[0], di * rv[1], di * rv[2]);
  } else {
    b0[row] = Vec<R>::mk(rv[0], rv[1], rv[2]);
    const R d = om0 * di;
    x0[row] = Vec<R>::mk(d * rv[0], d * rv[1], d * rv[2]);
  }
  ROWS_END
}

// ------------------------------------------------------------------ multigrid V-cycle (preconditioner)
// SpMV helpers on one level's arrays (SELL-32: the folded prolongation Ps, and the level-0 operator).
template <typename R>
struct LevelVal;
template <>
struct LevelVal<float> {
  __device__ static const float *a(const AmgDev &L) { return L.a_val32; }
  __device__ static const float *p(const AmgDev &L) { return L.p_val32; }
  __device__ static const float *r(const AmgDev &L) { return L.r_val32; }
  __device__ static const float *dinv(const AmgDev &L) { return L.dinv32; }
  __device__ static const float *cinv(const Inst &I) { return I.amg_cinv32; }
  __device__ static const float *dense(const Inst &I) { return I.amg_dense32; }
};
template <>
struct LevelVal<double> {
  __device__ static const double *a(const AmgDev &L) { return L.a_val64; }
  __device__ static const double *p(const AmgDev &L) { return L.p_val64; }
  __device__ static const double *r(const AmgDev &L) { return L.r_val64; }
  __device__ static const double *dinv(const AmgDev &L) { return L.dinv64; }
  __device__ static const double *cinv(const Inst &I) { return I.amg_cinv64; }
  __device__ static const double *dense(const Inst &I) { return I.amg_dense64; }
};

// plain y_i = sum_j m_ij v_j over a SELL-32 matrix (the folded prolongation Ps; the level-0 operator in FP64)
template <typename R, typename G>
__device__ inline void sell_plain(const int32_t *sp, const int32_t *sc, const R *sv, const G *v, int row, R &ax,
                                  R &ay, R &az) {
  constexpr int U = 4;
  const int s = row >> 5, lane = row & 31;
  const int b1 = sp[s + 1];
  ax = ay = az = R(0);
  for (int p = sp[s] + lane; p < b1; p += 32 * U) {
    int c[U];
    R a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? sc[q] : 0;
      a[j] = ok ? sv[q] : R(0);
    }
    G t[U];
#pragma unroll
    for (int j = 0; j < U; ++j) t[j] = ldg4(v + c[j]);
#pragma unroll
    for (int j = 0; j < U; ++j) {
      ax += a[j] * R(t[j].x);
      ay += a[j] * R(t[j].y);
      az += a[j] * R(t[j].z);
    }
  }
}

// level operator: FP32 in difference form (row sums), FP64 plain
__device__ inline void level_a(const AmgDev &L, const float4 *v, int row, float &ax, float &ay, float &az) {
  constexpr int U = 8;
  const int s = row >> 5, lane = row & 31;
  const int b1 = L.a_ptr[s + 1];
  const float4 ui = v[row];
  const float rs = L.rs32[row];
  ax = rs * ui.x;
  ay = rs * ui.y;
  az = rs * ui.z;
  for (int p = L.a_ptr[s] + lane; p < b1; p += 32 * U) {
    int c[U];
    float a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int q = p + 32 * j;
      const bool ok = q < b1;
      c[j] = ok ? L.a_col[q] : row;
      a[j] = ok ? L.a_val32[q] : 0.0f;
    }
    float4 t[U];
#pragma unroll
    for (int j = 0; j < U; ++j) t[j] = v[c[j]];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      ax += a[j] * (t[j].x - ui.x);
      ay += a[j] * (t[j].y - ui.y);
      az += a[j] * (t[j].z - ui.z);
    }
  }
}
__device__ inline void level_a(const AmgDev &L, const D4 *v, int row, double &ax, double &ay, double &az) {
  sell_plain<double, D4>(L.a_ptr, L.a_col, L.a_val64, v, row, ax, ay, az);
}

#define LEVEL_ROWS_BEGIN(n, tm)                                              \
  for (int ch = (tm).rank; ch * kBlock < (n); ch += (tm).size) {            \
    const int row = ch * kBlock + (int)threadIdx.x;                         \
    if (row < (n)) {
#define LEVEL_ROWS_END \
  }                    \
  }
// Row phases of one level, each instantiated with and without shared-memory staging (ST; FP32 only), so
// that a launch's loop carries only the live values of the path it takes.

// ---- one V(1,1) cycle with the damped-Jacobi sweeps folded into the transfers. A level's down step reads
// only its right-hand side b (and x = omega D^-1 b, the row-local pre-smoothing from zero, written with b):
//   r  = b - A x                            residual of the pre-smoothing, kept for the up step
//   bc = Rs b = R r,  Rs = R (I - omega A D^-1)
//   xc = omega_c Dc^-1 bc                   pre-smoothing of the next level (when it is smoothed)
// and its up step reads only x, r and the coarse solution yc:
//   y  = x + omega D^-1 r + Ps yc,  Ps = (I - omega D^-1 A) P = Rs^T
// which is the post-smoothing sweep z + omega D^-1 (b - A z) of the corrected z = x + P yc, expanded. So a
// level costs two team phases instead of four (residual, restriction, correction, post-smoothing).

// residual of one 256-row block of level 0: r = b - A x
template <typename R, bool ST>
__device__ __forceinline__ void resid_blk(const AmgDev &A, int blk) {
  typedef typename Vec<R>::G G;
  const G *b = reinterpret_cast<const G *>(A.b);
  const G *x = reinterpret_cast<const G *>(A.x);
  G *rr = reinterpret_cast<G *>(A.r);
  const int row = blk * kBlock + (int)threadIdx.x;
  R ax, ay, az;
  if constexpr (ST) {
    float4 ui;
    staged_row<true>(A.ha, blk, x, A.a_ptr, A.a_val32, A.rs32, row, row < A.n, ax, ay, az, ui);
    if (row >= A.n) return;
  } else {
    if (row >= A.n) return;
    level_a(A, x, row, ax, ay, az);
  }
  const G bi = ldg4(b + row);
  rr[row] = Vec<R>::mk(R(bi.x) - ax, R(bi.y) - ay, R(bi.z) - az);
}

// restriction of one 64-row block of the next level with its pre-smoothing from zero fused: bc = Rs b;
// xc = omega_c Dc^-1 bc. Rs has 4 lanes per row (its rows are long): lane k % 4 of a row sums the entries
// k, k + 4, ... in increasing order, and the four partial sums are added in a fixed shuffle tree; staged
// (FP32) and unstaged products run the same arithmetic. The loads that do not depend on the staged vector
// (slice bounds, first nonzeros) are issued before the staging barrier.
template <typename R, bool ST>
__device__ __forceinline__ void restrict_blk(const AmgDev &A, const AmgDev &C, bool pre, int blk) {
  typedef typename Vec<R>::G G;
  constexpr int U = 8;
  constexpr int kRows = kBlock / 4;   // coarse rows per CTA pass
  const G *bf = reinterpret_cast<const G *>(A.b);
  G *bc = reinterpret_cast<G *>(C.b);
  G *xc = reinterpret_cast<G *>(C.x);
  const R *dinvc = LevelVal<R>::dinv(C);
  const R *val = LevelVal<R>::r(A);
  const R omc = R(C.omega);
  const int n = A.n_next;
  const int lane = threadIdx.x & 31;
  const int row = blk * kRows + (int)(threadIdx.x >> 2);
  const bool valid = row < n;
  int p = 0, b1 = 0;
  if (valid) {
    const int s = row >> 3;
    p = A.r_ptr[s] + lane;
    b1 = A.r_ptr[s + 1];
  }
  int c[U];
  R a[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = p + 32 * j;
    const bool ok = q < b1;
    c[j] = ok ? (ST ? (int)A.hr.c16[q] : A.r_col[q]) : 0;
    a[j] = ok ? val[q] : R(0);
  }
  if constexpr (ST) stage_block(A.hr, blk, reinterpret_cast<const float4 *>(bf));
  R ax = R(0), ay = R(0), az = R(0);
  if (valid) {
    for (;;) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        G t;
        if constexpr (ST)
          t = sh_halo[c[j]];
        else
          t = ldg4(bf + c[j]);
        ax += a[j] * R(t.x);
        ay += a[j] * R(t.y);
        az += a[j] * R(t.z);
      }
      p += 32 * U;
      if (p >= b1) break;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int q = p + 32 * j;
        const bool ok = q < b1;
        c[j] = ok ? (ST ? (int)A.hr.c16[q] : A.r_col[q]) : 0;
        a[j] = ok ? val[q] : R(0);
      }
    }
  }
  ax += __shfl_xor_sync(0xffffffffu, ax, 1);
  ay += __shfl_xor_sync(0xffffffffu, ay, 1);
  az += __shfl_xor_sync(0xffffffffu, az, 1);
  ax += __shfl_xor_sync(0xffffffffu, ax, 2);
  ay += __shfl_xor_sync(0xffffffffu, ay, 2);
  az += __shfl_xor_sync(0xffffffffu, az, 2);
  if (valid && (threadIdx.x & 3) == 0) {
    bc[row] = Vec<R>::mk(ax, ay, az);
    if (pre) {
      const R d = omc * dinvc[row];
      xc[row] = Vec<R>::mk(d * ax, d * ay, d * az);
    }
  }
}

// up step of a level: y = x + omega D^-1 r + Ps yc (256-row blocks, Ps in SELL-32). MK (level 0 of an instance
// with per-component constraints): y is zeroed at the components fix marks, so the preconditioned vector stays
// on the free components.
template <typename R, bool ST, bool MK = false>
__device__ void lv_up(const AmgDev &A, const AmgDev &C, typename Vec<R>::G *y, const Team &tm,
                      const uint8_t *fix = nullptr) {
  typedef typename Vec<R>::G G;
  const G *x = reinterpret_cast<const G *>(A.x);
  const G *rr = reinterpret_cast<const G *>(A.r);
  const G *yc = reinterpret_cast<const G *>(C.y);
  const R *dinv = LevelVal<R>::dinv(A);
  const R om = R(A.omega);
  for (int ch = tm.rank; ch * kBlock < A.n; ch += tm.size) {
    const int row = ch * kBlock + (int)threadIdx.x;
    R ax, ay, az;
    if constexpr (ST) {
      float4 unused;
      staged_row<false>(A.hp, ch, yc, A.p_ptr, A.p_val32, nullptr, row, row < A.n, ax, ay, az, unused);
      if (row >= A.n) continue;
    } else {
      if (row >= A.n) continue;
      sell_plain<R, G>(A.p_ptr, A.p_col, LevelVal<R>::p(A), yc, row, ax, ay, az);
    }
    const G xi = ldg4(x + row);
    const G ri = ldg4(rr + row);
    const R d = om * dinv[row];
    R yx = R(xi.x) + d * R(ri.x) + ax, yy = R(xi.y) + d * R(ri.y) + ay, yz = R(xi.z) + d * R(ri.z) + az;
    if constexpr (MK) {
      if (fix) {
        const unsigned fx = fix[row];
        if (fx & 1u) yx = R(0);
        if (fx & 2u) yy = R(0);
        if (fx & 4u) yz = R(0);
      }
    }
    y[row] = Vec<R>::mk(yx, yy, yz);
  }
}

// ---- coarse levels (l >= 1): A stored with 4 lanes per row (8-row slices, like R), 64-row CTA passes.
// One row of A x for the pass over block blk: lane k % 4 sums the entries k, k + 4, ... in increasing order,
// the four partial sums are added in a fixed shuffle tree; FP32 in difference form
// (A x)_i = rs_i x_i + sum_j a_ij (x_j - x_i), FP64 plain. Staged (ST, FP32) and unstaged products, and
// any team size, run the same arithmetic. All 4 lanes of a row return the row's value; ui = x_i.
template <typename R, bool ST>
__device__ __forceinline__ void coarse_row(const AmgDev &A, const typename Vec<R>::G *x, int blk, int row,
                                           bool valid, R &ax, R &ay, R &az, typename Vec<R>::G &ui) {
  typedef typename Vec<R>::G G;
  constexpr int U = 8;
  constexpr bool DIFF = sizeof(R) == 4;
  const R *val = LevelVal<R>::a(A);
  const int lane = threadIdx.x & 31;
  const int own = ST ? __ldg(A.ha.own + blk) + (int)(threadIdx.x >> 2) : row;
  int p = 0, b1 = 0;
  R r = R(0);
  if (valid) {
    const int s = row >> 3;
    p = A.a_ptr[s] + lane;
    b1 = A.a_ptr[s + 1];
    if constexpr (DIFF) r = A.rs32[row];
  }
  int c[U];
  R a[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = p + 32 * j;
    const bool ok = q < b1;
    c[j] = ok ? (ST ? (int)A.ha.c16[q] : A.a_col[q]) : own;
    a[j] = ok ? val[q] : R(0);
  }
  if constexpr (ST) stage_block(A.ha, blk, reinterpret_cast<const float4 *>(x));
  R px = R(0), py = R(0), pz = R(0);
  ui = G{};
  if (valid) {
    if constexpr (ST)
      ui = sh_halo[own];
    else
      ui = ldg4(x + row);
    for (;;) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        G t;
        if constexpr (ST)
          t = sh_halo[c[j]];
        else
          t = ldg4(x + c[j]);
        if constexpr (DIFF) {
          px += a[j] * (R(t.x) - R(ui.x));
          py += a[j] * (R(t.y) - R(ui.y));
          pz += a[j] * (R(t.z) - R(ui.z));
        } else {
          px += a[j] * R(t.x);
          py += a[j] * R(t.y);
          pz += a[j] * R(t.z);
        }
      }
      p += 32 * U;
      if (p >= b1) break;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int q = p + 32 * j;
        const bool ok = q < b1;
        c[j] = ok ? (ST ? (int)A.ha.c16[q] : A.a_col[q]) : own;
        a[j] = ok ? val[q] : R(0);
      }
    }
  }
  px += __shfl_xor_sync(0xffffffffu, px, 1);
  py += __shfl_xor_sync(0xffffffffu, py, 1);
  pz += __shfl_xor_sync(0xffffffffu, pz, 1);
  px += __shfl_xor_sync(0xffffffffu, px, 2);
  py += __shfl_xor_sync(0xffffffffu, py, 2);
  pz += __shfl_xor_sync(0xffffffffu, pz, 2);
  if constexpr (DIFF) {
    ax = r * R(ui.x) + px;
    ay = r * R(ui.y) + py;
    az = r * R(ui.z) + pz;
  } else {
    ax = px;
    ay = py;
    az = pz;
  }
}

// residual of one 64-row block of a coarse level: r = b - A x
template <typename R, bool ST>
__device__ __forceinline__ void resid4_blk(const AmgDev &A, int blk) {
  typedef typename Vec<R>::G G;
  const G *b = reinterpret_cast<const G *>(A.b);
  const G *x = reinterpret_cast<const G *>(A.x);
  G *rr = reinterpret_cast<G *>(A.r);
  const int row = blk * (kBlock / 4) + (int)(threadIdx.x >> 2);
  const bool valid = row < A.n;
  R ax, ay, az;
  G ui;
  coarse_row<R, ST>(A, x, blk, row, valid, ax, ay, az, ui);
  if (valid && (threadIdx.x & 3) == 0) {
    const G bi = ldg4(b + row);
    rr[row] = Vec<R>::mk(R(bi.x) - ax, R(bi.y) - ay, R(bi.z) - az);
  }
}

// damped-Jacobi sweep of a coarse level: y = x + omega D^-1 (b - A x), x the previous sweep (the coarsest
// level's sweeps when it is too large for a dense inverse)
template <typename R, bool ST>
__device__ void lv_smooth4(const AmgDev &A, const typename Vec<R>::G *x, typename Vec<R>::G *y, const Team &tm) {
  typedef typename Vec<R>::G G;
  const G *b = reinterpret_cast<const G *>(A.b);
  const R *dinv = LevelVal<R>::dinv(A);
  const R om = R(A.omega);
  for (int ch = tm.rank; ch * (kBlock / 4) < A.n; ch += tm.size) {
    const int row = ch * (kBlock / 4) + (int)(threadIdx.x >> 2);
    const bool valid = row < A.n;
    R ax, ay, az;
    G xi;
    coarse_row<R, ST>(A, x, ch, row, valid, ax, ay, az, xi);
    if (valid && (threadIdx.x & 3) == 0) {
      const G bi = ldg4(b + row);
      const R d = om * dinv[row];
      y[row] = Vec<R>::mk(R(xi.x) + d * (R(bi.x) - ax), R(xi.y) + d * (R(bi.y) - ay), R(xi.z) + d * (R(bi.z) - az));
    }
  }
}

// staging applies to FP32 products whose lists fit the launch's buffer
template <typename R>
__device__ inline bool staged(const HaloDev &H, int cap) {
  return sizeof(R) == 4 && halo_on(H, cap);
}

// Down step of level l in one team phase: the residual blocks of level l and the restriction blocks of level
// l + 1 are independent (both read only b and x), so the team's CTAs take them from one list of units.
template <typename R>
__device__ bool down_step(const Inst &I, int l, const Team &tm) {
  const AmgDev &A = I.amg[l];
  const AmgDev &C = I.amg[l + 1];
  // levels at and below the dense level, and the coarsest, are solved, not smoothed
  const int top = I.amg_dense_level > 0 ? I.amg_dense_level : I.amg_levels - 1;
  const bool pre = l + 1 < top;
  const int fr = l == 0 ? kBlock : kBlock / 4;   // rows per residual block
  const int nf = (A.n + fr - 1) / fr;
  const int nu = nf + (A.n_next + kBlock / 4 - 1) / (kBlock / 4);
  const bool sa = staged<R>(A.ha, tm.cap), sr = staged<R>(A.hr, tm.cap);
  for (int u = tm.rank; u < nu; u += tm.size) {
    if (u < nf) {
      if (l == 0) {
        if (sa)
          resid_blk<R, (sizeof(R) == 4)>(A, u);
        else
          resid_blk<R, false>(A, u);
      } else {
        if (sa)
          resid4_blk<R, (sizeof(R) == 4)>(A, u);
        else
          resid4_blk<R, false>(A, u);
      }
    } else {
      if (sr)
        restrict_blk<R, (sizeof(R) == 4)>(A, C, pre, u - nf);
      else
        restrict_blk<R, false>(A, C, pre, u - nf);
    }
  }
  return team_sync(tm);
}

// coarsest level: y = C^-1 b (dense inverse) or damped-Jacobi sweeps from zero
template <typename R>
__device__ bool coarsest(const Inst &I, const Team &tm) {
  typedef typename Vec<R>::G G;
  const AmgDev &C = I.amg[I.amg_levels - 1];
  const G *b = reinterpret_cast<const G *>(C.b);
  G *y = reinterpret_cast<G *>(C.y);
  if (I.amg_coarse_sweeps == 0) {
    const R *ci = LevelVal<R>::cinv(I);
    const int n = C.n;
    LEVEL_ROWS_BEGIN(n, tm)
    R ax = R(0), ay = R(0), az = R(0);
    for (int j = 0; j < n; ++j) {
      const R a = ci[(size_t)row * n + j];
      const G t = ldg4(b + j);
      ax += a * R(t.x);
      ay += a * R(t.y);
      az += a * R(t.z);
    }
    y[row] = Vec<R>::mk(ax, ay, az);
    LEVEL_ROWS_END
    return team_sync(tm);
  }
  G *x = reinterpret_cast<G *>(C.x);
  const R *dinv = LevelVal<R>::dinv(C);
  const R om = R(C.omega);
  LEVEL_ROWS_BEGIN(C.n, tm)
  const G bi = ldg4(b + row);
  const R d = om * dinv[row];
  y[row] = Vec<R>::mk(d * R(bi.x), d * R(bi.y), d * R(bi.z));
  LEVEL_ROWS_END
  if (!team_sync(tm)) return false;
  for (int sw = 1; sw < I.amg_coarse_sweeps; ++sw) {
    G *src = (sw & 1) ? y : x;
    G *dst = (sw & 1) ? x : y;
    lv_smooth4<R, false>(C, src, dst, tm);
    if (!team_sync(tm)) return false;
  }
  if ((I.amg_coarse_sweeps & 1) == 0) {   // the last sweep wrote x: move it to y
    LEVEL_ROWS_BEGIN(C.n, tm)
    y[row] = ldg4(x + row);
    LEVEL_ROWS_END
    if (!team_sync(tm)) return false;
  }
  return true;
}

// Up step of level l in one team phase (coarse correction and post-smoothing); the output of level 0 is u
// (in g), projected onto the free components when MK and the instance has per-component constraints.
template <typename R, bool MK = false>
__device__ bool up_step(const Inst &I, int l, const Team &tm) {
  typedef typename Vec<R>::G G;
  const AmgDev &A = I.amg[l];
  const AmgDev &C = I.amg[l + 1];
  G *y = (l == 0) ? Vec<R>::g(I) : reinterpret_cast<G *>(A.y);
  const uint8_t *fix = (MK && l == 0) ? I.fix : nullptr;
  if (staged<R>(A.hp, tm.cap))
    lv_up<R, (sizeof(R) == 4), MK>(A, C, y, tm, fix);
  else
    lv_up<R, false, MK>(A, C, y, tm, fix);
  return team_sync(tm);
}

// y_d = B b_d on the dense level d: B is the cycle of levels >= d (started from zero), a fixed linear map
// set up on the host as a dense column-major matrix. This replaces that part of the cycle, a chain of
// small dependent phases, by one product. Rows are split into contiguous chunks, one per CTA of the team;
// inside a CTA, warp w sums the columns j = w, w + 8, ... in increasing order for 32 consecutive rows
// (coalesced column reads of B), and the eight partial sums of a row are added in warp order: the same
// operations whatever the team size.
template <typename R>
__device__ bool dense_level(const Inst &I, const Team &tm) {
  typedef typename Vec<R>::G G;
  constexpr int U = 8;
  const AmgDev &D = I.amg[I.amg_dense_level];
  const G *b = reinterpret_cast<const G *>(D.b);
  G *y = reinterpret_cast<G *>(D.y);
  const R *B = LevelVal<R>::dense(I);
  const int n = I.amg_dense_n;
  const int per = (n + tm.size - 1) / tm.size;
  const int r0 = tm.rank * per, r1 = min(n, r0 + per);
  double(*part)[kBlock / 32][3] = stage_buf();   // [32 rows][8 warps][3], free between reductions
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = r0; base < r1; base += 32) {
    const int i = base + lane;
    R ax = R(0), ay = R(0), az = R(0);
    if (i < r1) {
      for (int j0 = w; j0 < n; j0 += 8 * U) {
        R a[U];
        G t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + 8 * u;
          a[u] = j < n ? B[(size_t)j * n + i] : R(0);
          t[u] = ldg4(b + (j < n ? j : 0));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          ax += a[u] * R(t[u].x);
          ay += a[u] * R(t[u].y);
          az += a[u] * R(t[u].z);
        }
      }
    }
    part[lane][w][0] = double(ax);
    part[lane][w][1] = double(ay);
    part[lane][w][2] = double(az);
    __syncthreads();
    if (w == 0 && i < r1) {
      R sx = R(part[lane][0][0]), sy = R(part[lane][0][1]), sz = R(part[lane][0][2]);
      for (int g = 1; g < kBlock / 32; ++g) {
        sx += R(part[lane][g][0]);
        sy += R(part[lane][g][1]);
        sz += R(part[lane][g][2]);
      }
      y[i] = Vec<R>::mk(sx, sy, sz);
    }
    __syncthreads();
  }
  return team_sync(tm);
}

// u = B r: one symmetric V(1,1) cycle with damped-Jacobi smoothing and Galerkin coarse operators, two team
// phases per level (the sweeps folded into the transfers); the part of the cycle from the dense level down
// is one dense product (else the coarsest level is solved with its dense inverse or Jacobi sweeps); output
// u in g (AoS). Expects the level-0 pre-smoothing (done by the phase that wrote r) and a team barrier
// before it. The pre-smoothing of each coarser level is fused into the restriction that produces its
// right-hand side. Returns false on abort.
template <typename R, bool MK = false>
__device__ bool vcycle(const Inst &I, const Team &tm) {
  const int top = I.amg_dense_level > 0 ? I.amg_dense_level : I.amg_levels - 1;
  for (int l = 0; l < top; ++l)
    if (!down_step<R>(I, l, tm)) return false;
  if (!(I.amg_dense_level > 0 ? dense_level<R>(I, tm) : coarsest<R>(I, tm))) return false;
  for (int l = top - 1; l >= 0; --l)
    if (!up_step<R, MK>(I, l, tm)) return false;
  return true;
}

// Chronopoulos-Gear PCG iterations on A x = r0, given r (initial residual), x (initial guess) and
// g = D^-1 r. Stops when (r,r) <= tol2 (absolute). Returns iterations (>= 0), -1 on cap, -2 on abort,
// -3 on a non-finite reduction.
template <typename R, bool NT>
__device__ int cg_loop(const Inst &I, Team &tm, double *x, double tol2, int max_it, double *rho_out) {
  if (!team_sync(tm)) return -2;
  if (I.amg_levels > 0 && !vcycle<R, NT>(I, tm)) return -2;
  phase_spmv<R, NT>(I, tm);
  if (!team_sync(tm)) return -2;
  double red[3];
  team_reduce(I, tm, red);
  double gamma = red[0], delta = red[1], rho = red[2];
  *rho_out = rho;
  if (!isfinite(rho) || !isfinite(gamma) || !isfinite(delta)) return -3;
  if (rho <= tol2) return 0;
  double alpha = gamma / delta, beta = 0.0;
  bool first = true;
  for (int it = 1; it <= max_it; ++it) {
    phase_update<R>(I, tm, R(alpha), R(beta), first, x, alpha);
    if (!team_sync(tm)) return -2;
    if (I.amg_levels > 0 && !vcycle<R, NT>(I, tm)) return -2;
    phase_spmv<R, NT>(I, tm);
    if (!team_sync(tm)) return -2;
    team_reduce(I, tm, red);
    const double gn = red[0], dn = red[1];
    rho = red[2];
    *rho_out = rho;
    if (!isfinite(rho) || !isfinite(gn) || !isfinite(dn)) return -3;
    if (rho <= tol2) return it;
    const double bn = gn / gamma;
    alpha = gn / (dn - bn * gn / alpha);
    beta = bn;
    gamma = gn;
    first = false;
  }
  return -1;
}

// sol += xs (the inner correction, accumulated in FP64); g64 = sol
__device__ void phase_accumulate(const Inst &I, const Team &tm) {
  const int nv = I.nv;
  const double *xs = reinterpret_cast<const double *>(I.xs);
  ROWS_BEGIN(I, tm)
  double sv[3];
  for (int c = 0; c < 3; ++c) {
    const int k = c * nv + row;
    sv[c] = I.sol[k] + xs[k];
    I.sol[k] = sv[c];
  }
  reinterpret_cast<D4 *>(I.g64)[row] = {sv[0], sv[1], sv[2], 0.0};
  ROWS_END
}

// v_prev3 = v_prev2; v_prev2 = v_prev; v_prev = v; v = sol; x += dt v. Quasi-static solve: x += dt sol and the
// velocity and its history are zero (the equilibrium is at rest).
__device__ void phase_commit(const Inst &I, const Team &tm) {
  const int nv = I.nv;
  const bool st = I.nl_static != 0;
  ROWS_BEGIN(I, tm)
  for (int c = 0; c < 3; ++c) {
    const int k = c * nv + row;
    const double v = I.sol[k];
    I.vprev3[k] = st ? 0.0 : I.vprev2[k];
    I.vprev2[k] = st ? 0.0 : I.vprev[k];
    I.vprev[k] = st ? 0.0 : I.v[k];
    I.v[k] = st ? 0.0 : v;
    I.x[k] += I.dt * v;
  }
  ROWS_END
}

// Largest |sol - v_k| over the instance's rows and components (v_k = 0 at the first iteration): per-chunk
// maxima (warp shuffles, then the warps), then every CTA takes the maximum of all chunks (order-independent).
// Returns false on abort.
__device__ bool team_max_step(const Inst &I, Team &tm, double *out) {
  __shared__ double wmax[kBlock / 32];
  __shared__ double res;
  const int nv = I.nv, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool first = tm.chord_k == 0;
  for (int ch = tm.rank; ch < I.n_chunks; ch += tm.size) {
    double mx = 0.0;
    for (int rr = 0; rr < I.rows_per_thread; ++rr) {
      const int row = (ch * I.rows_per_thread + rr) * kBlock + (int)threadIdx.x;
      if (row >= nv) continue;
      for (int c = 0; c < 3; ++c) {
        const int k = c * nv + row;
        mx = fmax(mx, fabs(I.sol[k] - (first ? 0.0 : I.vk[k])));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = wmax[0];
      for (int w = 1; w < kBlock / 32; ++w) m = fmax(m, wmax[w]);
      part_of(I, tm, ch)[0] = m;
    }
    __syncthreads();
  }
  if (!team_sync(tm)) return false;
  const double *part = I.part + 4 * (size_t)tm.bank * I.n_chunks;
  tm.bank ^= 1;
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int c = threadIdx.x; c < I.n_chunks; c += 32) m = fmax(m, __ldcg(part + 4 * c));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) res = m;
  }
  __syncthreads();
  *out = res;
  return true;
}

// hand-off to the next iteration: the new iterate v_{k+1} = sol, or with the quasi-static limiter
// v_k + alpha (sol - v_k); sol = vk = g64 = v_{k+1}, xk = x + dt v_{k+1} (where the next forces are evaluated)
__device__ void phase_chord(const Inst &I, const Team &tm, double alpha, bool limit) {
  const int nv = I.nv;
  const bool first = tm.chord_k == 0;
  ROWS_BEGIN(I, tm)
  double sv[3];
  for (int c = 0; c < 3; ++c) {
    const int k = c * nv + row;
    sv[c] = I.sol[k];
    if (limit) {
      const double v0 = first ? 0.0 : I.vk[k];
      sv[c] = v0 + alpha * (sv[c] - v0);
      I.sol[k] = sv[c];
      I.vk[k] = sv[c];
    }
    I.xk[k] = I.x[k] + I.dt * sv[c];
  }
  reinterpret_cast<D4 *>(I.g64)[row] = {sv[0], sv[1], sv[2], 0.0};
  ROWS_END
}

// stop test of an iteration of exact backward Euler or of the quasi-static solve: the current iterate's
// residual r2 = ||R(v_k)||^2 meets nl_rtol ||R(0)|| (r0 = ||R(0)||^2) or dt nl_atol
__device__ inline bool nl_done(const Inst &I, double r2, double r0) {
  const double a = I.dt * I.nl_atol;
  return r2 <= fmax(I.nl_rtol * I.nl_rtol * r0, a * a);
}

// squared floor of the linear solves of iterations k > 0: a tenth of the nonlinear target, since solving the
// correction beyond what the stop test can see only costs iterations (and in FP32 with refinement runs into
// the FP64 residual's rounding once ||R(v_k)|| is far below ||R(0)||)
__device__ inline double nl_floor2(const Inst &I) {
  const double r0 = __ldcg(&I.status->nl_r0);
  const double a = I.dt * I.nl_atol;
  return 0.01 * fmax(I.nl_rtol * I.nl_rtol * r0, a * a);
}

__device__ void set_status(const Inst &I, const Team &tm, int err, int iters, int rounds, double rel) {
  if (tm.rank == 0 && threadIdx.x == 0) {
    InstStatus *s = I.status;
    s->last_ns = (long long)(gtimer() - tm.t0);
    s->max_ns = s->last_ns > s->max_ns ? s->last_ns : s->max_ns;
    s->team_size = tm.size;
    if (err == SHELL_OK) {
      s->steps_done += 1;
      s->last_iters = iters;
      s->last_rounds = rounds;
      s->total_iters += iters;
      s->total_rounds += rounds;
      s->rel_res = rel;
    } else {
      s->err = err;
      s->fail_step = s->steps_done;
      s->last_iters = iters;
      s->last_rounds = rounds;
      s->rel_res = rel;
      s->nl_flags = 0;
    }
  }
}

// End of one solve of a step. Linearised step (nl_max <= 1): commit v, x. Exact backward Euler: commit
// when the chord iteration met its tolerance before this solve (done_early) or used its nl_max solves,
// else hand off to the next iteration. bb: ||b||^2 of this solve (at k = 0: ||R(0)||^2).
// Returns false, writing nothing, if a bounded wait of the launch has given up: a CTA that timed out leaves
// the launch, and its team mates may still pass the barrier before the commit (its last arrival completes
// it), so every CTA checks the abort flag once before it writes the state; an abandoned launch then commits
// nothing.
__device__ bool finish_step(const Inst &I, Team &tm, double bb, int iters, int rounds, double rel,
                            bool done_early) {
  const int k = tm.chord_k;
  if (ld_volatile_i(tm.abort_flag)) return false;
  if (I.nl_max <= 1) {
    phase_commit(I, tm);
    set_status(I, tm, SHELL_OK, iters, rounds, rel);
    return true;
  }
  const int solves = done_early ? k : k + 1;
  const bool last = done_early || solves >= I.nl_max;
  if (last && !done_early && I.nl_static) {
    // quasi-static: the iteration limit came before the residual met eps_f; nothing is committed
    set_status(I, tm, SHELL_ERR_NOT_CONVERGED, iters, rounds, rel);
    return true;
  }
  if (last) {
    phase_commit(I, tm);
  } else {
    const bool limit = I.nl_static && I.nl_eps_u > 0.0;
    double alpha = 1.0;
    if (limit) {
      double mx = 0.0;
      if (!team_max_step(I, tm, &mx)) return false;
      const double d = I.dt * mx;
      alpha = d > I.nl_eps_u ? I.nl_eps_u / d : 1.0;
    }
    phase_chord(I, tm, alpha, limit);
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    InstStatus *s = I.status;
    const long long step_pcg = (k == 0 ? 0 : s->nl_step_pcg) + iters;
    s->last_ns = (long long)(gtimer() - tm.t0);
    s->max_ns = s->last_ns > s->max_ns ? s->last_ns : s->max_ns;
    s->team_size = tm.size;
    s->total_iters += iters;
    s->total_rounds += rounds;
    s->nl_iters = solves;
    if (k == 0) s->nl_r0 = bb;
    if (last) {
      s->steps_done += 1;
      s->last_iters = (int)step_pcg;
      s->last_rounds = rounds;
      s->rel_res = rel;
      s->nl_flags = done_early ? 0 : 2;
    } else {
      s->nl_step_pcg = step_pcg;
      s->nl_flags = 1;
    }
  }
  return true;
}

// returns false if the kernel must stop (abort). Chord iteration k > 0 of an exact backward-Euler step: the
// first residual of the solve is the backward-Euler residual R(v_k); if it meets nl_rtol ||R(0)|| the step
// commits v_k without solving, else the solve's tolerance refers to it.
// FP64 instances get their forces from the standalone force launch before this one: the FP64 stencil needs
// more registers than the FP64 solve variant has (126 at 2 CTAs per SM) and spilled there (a batch256 step of
// the plain FP64 path took 16.6 instead of 14.6 ms with the phase inside).
template <bool NT>
__device__ bool solve_fp64(const Inst &I, Team &tm) {
  const int k = tm.chord_k;
  phase_rhs<double, NT>(I, tm);
  if (!team_sync(tm)) return false;
  double red[3];
  team_reduce(I, tm, red);
  const double bb = red[0];
  if (!isfinite(bb)) {
    set_status(I, tm, SHELL_ERR_NONFINITE, 0, 0, 0.0);
    return true;
  }
  int iters = 0;
  double rho = 0.0, ref = bb;
  // quasi-static, first iteration: the start (v_0 = 0, b = dt (f + f_ext)) may already be in equilibrium
  bool early = k == 0 && I.nl_static && nl_done(I, bb, bb);
  if (early) rho = bb;
  if (bb > 0.0 && !early) {
    phase_resid<double, NT>(I, tm);   // r = b - A sol, g = D^-1 r
    if (k > 0) {
      if (!team_sync(tm)) return false;
      team_reduce(I, tm, red);
      rho = red[0];
      if (!isfinite(rho)) {
        set_status(I, tm, SHELL_ERR_NONFINITE, 0, 0, 0.0);
        return true;
      }
      const double r0 = __ldcg(&I.status->nl_r0);
      early = nl_done(I, rho, r0);
      ref = early ? r0 : rho;
    }
    if (!early) {
      // iteration k > 0: no need to solve below a tenth of the nonlinear target (inexact Newton)
      const double tol2 = fmax(I.pcg_rtol * I.pcg_rtol * ref, k > 0 ? nl_floor2(I) : 0.0);
      iters = cg_loop<double, NT>(I, tm, I.sol, tol2, I.pcg_max_it, &rho);
      if (iters == -2) return false;
      if (iters < 0) {
        set_status(I, tm, iters == -1 ? SHELL_ERR_NOT_CONVERGED : SHELL_ERR_NONFINITE, I.pcg_max_it, 0,
                   sqrt(rho / ref));
        return true;
      }
    }
  } else if (!early) {
    // b = 0: the solution is v' = 0
    ROWS_BEGIN(I, tm)
    for (int c = 0; c < 3; ++c) I.sol[c * I.nv + row] = 0.0;
    ROWS_END
  }
  // quasi-static: the reported residual is ||f + f_ext|| of the committed iterate
  const double rel = (I.nl_static && early) ? sqrt(rho) / I.dt : (ref > 0.0 ? sqrt(rho / ref) : 0.0);
  return finish_step(I, tm, bb, iters, 0, rel, early);
}

template <bool NT>
__device__ bool solve_fp32r(const Inst &I, Team &tm) {
  const int k = tm.chord_k;
  phase_forces<float, NT>(I, tm);
  if (!team_sync(tm)) return false;
  phase_rhs<float, NT>(I, tm);
  if (!team_sync(tm)) return false;
  double red[3];
  team_reduce(I, tm, red);
  const double bb = red[0];
  if (!isfinite(bb)) {
    set_status(I, tm, SHELL_ERR_NONFINITE, 0, 0, 0.0);
    return true;
  }
  int total = 0, rounds = 0;
  double rel = 0.0, ref = bb;
  bool early = false;
  if (bb > 0.0) {
    double tol_ref2 = I.refine_rtol * I.refine_rtol * bb;
    const double tin2 = I.pcg_rtol * I.pcg_rtol;
    for (;;) {
      phase_resid<float, NT>(I, tm);
      if (!team_sync(tm)) return false;
      team_reduce(I, tm, red);
      const double r2 = red[0];
      if (!isfinite(r2)) {
        set_status(I, tm, SHELL_ERR_NONFINITE, total, rounds, sqrt(r2 / ref));
        return true;
      }
      if (rounds == 0 && (k > 0 || I.nl_static)) {   // iteration k: r2 = ||R(v_k)||^2 (v_0 = 0 when static)
        const double r0 = k > 0 ? __ldcg(&I.status->nl_r0) : r2;
        if (nl_done(I, r2, r0)) {
          early = true;
          rel = I.nl_static ? sqrt(r2) / I.dt : (r0 > 0.0 ? sqrt(r2 / r0) : 0.0);
          break;
        }
        ref = r2;
        // no need to solve below a tenth of the nonlinear target (inexact Newton)
        tol_ref2 = fmax(I.refine_rtol * I.refine_rtol * r2, k > 0 ? nl_floor2(I) : 0.0);
      }
      rel = sqrt(r2 / ref);
      if (r2 <= tol_ref2) break;
      if (rounds >= I.refine_max) {
        set_status(I, tm, SHELL_ERR_NOT_CONVERGED, total, rounds, rel);
        return true;
      }
      // inner target: the relative reduction pcg_rtol, but no further than 0.7 of the refinement target (a
      // round that starts close to it needs only a few iterations; the FP64 test above decides, and a
      // margin of 0.7 leaves room for the FP32 recurrence's drift), and at least a halving
      const double tol2 = fmin(fmax(tin2 * r2, 0.5 * tol_ref2), 0.25 * r2);
      double rho = 0.0;
      const int it = cg_loop<float, NT>(I, tm, reinterpret_cast<double *>(I.xs), tol2, I.pcg_max_it, &rho);
      if (it == -2) return false;
      if (it == -3) {
        set_status(I, tm, SHELL_ERR_NONFINITE, total, rounds, rel);
        return true;
      }
      total += (it < 0 ? I.pcg_max_it : it);
      phase_accumulate(I, tm);
      if (!team_sync(tm)) return false;
      ++rounds;
    }
  } else {
    ROWS_BEGIN(I, tm)
    for (int c = 0; c < 3; ++c) I.sol[c * I.nv + row] = 0.0;
    ROWS_END
  }
  return finish_step(I, tm, bb, total, rounds, rel, early);
}

// PREC: 0 = instances of either precision, 1 = FP64 instances only, 2 = FP32-refinement instances only.
// MINB: CTAs per SM the register allocation is bounded for (the FP32 variant is compiled for 3, 4 and 5;
// more resident warps mean more loads in flight, at the price of register spills; the autotuner picks).
// NT: the variant carries the Newton tangent (launched for batches with a Newton instance; the others run
// variants without that code, whose register allocation it would otherwise burden).
template <int PREC, int MINB, bool NT = false>
__global__ void __launch_bounds__(kBlock, MINB) k_solve(const Inst *__restrict__ insts, Sched sch) {
  Team tm;
  tm.team = sch.cta_team[blockIdx.x];
  if (tm.team < 0) return;
  tm.rank = sch.cta_rank[blockIdx.x];
  tm.size = sch.team_size[tm.team];
  tm.bar = sch.bar + kBarWords * tm.team;
  tm.abort_flag = sch.abort_flag;
  tm.bank = 0;
  tm.cluster = sch.cluster;
  tm.cluster_ok = sch.cluster_ok;
  tm.cap = sch.halo_cap;
  tm.chord_k = sch.chord_k;
  tm.wait_ns = sch.wait_ns;
  if (tm.size == 1)
    tm.mode = 0;
  else if (sch.cluster > 0 && tm.size % sch.cluster == 0)
    tm.mode = (tm.size == sch.cluster) ? 2 : 3;
  else
    tm.mode = 1;
  // The team's own list first, then the shared queue of one-CTA instances, which every CTA serves once its
  // team's list is done (results do not depend on which CTA solves an instance). Both feed the same solver
  // call: a second, separately inlined call with the team size known to be 1 compiled to different rounding.
  __shared__ int s_q;
  const int q_end = sch.team_ptr[tm.team + 1];
  int q = sch.team_ptr[tm.team];
  const int team_size = tm.size, team_rank = tm.rank, team_mode = tm.mode;
  bool in_queue = false;
  for (;;) {
    int idx;
    if (q < q_end) {
      idx = sch.team_list[q++];
    } else {
      if (sch.n_queue <= 0) break;
      if (threadIdx.x == 0) s_q = ld_volatile_i(tm.abort_flag) ? sch.n_queue : (int)atomicAdd(sch.queue_ctr, 1u);
      __syncthreads();
      const int qq = s_q;
      __syncthreads();
      if (qq >= sch.n_queue) break;
      idx = sch.queue[qq];
      in_queue = true;
    }
    tm.size = in_queue ? 1 : team_size;
    tm.rank = in_queue ? 0 : team_rank;
    tm.mode = in_queue ? 0 : team_mode;
    const Inst &I = insts[idx];
    if (I.status->err != SHELL_OK) continue;
    if (sch.chord_k > 0 && !(I.status->nl_flags & 1)) continue;   // no chord iteration in progress
    tm.t0 = gtimer();
    bool ok;
    if (PREC == 1 || (PREC == 0 && I.precision == SHELL_FP64))
      ok = solve_fp64<NT>(I, tm);
    else
      ok = solve_fp32r<NT>(I, tm);
    if (!ok) return;
    // make this instance's final writes (status) ordered before the team moves on
    if (!team_sync(tm)) return;
  }
}

}  // namespace

// kernel of a precision mode and an occupancy variant (FP32: 3, 4 or 5 CTAs per SM; others: 2); prec 3: either
// precision with the Newton tangent
typedef void (*SolveFn)(const Inst *, Sched);
static SolveFn solve_fn(int prec, int occ) {
  if (prec == 3) return k_solve<0, 2, true>;
  if (prec == 2) {
    if (occ >= 5) return k_solve<2, 5>;
    if (occ == 4) return k_solve<2, 4>;
    return k_solve<2, 3>;
  }
  if (prec == 1) return k_solve<1, 2>;
  return k_solve<0, 2>;
}

// Entries of the shared-memory staging buffer per CTA: as many as fit beside the static shared memory at the
// variant's CTAs per SM (228 KB per SM, 1 KB reserved per CTA). FP64-only launches stage nothing.
int solve_halo_cap(int prec, int occ) {
  if (prec == 1) return 0;
  if (prec == 2 && occ >= 5) return 2048;
  if (prec == 2 && occ == 4) return 3072;
  return 4096;
}

static cudaError_t prepare_solve_fn(int prec, int occ) {
  static bool done[4][6];
  const int o = std::min(5, std::max(0, occ));
  if (done[prec][o]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(solve_fn(prec, occ), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       16 * solve_halo_cap(prec, occ));
  if (e == cudaSuccess) done[prec][o] = true;
  return e;
}

int solve_blocks_per_sm(int prec, int occ) {
  int n = 0;
  if (prepare_solve_fn(prec, occ) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, solve_fn(prec, occ), kBlock, 16 * solve_halo_cap(prec, occ));
  return n;
}

// Cluster launches are not cooperative: the scheduler uses clusters only when every team is one CTA or one
// whole cluster (hardware co-schedules a cluster, and no team waits for CTAs outside its cluster); teams
// larger than a cluster need the cooperative launch (all CTAs co-resident) and use global barriers.
cudaError_t launch_solve(const Inst *d_insts, const Sched &sched, int grid, int prec, int occ, cudaStream_t st) {
  cudaError_t e = prepare_solve_fn(prec, occ);
  if (e != cudaSuccess) return e;
  Sched sc = sched;
  sc.halo_cap = solve_halo_cap(prec, occ);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 16 * (size_t)sc.halo_cap;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (sched.cluster > 0) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sched.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  } else {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, solve_fn(prec, occ), d_insts, sc);
}

int solve_max_clusters(int prec, int cluster) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kBlock);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.dynamicSmemBytes = 16 * (size_t)solve_halo_cap(prec, 3);
  int n = 0;
  cudaError_t e = prepare_solve_fn(prec, 3);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, solve_fn(prec, 3), &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// ---------------------------------------------------------------- step without device allocation
// The launch scratch of the persistent solve (team schedule, barrier words, abort flag, status read-back)
// for callers that cannot allocate device memory: it lives in this file-scope array, which every GPU that
// loads the library holds until the process exits. Layout (32-bit words): [0, kStaticMaxCtas) team of each
// CTA, [kStaticMaxCtas, 2 kStaticMaxCtas) rank, then team_size[1], team_ptr[2], team_list[1], the barrier
// words (kBarWords), the abort flag, its read-back copy, and one InstStatus.
constexpr int kStaticMaxCtas = 2048;
constexpr int kStaticBar = 2 * kStaticMaxCtas + 32;                 // 128-byte aligned word offset
constexpr int kStaticAbort = kStaticBar + kBarWords;                // abort flag, then its read-back copy
constexpr int kStaticStatus = kStaticAbort + 8;                     // one InstStatus (8-byte aligned)
constexpr int kStaticWords = kStaticStatus + (int)(sizeof(InstStatus) / 4) + 4;
static __device__ __align__(256) unsigned int g_static_scratch[kStaticWords];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_static_scratch, per device. Threads calling on different handles may fill an entry at
// the same time: each then looks the address up itself (the same value) and stores it, so the entries are
// atomics and the race is benign.
std::atomic<unsigned int *> g_static_addr[kMaxDevices];
}  // namespace

cudaError_t static_scratch_setup(unsigned int **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned int *a = g_static_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    a = reinterpret_cast<unsigned int *>(p);
    g_static_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return cudaSuccess;
}

int static_max_ctas() { return kStaticMaxCtas; }

cudaError_t launch_step_static(const Inst *d_inst, const Tile *d_tiles, int n_tiles, int fp32, int newton,
                               int team_ctas, int n_steps, int chord_launches, InstStatus *h_status,
                               int32_t *h_aborted, cudaStream_t st) {
  unsigned int *base = nullptr;
  cudaError_t e = static_scratch_setup(&base);
  if (e != cudaSuccess) return e;
  if (team_ctas < 1 || team_ctas > kStaticMaxCtas) return cudaErrorInvalidValue;
  // schedule: one team of team_ctas CTAs working on instance 0
  int32_t *w = reinterpret_cast<int32_t *>(base);
  Sched sc;
  sc.cta_team = w;
  sc.cta_rank = w + kStaticMaxCtas;
  sc.team_size = w + 2 * kStaticMaxCtas;
  sc.team_ptr = w + 2 * kStaticMaxCtas + 1;
  sc.team_list = w + 2 * kStaticMaxCtas + 3;
  sc.bar = base + kStaticBar;
  sc.abort_flag = w + kStaticAbort;
  int32_t *abort_out = sc.abort_flag + 1;
  InstStatus *status_out = reinterpret_cast<InstStatus *>(base + kStaticStatus);
  sc.n_ctas = team_ctas;
  sc.cluster = 0;
  sc.cluster_ok = nullptr;
  sc.wait_ns = (unsigned long long)kMaxTeamWaitMs * 1000000ull;
  sc.queue = nullptr;
  sc.queue_ctr = nullptr;
  sc.n_queue = 0;
  static thread_local int32_t host_tab[2 * kStaticMaxCtas + 4];
  for (int c = 0; c < team_ctas; ++c) {
    host_tab[c] = 0;
    host_tab[kStaticMaxCtas + c] = c;
  }
  host_tab[2 * kStaticMaxCtas] = team_ctas;
  host_tab[2 * kStaticMaxCtas + 1] = 0;
  host_tab[2 * kStaticMaxCtas + 2] = 1;
  host_tab[2 * kStaticMaxCtas + 3] = 0;
  if ((e = cudaMemcpyAsync(sc.cta_team, host_tab, 4 * team_ctas, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(sc.cta_rank, host_tab + kStaticMaxCtas, 4 * team_ctas, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(sc.team_size, host_tab + 2 * kStaticMaxCtas, 16, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  // the barrier words and the abort flag must start at zero; the array keeps the previous call's contents
  if ((e = cudaMemsetAsync(sc.bar, 0, 4 * (kBarWords + 2), st)) != cudaSuccess) return e;
  for (int step = 0; step < n_steps; ++step) {
    for (int k = 0; k < chord_launches; ++k) {   // chord iterations of an exact backward-Euler step
      if (!fp32 && (e = launch_forces(d_inst, d_tiles, n_tiles, 0, 0, st, k)) != cudaSuccess) return e;
      sc.chord_k = k;
      if ((e = launch_solve(d_inst, sc, team_ctas, newton ? 3 : (fp32 ? 2 : 1), 3, st)) != cudaSuccess) return e;
    }
  }
  if ((e = launch_gather_status(d_inst, 1, status_out, sc.abort_flag, abort_out, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(h_status, status_out, sizeof(InstStatus), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(h_aborted, abort_out, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *h_aborted) {
    cudaMemsetAsync(sc.bar, 0, 4 * (kBarWords + 2), st);
    e = cudaStreamSynchronize(st);
  }
  return e;
}

}  // namespace shl
