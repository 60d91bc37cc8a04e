// kernels_force.cu -- per-stencil elastic forces and energies (standalone launches: shell_forces,
// shell_energy), state layout conversions.
//
// One thread per stencil (the stencil arithmetic is in stencil_force.cuh). Each stencil writes its nodal forces
// to its own contribution slots; the right-hand side (and shell_forces) later sums each vertex's slots in a
// fixed order, so results are deterministic.
#include <cmath>

#include "stencil_force.cuh"

namespace shl {
namespace {

// FP64 forces of the instances in the tiles (FP64 steps, energies, shell_forces; FP32 instances evaluate their
// forces inside the step kernel). chord_k > 0: a later iteration of the exact backward-Euler step; only
// instances whose step is in such an iteration take part, with forces at their iterate positions xk.
template <typename R>
__global__ void __launch_bounds__(kForceBlock, 1)
    k_forces(const Inst *__restrict__ insts, const Tile *__restrict__ tiles, int want_energy, int chord_k) {
  const Tile tl = tiles[blockIdx.x];
  const Inst &I = insts[tl.inst];
  if (!want_energy && I.status->err != SHELL_OK) return;
  if (chord_k > 0 && !(I.status->nl_flags & 1)) return;
  if ((int)threadIdx.x >= tl.count) return;
  const int s = tl.first + threadIdx.x;
  const Data<R> D(I, chord_k > 0 ? I.xk : I.x);
  if (tl.kind == 0)
    tri_stencil<R>(I, D, s, want_energy != 0);
  else
    edge_stencil<R>(I, D, s, want_energy != 0);
}

// per-vertex sum of FP64 contributions, written row-major [V][3]
__global__ void k_gather_forces(const Inst *__restrict__ pI, double *out) {
  const Inst &I = *pI;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.nv) return;
  const double *c = reinterpret_cast<const double *>(I.contrib);
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int q = I.vtx_ptr[i]; q < I.vtx_ptr[i + 1]; ++q) {
    const int s = I.vtx_slot[q];
    fx += c[3 * (size_t)s];
    fy += c[3 * (size_t)s + 1];
    fz += c[3 * (size_t)s + 2];
  }
  out[3 * i] = fx;
  out[3 * i + 1] = fy;
  out[3 * i + 2] = fz;
}

// energies: one block, fixed-order strided sums then a fixed tree
__global__ void k_energy_reduce(const Inst *__restrict__ pI, double *out4) {
  const Inst &I = *pI;
  __shared__ double sm[4][256];
  double eb = 0.0, em = 0.0, ek = 0.0, ex = 0.0;
  const int ns = I.nt + I.ne;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    eb += I.ebuf[2 * s];
    em += I.ebuf[2 * s + 1];
  }
  const int nv = I.nv;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double v = I.v[c * nv + i];
      ek += 0.5 * I.mass[i] * v * v;
      ex -= I.fext[c * nv + i] * (I.x[c * nv + i] - I.rest[c * nv + i]);
    }
  }
  sm[0][threadIdx.x] = em;
  sm[1][threadIdx.x] = eb;
  sm[2][threadIdx.x] = ek;
  sm[3][threadIdx.x] = ex;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out4[threadIdx.x] = sm[threadIdx.x][0];
}

// out = A in for row-major [V][3] FP64 vectors (SELL-32 FP64 values)
__global__ void k_matvec64(const Inst *__restrict__ pI, const double *in, double *out) {
  const Inst &I = *pI;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.nv) return;
  const int s = i >> 5, lane = i & 31;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int p = I.sl_ptr[s] + lane; p < I.sl_ptr[s + 1]; p += 32) {
    const int c = I.sl_col[p];
    const double a = I.val64[p];
    a0 += a * in[3 * c];
    a1 += a * in[3 * c + 1];
    a2 += a * in[3 * c + 2];
  }
  out[3 * i] = a0;
  out[3 * i + 1] = a1;
  out[3 * i + 2] = a2;
}

// batch state transfer: rows of all instances concatenated in table order, offs[k] = first row of
// instance k (offs[n] = total); pack: SoA x, v of every instance -> AoS [rows][3] x then v; unpack: reverse
__device__ inline int find_inst(const long long *offs, int n, long long row) {
  int lo = 0, hi = n;   // largest k with offs[k] <= row
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= row) lo = mid; else hi = mid;
  }
  return lo;
}
// One row per thread (any alignment of the packed buffers).
__global__ void k_pack_states(const Inst *__restrict__ insts, int n, const long long *__restrict__ offs, double *x,
                              double *v, int unpack) {
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= offs[n]) return;
  const int k = find_inst(offs, n, row);
  const Inst &I = insts[k];
  const int i = (int)(row - offs[k]);
  for (int c = 0; c < 3; ++c) {
    if (unpack) {
      I.x[c * I.nv + i] = x[3 * row + c];
      I.v[c * I.nv + i] = v[3 * row + c];
    } else {
      x[3 * row + c] = I.x[c * I.nv + i];
      v[3 * row + c] = I.v[c * I.nv + i];
    }
  }
}

// Packed buffers with 16-byte aligned bases: each warp moves the 64 rows [64 w, 64 w + 64) as one contiguous
// run of 1,536 bytes per array, lane L of pass j taking the 16-byte chunk 32 j + L (three fully coalesced
// passes, also over the host link when the buffers are mapped host memory), and the rows are distributed
// through shared memory to the per-instance SoA arrays (lane L: rows 64 w + L and 64 w + 32 + L). A run
// ending on half a chunk moves its last value alone.
constexpr int kPackRowsPerWarp = 64;
__global__ void __launch_bounds__(256) k_pack_states_vec(const Inst *__restrict__ insts, int n,
                                                         const long long *__restrict__ offs, double *x, double *v,
                                                         int unpack) {
  __shared__ double sx[8][3 * kPackRowsPerWarp], sv[8][3 * kPackRowsPerWarp];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long rows = offs[n];
  const long long r0 = ((long long)blockIdx.x * 8 + w) * kPackRowsPerWarp;
  if (r0 >= rows) return;
  const long long d0 = 3 * r0;
  const int nd = (int)(3 * (rows - r0 < kPackRowsPerWarp ? rows - r0 : kPackRowsPerWarp));   // doubles of the run
  double *bx = sx[w], *bv = sv[w];
  if (unpack) {
    for (int j = 0; j < 3; ++j) {
      const int q = 2 * (32 * j + lane);
      if (q + 1 < nd) {
        const double2 a = *reinterpret_cast<const double2 *>(x + d0 + q);
        const double2 b = *reinterpret_cast<const double2 *>(v + d0 + q);
        bx[q] = a.x;
        bx[q + 1] = a.y;
        bv[q] = b.x;
        bv[q + 1] = b.y;
      } else if (q < nd) {
        bx[q] = x[d0 + q];
        bv[q] = v[d0 + q];
      }
    }
    __syncwarp();
  }
  for (int h = 0; h < 2; ++h) {
    const int l = 32 * h + lane;
    const long long row = r0 + l;
    if (row < rows) {
      const int k = find_inst(offs, n, row);
      const Inst &I = insts[k];
      const int i = (int)(row - offs[k]);
      for (int c = 0; c < 3; ++c) {
        if (unpack) {
          I.x[c * I.nv + i] = bx[3 * l + c];
          I.v[c * I.nv + i] = bv[3 * l + c];
        } else {
          bx[3 * l + c] = I.x[c * I.nv + i];
          bv[3 * l + c] = I.v[c * I.nv + i];
        }
      }
    }
  }
  if (!unpack) {
    __syncwarp();
    for (int j = 0; j < 3; ++j) {
      const int q = 2 * (32 * j + lane);
      if (q + 1 < nd) {
        *reinterpret_cast<double2 *>(x + d0 + q) = make_double2(bx[q], bx[q + 1]);
        *reinterpret_cast<double2 *>(v + d0 + q) = make_double2(bv[q], bv[q + 1]);
      } else if (q < nd) {
        x[d0 + q] = bx[q];
        v[d0 + q] = bv[q];
      }
    }
  }
}

__global__ void k_aos_to_soa(const double *src, double *dst, int nv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  for (int c = 0; c < 3; ++c) dst[c * nv + i] = src[3 * i + c];
}
__global__ void k_soa_to_aos(const double *src, double *dst, int nv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  for (int c = 0; c < 3; ++c) dst[3 * i + c] = src[c * nv + i];
}

__global__ void k_gather_status(const Inst *__restrict__ insts, int n, InstStatus *out, const int32_t *abort_flag,
                                int32_t *out_abort) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    out[k] = *insts[k].status;
    insts[k].status->max_ns = 0;
  }
  if (k == 0) *out_abort = *abort_flag;
}

}  // namespace

cudaError_t launch_gather_status(const Inst *d_insts, int n, InstStatus *d_out, const int32_t *d_abort,
                                 int32_t *d_out_abort, cudaStream_t st) {
  k_gather_status<<<(n + 127) / 128, 128, 0, st>>>(d_insts, n, d_out, d_abort, d_out_abort);
  return cudaGetLastError();
}

// fp32 != 0 is not a launch of this kernel any more: FP32 forces are a phase of the step kernel
cudaError_t launch_forces(const Inst *d_insts, const Tile *d_tiles, int n_tiles, int want_energy, int fp32,
                          cudaStream_t st, int chord_k) {
  if (fp32) return cudaErrorInvalidValue;
  if (n_tiles <= 0) return cudaSuccess;
  k_forces<double><<<n_tiles, kForceBlock, 0, st>>>(d_insts, d_tiles, want_energy, chord_k);
  return cudaGetLastError();
}

cudaError_t launch_gather_forces(const Inst *d, const Inst &h, double *out, cudaStream_t st) {
  k_gather_forces<<<(h.nv + 255) / 256, 256, 0, st>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const Inst *d, const Inst &h, double *out4, cudaStream_t st) {
  (void)h;
  k_energy_reduce<<<1, 256, 0, st>>>(d, out4);
  return cudaGetLastError();
}

cudaError_t launch_matvec64(const Inst *d, const Inst &h, const double *in, double *out, cudaStream_t st) {
  k_matvec64<<<(h.nv + 255) / 256, 256, 0, st>>>(d, in, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_states(const Inst *d_insts, int n, const long long *d_offs, long long rows, double *d_x,
                               double *d_v, int unpack, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(d_x) | reinterpret_cast<uintptr_t>(d_v)) % 16 == 0) {
    const long long per_block = 8LL * kPackRowsPerWarp;
    k_pack_states_vec<<<(unsigned)((rows + per_block - 1) / per_block), 256, 0, st>>>(d_insts, n, d_offs, d_x, d_v,
                                                                                    unpack);
  } else {
    k_pack_states<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(d_insts, n, d_offs, d_x, d_v, unpack);
  }
  return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double *src, double *dst, int nv, cudaStream_t st) {
  k_aos_to_soa<<<(nv + 255) / 256, 256, 0, st>>>(src, dst, nv);
  return cudaGetLastError();
}
cudaError_t launch_soa_to_aos(const double *src, double *dst, int nv, cudaStream_t st) {
  k_soa_to_aos<<<(nv + 255) / 256, 256, 0, st>>>(src, dst, nv);
  return cudaGetLastError();
}

}  // namespace shl
