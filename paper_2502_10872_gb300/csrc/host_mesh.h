// host_mesh.h -- host-side topology: stencils, force-gather incidence, SELL sparsity, assembly sources.
#pragma once
#include <cstdint>
#include <vector>

namespace shl {

struct HostTopo {
  int nv = 0, nt = 0, model = 0;
  int kt = 3;                        // contribution slots per triangle
  std::vector<int32_t> t_idx;        // [6][nt] relabelled triangle stencils (-1 = virtual)
  std::vector<uint8_t> t_bc;         // [3][nt]
  int ne = 0, ne_int = 0;            // edge stencils (interior first, then clamped)
  std::vector<int32_t> e_idx;        // [4][ne]
  int n_slots = 0;
  std::vector<int32_t> vtx_ptr, vtx_slot;
  int n_slices = 0;
  std::vector<int32_t> sl_ptr, sl_col, diag_pos;
  int64_t nnz = 0;                   // structural nonzeros (without padding)
  std::vector<int32_t> row_ptr;      // CSR structure of the scalar matrix (row lengths)
  int n_local = 0;
  std::vector<int32_t> asm_ptr, asm_src;
};

// Builds the topology of a consistently oriented manifold mesh. Returns SHELL_OK or
// SHELL_ERR_INVALID_ARG / SHELL_ERR_NON_MANIFOLD / SHELL_ERR_BAD_ORIENTATION.
int build_topology(int nv, int nt, const int32_t *tris, int n_clamped, const int32_t *clamped, int model,
                   HostTopo *out);

}  // namespace shl
