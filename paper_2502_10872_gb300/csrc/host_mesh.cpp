// host_mesh.cpp -- stencils and sparsity of a triangle mesh, built once per mesh on the host.
//
// Edge-based stencil (Section 4.3): hinge edge 2-3 and wings 1, 4; T123 and T432 are the mesh's own
// triangles. Triangle-centred stencil (Section 4.4-4.5, App. C Eq. 78): central triangle 1-2-3 and the
// vertex i+3 across the edge opposite vertex i. A missing neighbour (boundary edge) is a virtual node
// (Section 4.3 boundary conditions); its index is -1 and the device precompute places it at M + N - L.
// A triangle with a free boundary edge is rotated so its first free edge (order 1-2, 2-3, 3-1) becomes
// edge 1-2: the corotational x axis (along x_12, App. A) then follows the boundary, the frame in which the
// FVM hinge drops its twist term on free edges (Section 4.4, boundary conditions).
#include "host_mesh.h"

#include <algorithm>
#include <cstring>

#include "../../include/shell.h"

namespace shl {

namespace {

struct DirEdge {
  uint64_t key;   // p * nv + q
  int32_t tri;
  int32_t opp;    // vertex opposite the directed edge p -> q
};

}  // namespace

int build_topology(int nv, int nt, const int32_t *tris, int n_clamped, const int32_t *clamped, int model,
                   HostTopo *out) {
  HostTopo &T = *out;
  T = HostTopo();
  T.nv = nv;
  T.nt = nt;
  T.model = model;
  const bool edge_model = (model == SHELL_EP || model == SHELL_ES);
  T.kt = edge_model ? 3 : 6;
  const uint64_t N = (uint64_t)nv;

  for (int t = 0; t < nt; ++t) {
    int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return SHELL_ERR_INVALID_ARG;
    if (a == b || b == c || a == c) return SHELL_ERR_INVALID_ARG;
  }

  // ---- directed edges, sorted by key p * nv + q: bucketed by the source vertex p (a counting sort), then
  // ordered by q inside each bucket (a few entries)
  std::vector<DirEdge> de((size_t)nt * 3);
  std::vector<int32_t> out_ptr(nv + 1, 0);   // de[out_ptr[p] .. out_ptr[p + 1]): the edges leaving p
  for (size_t i = 0; i < (size_t)nt * 3; ++i) out_ptr[tris[i] + 1]++;
  for (int i = 0; i < nv; ++i) out_ptr[i + 1] += out_ptr[i];
  {
    std::vector<int32_t> fill(out_ptr.begin(), out_ptr.end() - 1);
    for (int t = 0; t < nt; ++t) {
      const int32_t *v = tris + 3 * t;
      for (int k = 0; k < 3; ++k) {
        const int p = v[k], q = v[(k + 1) % 3], r = v[(k + 2) % 3];
        de[fill[p]++] = {(uint64_t)p * N + (uint64_t)q, t, r};
      }
    }
  }
  for (int p = 0; p < nv; ++p)
    for (int i = out_ptr[p] + 1; i < out_ptr[p + 1]; ++i)   // insertion sort: keys are distinct or an error
      for (int j = i; j > out_ptr[p] && de[j].key < de[j - 1].key; --j) std::swap(de[j], de[j - 1]);
  for (size_t i = 1; i < de.size(); ++i) {
    if (de[i].key == de[i - 1].key) {
      // the same directed edge twice: either >2 triangles on the edge or a flipped neighbour
      uint64_t p = de[i].key / N, q = de[i].key % N;
      uint64_t tw = q * N + p;
      auto it = std::lower_bound(de.begin(), de.end(), tw, [](const DirEdge &x, uint64_t k) { return x.key < k; });
      int mult = 2;
      while (it != de.end() && it->key == tw) { ++mult; ++it; }
      return mult > 2 ? SHELL_ERR_NON_MANIFOLD : SHELL_ERR_BAD_ORIENTATION;
    }
  }
  auto find = [&](uint64_t key) -> const DirEdge * {
    auto it = std::lower_bound(de.begin(), de.end(), key, [](const DirEdge &x, uint64_t k) { return x.key < k; });
    return (it != de.end() && it->key == key) ? &*it : nullptr;
  };
  // twin[i]: index in de of the reverse of directed edge i (-1 on the boundary), found in the bucket of its
  // target vertex; at[3 t + k]: index in de of triangle t's edge k. Lookups of the hot loops below then cost
  // O(1) instead of a binary search over all directed edges.
  std::vector<int32_t> twin(de.size(), -1), at(de.size());
  for (size_t i = 0; i < de.size(); ++i) {
    const uint64_t p = de[i].key / N, q = de[i].key % N;
    const uint64_t rk = q * N + p;
    for (int j = out_ptr[q]; j < out_ptr[q + 1]; ++j)
      if (de[j].key == rk) {
        twin[i] = j;
        break;
      }
    const int32_t *v = tris + 3 * (size_t)de[i].tri;
    const int k = (v[0] == (int)p) ? 0 : (v[1] == (int)p) ? 1 : 2;
    at[3 * (size_t)de[i].tri + k] = (int32_t)i;
  }

  // ---- clamped boundary edges (undirected keys)
  std::vector<uint64_t> clamp_keys;
  for (int i = 0; i < n_clamped; ++i) {
    int a = clamped[2 * i], b = clamped[2 * i + 1];
    if (a < 0 || b < 0 || a >= nv || b >= nv || a == b) return SHELL_ERR_INVALID_ARG;
    const DirEdge *ab = find((uint64_t)a * N + b), *ba = find((uint64_t)b * N + a);
    if ((ab != nullptr) == (ba != nullptr)) return SHELL_ERR_INVALID_ARG;  // not a boundary edge
    clamp_keys.push_back((uint64_t)std::min(a, b) * N + std::max(a, b));
  }
  std::sort(clamp_keys.begin(), clamp_keys.end());
  auto is_clamped = [&](int a, int b) {
    uint64_t k = (uint64_t)std::min(a, b) * N + std::max(a, b);
    return std::binary_search(clamp_keys.begin(), clamp_keys.end(), k);
  };
  // neighbour across edge k (v[k] -> v[k+1]) of triangle t, and the hinge condition
  auto hinge = [&](int t, int k, int *nb) -> uint8_t {
    const int32_t tw = twin[at[3 * (size_t)t + k]];
    if (tw >= 0) { *nb = de[tw].opp; return 0; }
    *nb = -1;
    const int32_t *v = tris + 3 * (size_t)t;
    return is_clamped(v[k], v[(k + 1) % 3]) ? 2 : 1;
  };

  // ---- triangle stencils
  T.t_idx.assign((size_t)6 * nt, -1);
  T.t_bc.assign((size_t)3 * nt, 0);
  for (int t = 0; t < nt; ++t) {
    int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    int dummy;
    int r0 = 0;   // the rotation: edge r0 of the input triangle becomes edge 1-2
    for (int rot = 0; rot < 3; ++rot) {
      if (hinge(t, rot, &dummy) == 1) {
        int w[3] = {v[rot], v[(rot + 1) % 3], v[(rot + 2) % 3]};
        std::memcpy(v, w, sizeof(v));
        r0 = rot;
        break;
      }
    }
    // edges of the rotated triangle: 2-3, 3-1 and 1-2 are input edges r0 + 1, r0 + 2 and r0
    int n4, n5, n6;
    uint8_t c4 = hinge(t, (r0 + 1) % 3, &n4);
    uint8_t c5 = hinge(t, (r0 + 2) % 3, &n5);
    uint8_t c6 = hinge(t, r0, &n6);
    const int idx[6] = {v[0], v[1], v[2], n4, n5, n6};
    for (int j = 0; j < 6; ++j) T.t_idx[(size_t)j * nt + t] = idx[j];
    T.t_bc[(size_t)0 * nt + t] = c4;
    T.t_bc[(size_t)1 * nt + t] = c5;
    T.t_bc[(size_t)2 * nt + t] = c6;
  }

  // ---- edge stencils (edge-hinge models only): interior edges, then clamped boundary edges
  std::vector<int32_t> ei[4];
  if (edge_model) {
    for (size_t i = 0; i < de.size(); ++i) {
      const DirEdge &d = de[i];
      int p = (int)(d.key / N), q = (int)(d.key % N);
      if (p >= q) continue;
      if (twin[i] < 0) continue;
      ei[0].push_back(d.opp);
      ei[1].push_back(p);
      ei[2].push_back(q);
      ei[3].push_back(de[twin[i]].opp);
    }
    T.ne_int = (int)ei[0].size();
    for (size_t i = 0; i < de.size(); ++i) {
      const DirEdge &d = de[i];
      int p = (int)(d.key / N), q = (int)(d.key % N);
      if (twin[i] >= 0) continue;
      if (!is_clamped(p, q)) continue;
      ei[0].push_back(d.opp);
      ei[1].push_back(p);
      ei[2].push_back(q);
      ei[3].push_back(-1);
    }
  }
  T.ne = (int)ei[0].size();
  T.e_idx.resize((size_t)4 * T.ne);
  for (int j = 0; j < 4; ++j)
    for (int e = 0; e < T.ne; ++e) T.e_idx[(size_t)j * T.ne + e] = ei[j][e];

  // ---- contribution slots and the vertex incidence
  T.n_slots = nt * T.kt + T.ne * 4;
  auto slot_vertex = [&](int s) -> int {
    if (s < nt * T.kt) {
      int t = s / T.kt, j = s % T.kt;
      return T.t_idx[(size_t)j * nt + t];
    }
    int r = s - nt * T.kt;
    int e = r / 4, j = r % 4;
    return T.e_idx[(size_t)j * T.ne + e];
  };
  T.vtx_ptr.assign(nv + 1, 0);
  for (int s = 0; s < T.n_slots; ++s) {
    int v = slot_vertex(s);
    if (v >= 0) T.vtx_ptr[v + 1]++;
  }
  for (int i = 0; i < nv; ++i) T.vtx_ptr[i + 1] += T.vtx_ptr[i];
  T.vtx_slot.resize(T.vtx_ptr[nv]);
  {
    std::vector<int32_t> fill(T.vtx_ptr.begin(), T.vtx_ptr.end() - 1);
    for (int s = 0; s < T.n_slots; ++s) {
      int v = slot_vertex(s);
      if (v >= 0) T.vtx_slot[fill[v]++] = s;
    }
  }

  // ---- sparsity: every pair of vertices that share a bending stencil or a membrane triangle. A row's distinct
  // columns are collected with a marker array (mark[c] == i: c is already in row i), then only they are sorted.
  auto stencil_of_slot = [&](int s, int *verts) -> int {   // returns vertex count, fills verts
    if (s < nt * T.kt) {
      int t = s / T.kt;
      int k = edge_model ? 3 : 6;
      for (int j = 0; j < k; ++j) verts[j] = T.t_idx[(size_t)j * nt + t];
      return k;
    }
    int e = (s - nt * T.kt) / 4;
    for (int j = 0; j < 4; ++j) verts[j] = T.e_idx[(size_t)j * T.ne + e];
    return 4;
  };
  std::vector<int32_t> row_ptr(nv + 1, 0);
  std::vector<int32_t> cols;
  cols.reserve((size_t)nv * 20);
  std::vector<int32_t> tmp, mark(nv, -1);
  for (int i = 0; i < nv; ++i) {
    tmp.clear();
    tmp.push_back(i);
    mark[i] = i;
    for (int q = T.vtx_ptr[i]; q < T.vtx_ptr[i + 1]; ++q) {
      int verts[6];
      int k = stencil_of_slot(T.vtx_slot[q], verts);
      for (int j = 0; j < k; ++j)
        if (verts[j] >= 0 && mark[verts[j]] != i) {
          mark[verts[j]] = i;
          tmp.push_back(verts[j]);
        }
    }
    std::sort(tmp.begin(), tmp.end());
    cols.insert(cols.end(), tmp.begin(), tmp.end());
    row_ptr[i + 1] = (int32_t)cols.size();
  }
  T.nnz = (int64_t)cols.size();
  T.row_ptr = row_ptr;

  // ---- SELL-32 layout
  T.n_slices = (nv + 31) / 32;
  T.sl_ptr.assign(T.n_slices + 1, 0);
  for (int s = 0; s < T.n_slices; ++s) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      int r = s * 32 + l;
      if (r < nv) w = std::max(w, row_ptr[r + 1] - row_ptr[r]);
    }
    T.sl_ptr[s + 1] = T.sl_ptr[s] + 32 * w;
  }
  const int nnz_pad = T.sl_ptr[T.n_slices];
  T.sl_col.assign(nnz_pad, 0);
  T.diag_pos.assign(nv, -1);
  for (int s = 0; s < T.n_slices; ++s) {
    int w = (T.sl_ptr[s + 1] - T.sl_ptr[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      int r = s * 32 + l;
      for (int k = 0; k < w; ++k) {
        int pos = T.sl_ptr[s] + k * 32 + l;
        if (r < nv && k < row_ptr[r + 1] - row_ptr[r]) {
          int c = cols[row_ptr[r] + k];
          T.sl_col[pos] = c;
          if (c == r) T.diag_pos[r] = pos;
        } else {
          T.sl_col[pos] = (r < nv) ? r : 0;  // padding: own row, value 0
        }
      }
    }
  }
  // ---- assembly sources. Local matrix layout:
  //   triangle-stencil models: [nt][36] bending (L^T W L), then [nt][9] membrane
  //   edge-hinge models:       [nt][9] membrane, then [ne][16] bending (w L L^T)
  // Generated row by row from the row's slots, the SELL position of (r, c) from a column -> rank map of row r;
  // a first pass counts the entries of every position, a second fills them in. Per position the sources come
  // in increasing local index: the bending (triangle models) or membrane (edge models) entries of the row's
  // slots in slot order first, then the other kind in slot order.
  const int mem_off = edge_model ? 0 : nt * 36;
  const int edge_off = nt * 9;
  T.n_local = edge_model ? nt * 9 + T.ne * 16 : nt * 45;
  std::vector<int32_t> rank(nv, -1);
  auto row_entries = [&](int r, auto &&emit) {
    for (int k = row_ptr[r]; k < row_ptr[r + 1]; ++k) rank[cols[k]] = k - row_ptr[r];
    const int base = T.sl_ptr[r / 32] + r % 32;
    const int q0 = T.vtx_ptr[r], q1 = T.vtx_ptr[r + 1];
    for (int pass = 0; pass < 2; ++pass)
      for (int q = q0; q < q1; ++q) {
        const int sl = T.vtx_slot[q];
        if (sl < nt * T.kt) {
          const int t = sl / T.kt, j = sl % T.kt;
          if (!edge_model && pass == 0) {            // bending of the triangle stencil
            for (int k = 0; k < 6; ++k) {
              const int c = T.t_idx[(size_t)k * nt + t];
              if (c >= 0) emit(base + 32 * rank[c], t * 36 + j * 6 + k);
            }
          } else if ((edge_model ? pass == 0 : pass == 1) && j < 3) {   // membrane of the triangle
            for (int b = 0; b < 3; ++b) emit(base + 32 * rank[T.t_idx[(size_t)b * nt + t]], mem_off + t * 9 + j * 3 + b);
          }
        } else if (pass == 1) {                      // edge stencil (edge-hinge models)
          const int e = (sl - nt * T.kt) / 4, j = (sl - nt * T.kt) % 4;
          for (int k = 0; k < 4; ++k) {
            const int c = T.e_idx[(size_t)k * T.ne + e];
            if (c >= 0) emit(base + 32 * rank[c], edge_off + e * 16 + j * 4 + k);
          }
        }
      }
  };
  T.asm_ptr.assign(nnz_pad + 1, 0);
  for (int r = 0; r < nv; ++r) row_entries(r, [&](int pos, int) { T.asm_ptr[pos + 1]++; });
  for (int p = 0; p < nnz_pad; ++p) T.asm_ptr[p + 1] += T.asm_ptr[p];
  T.asm_src.resize(T.asm_ptr[nnz_pad]);
  {
    std::vector<int32_t> fill(T.asm_ptr.begin(), T.asm_ptr.end() - 1);
    for (int r = 0; r < nv; ++r) row_entries(r, [&](int pos, int local) { T.asm_src[fill[pos]++] = local; });
  }
  return SHELL_OK;
}

}  // namespace shl
