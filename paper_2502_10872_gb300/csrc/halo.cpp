// halo.cpp -- per-block gather lists of a SELL matrix (see halo.h).
#include "halo.h"

#include <algorithm>

namespace shl {

bool build_halo(int n_rows, int n_cols, const std::vector<int32_t> &sl_ptr, const std::vector<int32_t> &sl_col,
                const std::vector<int32_t> &row_ptr, bool square, HostHalo *out, int lanes) {
  *out = HostHalo();
  if (n_rows <= 0 || n_cols <= 0 || (lanes != 1 && lanes != 4)) return false;
  const int rows_blk = kHaloBlock / lanes, rows_slice = 32 / lanes;
  // position of entry k of row r in the SELL layout
  auto pos_of = [&](int r, int k) {
    const int s = r / rows_slice, i = r % rows_slice;
    return sl_ptr[s] + 32 * (k / lanes) + lanes * i + k % lanes;
  };
  const int n_blocks = (n_rows + rows_blk - 1) / rows_blk;
  HostHalo H;
  std::vector<std::vector<int32_t>> lists(n_blocks);
  H.own.assign(n_blocks, 0);
  H.c16.assign(sl_col.size(), 0);
  // loc[c]: local index of column c in the current block's list, -1 outside it (reset after each block), so
  // the distinct columns are collected in one pass and only they are sorted
  std::vector<int32_t> loc(std::max(n_cols, n_rows), -1);
  std::vector<int32_t> list;
  auto mark = [&](int c) {
    if (loc[c] < 0) {
      loc[c] = 0;
      list.push_back(c);
    }
  };
  for (int b = 0; b < n_blocks; ++b) {
    const int r0 = b * rows_blk, r1 = std::min(n_rows, r0 + rows_blk);
    list.clear();
    for (int r = r0; r < r1; ++r) {
      const int len = row_ptr[r + 1] - row_ptr[r];
      for (int k = 0; k < len; ++k) mark(sl_col[pos_of(r, k)]);
      if (square) mark(r);
    }
    if (list.empty()) mark(0);
    std::sort(list.begin(), list.end());
    if (list.size() > 65535) return false;
    for (size_t i = 0; i < list.size(); ++i) loc[list[i]] = (int32_t)i;
    H.max = std::max(H.max, (int)list.size());
    const int own = square ? loc[r0] : 0;
    H.own[b] = own;
    for (int r = r0; r < r1; ++r) {
      const int s = r / rows_slice;
      const int len = row_ptr[r + 1] - row_ptr[r];
      const int w = (sl_ptr[s + 1] - sl_ptr[s]) / 32 * lanes;   // stored entries of the row, padding included
      for (int k = 0; k < w; ++k) {
        const int pos = pos_of(r, k);
        H.c16[pos] = (uint16_t)(k < len ? loc[sl_col[pos]] : (square ? own + (r - r0) : 0));
      }
    }
    for (int c : list) loc[c] = -1;
    lists[b] = list;
  }
  H.col.assign((size_t)n_blocks * H.max, 0);
  for (int b = 0; b < n_blocks; ++b)
    for (int k = 0; k < H.max; ++k)
      H.col[(size_t)b * H.max + k] = k < (int)lists[b].size() ? lists[b][k] : lists[b][0];
  *out = std::move(H);
  return true;
}

}  // namespace shl
