// halo.h -- per-block gather lists of a SELL matrix, for products that stage the gathered vector in
// shared memory (host, once per matrix).
//
// Block b is the rows one CTA processes together: 256 (one lane per row) or 64 (four lanes per row). Its list holds, in
// ascending order, every column that a stored (non-padding) entry of those rows references; for a square
// matrix also each of its own rows. Lists are stored at a fixed stride (the longest list), padded with
// their first entry, so a block's list starts at b * max without a lookup. A product over the block first copies the vector entries of the list
// into shared memory, then reads every gathered value from there through a 16-bit local index per stored
// entry. Padding entries get the local index of their own row (square) or 0 (value 0 either way).
#pragma once
#include <cstdint>
#include <vector>

namespace shl {

constexpr int kHaloBlock = 256;   // rows per block (the CTA size of the solve kernel)

struct HostHalo {
  std::vector<int32_t> col;       // [n_blocks][max] lists, padded
  std::vector<int32_t> own;       // [n_blocks] local index of the block's first row (square matrices)
  std::vector<uint16_t> c16;      // [nnz_pad] local index of every stored entry
  int max = 0;                    // longest list
};

// row_ptr: CSR row offsets of the matrix (row r has row_ptr[r+1] - row_ptr[r] stored entries, the first ones
// of its SELL row). lanes: lanes per row of the SELL layout (1: SELL-32, slices of 32 rows, 256-row blocks;
// 4: slices of 8 rows with 4 lanes each, 64-row blocks). Returns false (out left empty) if a list would not
// fit 16-bit local indices.
bool build_halo(int n_rows, int n_cols, const std::vector<int32_t> &sl_ptr, const std::vector<int32_t> &sl_col,
                const std::vector<int32_t> &row_ptr, bool square, HostHalo *out, int lanes = 1);

}  // namespace shl
