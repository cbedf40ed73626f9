// Work units of an in-place square transposition (2^a x 2^a matrix,
// 2^b x 2^b tiles, T = 2^(a-b) tiles per side): the tile pairs (tr, tc)
// with tr < tc and the diagonal tiles, in plain or blocked order.  Used by
// the transposition kernels and by the pipelined batched kernel.
#pragma once

#include <cstdint>

namespace brev {

// Tile pair q of a square 2^a x 2^a transposition in place with 2^b x 2^b
// tiles: pairs (tr, tc) with tr < tc, enumerated column by column
// (q = tc (tc - 1) / 2 + tr), then the diagonal tiles.
__device__ __forceinline__ void unrank_upper(uint32_t q, uint32_t& tr, uint32_t& tc) {
  uint32_t col = (uint32_t)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
  // correct a rounding step either way
  while ((uint64_t)col * (col - 1) / 2 > q) --col;
  while ((uint64_t)(col + 1) * col / 2 <= q) ++col;
  tc = col;
  tr = q - (uint32_t)((uint64_t)col * (col - 1) / 2);
}

// The same units in blocked order (T = tiles per side, a multiple of 8):
// 64 consecutive units cover an 8 x 8 block of tile pairs, so the tiles
// (tr, tc) and their partners (tc, tr) both come in runs of 8 adjacent
// tiles.  Off-diagonal blocks (bi < bj) first, 64 pairs each; then the
// diagonal blocks, 28 pairs (r < c inside the block) and 8 diagonal tiles
// each.
__device__ __forceinline__ int blocked_upper(uint32_t q, uint32_t T, uint32_t& tr,
                                             uint32_t& tc) {
  const uint32_t Tb = T >> 3;
  const uint64_t off = (uint64_t)Tb * (Tb - 1) / 2 * 64;
  if (q < off) {
    uint32_t bi, bj;
    unrank_upper(q >> 6, bi, bj);
    tr = (bi << 3) + ((q >> 3) & 7u);
    tc = (bj << 3) + (q & 7u);
    return 2;
  }
  const uint32_t q2 = (uint32_t)(q - off);
  const uint32_t blk = q2 / 36u, u = q2 - blk * 36u;
  if (u < 28u) {
    uint32_t r, c;
    unrank_upper(u, r, c);
    tr = (blk << 3) + r;
    tc = (blk << 3) + c;
    return 2;
  }
  tr = tc = (blk << 3) + (u - 28u);
  return 1;
}

}  // namespace brev
