// Runtime-geometry tile bodies (tile exponents known only at run time),
// for kernels that meet many tile sizes in one launch (the batched kernel)
// or narrow matrices (transpositions).  Same layout, swizzle and register
// transpose as the compile-time bodies in brev_device.cuh.
#pragma once

#include "brev_device.cuh"

namespace brev {

// ------------------------------------------- runtime-geometry bodies --
// A 2^bx x 2^bz tile with both exponents run-time values, for kernels that
// meet many tile sizes in one launch (the batched kernel) or whose matrices
// may be narrow (transpositions).  Access width W: 16-byte vectors (V = 16/E
// elements per chunk; needs 2^bx, 2^bz >= V) or one element (W = E).  REV
// selects the bit-reversed index maps (rev(x) into shared memory, rev(z) out
// of it) or the identity ones (a plain matrix transposition).  Same layout
// and swizzle as Geom; rows may be narrower than 128 bytes, so the swizzle
// mask is clipped to the row width.
#ifndef BREV_RT_BATCH
#define BREV_RT_BATCH 4
#endif
constexpr int RT_BATCH = BREV_RT_BATCH;  // loads in flight per thread per batch

template <int E, int W, int NTHR, bool NC, bool REV>
__device__ __forceinline__ void load_tiles_g(typename ChunkT<W>::type* sm, const char* src0,
                                             const char* src1, uint64_t row_stride, int nt,
                                             int bx, int bz) {
  using C = typename ChunkT<W>::type;
  constexpr int V = W / E;
  constexpr int LOG_V = ilog2c(V);
  constexpr int PHASE = 128 / W;
  const int log_cin = bz - LOG_V;
  const int cin = 1 << log_cin;
  const int mask = (cin < PHASE ? cin : PHASE) - 1;
  const int chunks = 1 << (bx + log_cin);
  const int per = chunks >= NTHR ? chunks / NTHR : 1;
  const int total = per * nt;
  const int tid = threadIdx.x;
  if constexpr (W == 16) {
#pragma unroll 1
    for (int f = 0; f < total; ++f) {
      const int t = f / per, i = f - t * per;
      const int q = tid + i * NTHR;
      if (q < chunks) {
        const int x = q >> log_cin, c = q & (cin - 1);
        const int X = REV ? (int)rev_bits((uint32_t)x, bx) : x;
        const int pc = c ^ ((X >> LOG_V) & mask);
        cp_async16(sm + t * chunks + (X << log_cin) + pc,
                   (t == 0 ? src0 : src1) + (uint64_t)x * row_stride + (unsigned)c * 16);
      }
    }
    cp_async_wait_all();
  } else {
#pragma unroll 1
    for (int b0 = 0; b0 < total; b0 += RT_BATCH) {
      C r[RT_BATCH];
#pragma unroll
      for (int j = 0; j < RT_BATCH; ++j) {
        const int f = b0 + j;
        const int t = f / per, i = f - t * per;
        const int q = tid + i * NTHR;
        if (f < total && q < chunks) {
          const int x = q >> log_cin, c = q & (cin - 1);
          r[j] = gload<W, NC>((t == 0 ? src0 : src1) + (uint64_t)x * row_stride +
                              (unsigned)c * W);
        }
      }
#pragma unroll
      for (int j = 0; j < RT_BATCH; ++j) {
        const int f = b0 + j;
        const int t = f / per, i = f - t * per;
        const int q = tid + i * NTHR;
        if (f < total && q < chunks) {
          const int x = q >> log_cin, c = q & (cin - 1);
          const int X = REV ? (int)rev_bits((uint32_t)x, bx) : x;
          const int pc = c ^ ((X >> LOG_V) & mask);
          sm[t * chunks + (X << log_cin) + pc] = r[j];
        }
      }
    }
  }
}

template <int E, int W, int NTHR, bool REV>
__device__ __forceinline__ void store_tile_g(const typename ChunkT<W>::type* sm, char* dst_tile,
                                             uint64_t row_stride, int bx, int bz) {
  using C = typename ChunkT<W>::type;
  constexpr int V = W / E;
  constexpr int LOG_V = ilog2c(V);
  constexpr int PHASE = 128 / W;
  const int log_cin = bz - LOG_V;
  const int log_cout = bx - LOG_V;
  const int cin = 1 << log_cin;
  const int mask = (cin < PHASE ? cin : PHASE) - 1;
  const int units = 1 << (log_cin + log_cout);
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int u = tid; u < units; u += NTHR) {
    const int c = u >> log_cout, d = u & ((1 << log_cout) - 1);
    const int pc = c ^ (d & mask);
    C blk[V], out[V];
#pragma unroll
    for (int j = 0; j < V; ++j) blk[j] = sm[((d * V + j) << log_cin) + pc];
    xpose<E, W>(blk, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const uint32_t z = (uint32_t)(c * V + e);
      const uint32_t Z = REV ? rev_bits(z, bz) : z;
      gstore<W>(dst_tile + (uint64_t)Z * row_stride + (unsigned)d * W, out[e]);
    }
  }
}

// In-place unit q of a 2^k-element array with square tiles of runtime b
// (pairs first, then self-paired tiles; as tile_inplace_body).
template <int E, int W, int NTHR>
__device__ __forceinline__ void tile_inplace_body_rt(char* data, int k, int b, uint32_t q,
                                                     typename ChunkT<W>::type* sm,
                                                     int order = 0) {
  const int wy = k - 2 * b;
  const uint32_t npairs = count_lt(wy);
  uint32_t y, ry;
  int nt;
  if (order == 1 && wy >= BLOCK_ORDER_MIN_W) {
    blocked_unit(q, wy, y, ry);
    nt = y == ry ? 1 : 2;
  } else if (q < npairs) {
    y = unrank_lt(q, wy);
    ry = rev_bits(y, wy);
    nt = 2;
  } else {
    y = unrank_self(q - npairs, wy);
    ry = y;
    nt = 1;
  }
  const uint64_t stride = (uint64_t)E << (k - b);
  char* const ty = data + ((uint64_t)y << b) * E;
  char* const tr = data + ((uint64_t)ry << b) * E;
  load_tiles_g<E, W, NTHR, false, true>(sm, ty, tr, stride, nt, b, b);
  __syncthreads();
  store_tile_g<E, W, NTHR, true>(sm, tr, stride, b, b);
  constexpr int LOG_V = ilog2c(W / E);
  if (nt == 2) store_tile_g<E, W, NTHR, true>(sm + (1 << (2 * b - LOG_V)), ty, stride, b, b);
}

}  // namespace brev
