// Single-array kernels (one tile, tile pair or whole small array per CTA)
// and the macros that list them in per-element-size shape tables.
#pragma once

#include "brev_device.cuh"
#include "brev_internal.h"

namespace brev {

// Out-of-place: one CTA per tile (grid = 2^(k-BX-BZ)); ORDER 0 runs tile
// y = blockIdx.x, ORDER 1 the blocked order.
template <int E, int W, int BX, int BZ, int ORDER>
__global__ void __launch_bounds__(Geom<E, W, BX, BZ>::THREADS)
    k_tile_oop(char* __restrict__ dst, const char* __restrict__ src, int k) {
  using G = Geom<E, W, BX, BZ>;
  extern __shared__ uint4 smem_u4[];
  pdl_enter();
  const int wy = k - BX - BZ;
  const uint32_t y =
      (ORDER == 1 && wy >= BLOCK_ORDER_MIN_W) ? blocked_tile(blockIdx.x, wy) : blockIdx.x;
  tile_oop_body<G, G::THREADS>(dst, src, k, y,
                               reinterpret_cast<typename ChunkT<W>::type*>(smem_u4));
}

// In-place: CTA q runs unit q (tile pair or self-paired tile).
template <int E, int W, int B, int ORDER>
__global__ void __launch_bounds__(Geom<E, W, B, B>::THREADS)
    k_tile_inplace(char* data, int k) {
  using G = Geom<E, W, B, B>;
  extern __shared__ uint4 smem_u4[];
  pdl_enter();
  tile_inplace_body<G, G::THREADS, ORDER>(data, k, blockIdx.x,
                                          reinterpret_cast<typename ChunkT<W>::type*>(smem_u4));
}

// Small arrays: one CTA stages the whole array (dst may equal src).
template <int E>
__global__ void __launch_bounds__(256) k_small(char* dst, const char* src, int k) {
  extern __shared__ uint4 smem_u4[];
  pdl_enter();
  small_body<E>(dst, src, k, blockDim.x, reinterpret_cast<typename ChunkT<E>::type*>(smem_u4));
}

}  // namespace brev

#define BREV_OOP_O(E, W, BX, BZ, O)                                                    \
  ShapeEntry {                                                                          \
    E, W, BX, BZ, 0, O, (const void*)&k_tile_oop<E, W, BX, BZ, O>,                     \
        Geom<E, W, BX, BZ>::TILE_BYTES, Geom<E, W, BX, BZ>::THREADS                     \
  }
#define BREV_INP_O(E, W, B, O)                                                          \
  ShapeEntry {                                                                          \
    E, W, B, B, 1, O, (const void*)&k_tile_inplace<E, W, B, O>,                        \
        2u * Geom<E, W, B, B>::TILE_BYTES, Geom<E, W, B, B>::THREADS                    \
  }
// plain order only (element-wide path)
#define BREV_OOP(E, W, BX, BZ) BREV_OOP_O(E, W, BX, BZ, 0)
#define BREV_INP(E, W, B) BREV_INP_O(E, W, B, 0)
// both launch orders (16-byte path; the tuner picks)
#define BREV_OOP2(E, BX, BZ) BREV_OOP_O(E, 16, BX, BZ, 0), BREV_OOP_O(E, 16, BX, BZ, 1)
#define BREV_INP2(E, B) BREV_INP_O(E, 16, B, 0), BREV_INP_O(E, 16, B, 1)
