// Single-array kernels (one tile, tile pair or whole small array per CTA)
// and the macros that list them in per-element-size shape tables.
#pragma once

#include "brev_device.cuh"
#include "brev_internal.h"

namespace brev {

// Out-of-place: CTA y permutes tile y (grid = 2^(k-BX-BZ)).
template <int E, int W, int BX, int BZ>
__global__ void __launch_bounds__(Geom<E, W, BX, BZ>::THREADS)
    k_tile_oop(char* __restrict__ dst, const char* __restrict__ src, int k) {
  using G = Geom<E, W, BX, BZ>;
  extern __shared__ uint4 smem_u4[];
  tile_oop_body<G, G::THREADS>(dst, src, k, blockIdx.x,
                               reinterpret_cast<typename ChunkT<W>::type*>(smem_u4));
}

// In-place: CTA q runs unit q (tile pair or self-paired tile).
template <int E, int W, int B>
__global__ void __launch_bounds__(Geom<E, W, B, B>::THREADS)
    k_tile_inplace(char* data, int k) {
  using G = Geom<E, W, B, B>;
  extern __shared__ uint4 smem_u4[];
  tile_inplace_body<G, G::THREADS>(data, k, blockIdx.x,
                                   reinterpret_cast<typename ChunkT<W>::type*>(smem_u4));
}

// Small arrays: one CTA stages the whole array (dst may equal src).
template <int E>
__global__ void __launch_bounds__(256) k_small(char* dst, const char* src, int k) {
  extern __shared__ uint4 smem_u4[];
  small_body<E>(dst, src, k, blockDim.x, reinterpret_cast<typename ChunkT<E>::type*>(smem_u4));
}

}  // namespace brev

#define BREV_OOP(E, W, BX, BZ)                                                         \
  ShapeEntry {                                                                          \
    E, W, BX, BZ, 0, (const void*)&k_tile_oop<E, W, BX, BZ>,                           \
        Geom<E, W, BX, BZ>::TILE_BYTES, Geom<E, W, BX, BZ>::THREADS                     \
  }
#define BREV_INP(E, W, B)                                                               \
  ShapeEntry {                                                                          \
    E, W, B, B, 1, (const void*)&k_tile_inplace<E, W, B>, 2u * Geom<E, W, B, B>::TILE_BYTES, \
        Geom<E, W, B, B>::THREADS                                                       \
  }
