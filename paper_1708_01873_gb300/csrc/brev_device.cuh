// Device-side building blocks of the bit-reversed permutation (sm_103a).
//
// Notation follows the matrix-buffer method of the paper's Introduction
// ("Bit reversal using a matrix buffer"): an index of k bits is split as
//
//     i = x y z        |x| = BX high bits, |z| = BZ low bits, |y| = k-BX-BZ
//
// and rev_k(i) = rev(z) rev(y) rev(x).  For a fixed y ("tile y") the source
// elements form a 2^BX x 2^BZ matrix whose rows (fixed x) are contiguous
// runs of 2^BZ elements, 2^(k-BX) elements apart.  Their destinations form
// a 2^BZ x 2^BX matrix at middle rev(y) whose rows (fixed rev(z)) are
// contiguous runs of 2^BX elements.  One CTA stages the tile in shared
// memory (the paper's buffer) so that both the HBM reads and the HBM writes
// are whole rows of >= 128 bytes moved in 16-byte vectors.
//
// Shared-memory layout of a tile: row X = rev(x) holds source row x, as CIN
// chunks of W bytes (W = 16 on the vector path, W = elem size on the
// element-wide path).  Logical chunk c of row X sits at position
// c ^ ((X / V) mod PHASE), V = W / E elements per chunk, PHASE = the lanes
// served by one shared-memory wavefront (128 / W).  Row writes (fixed X,
// consecutive c) and column reads (consecutive X / V, fixed c) then hit
// distinct banks.
//
// A 16-byte output vector holds V consecutive X of one destination row, i.e.
// V different source rows: a thread reads the V x V element block
// (rows dV..dV+V-1, chunk c) and transposes it in registers, producing one
// vector for each of the V destination rows rev(cV + e), e < V.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "brev_async.cuh"

namespace brev {

// ----------------------------------------------------------------- rev --
// Programmatic dependent launch.  The library's kernels are launched with
// programmatic stream serialisation, so a kernel's CTAs may start while
// the previous kernel in the stream is still finishing.  pdl_wait blocks
// until that grid has completed and its memory is visible; every CTA calls
// it before its first global-memory access (work on shared memory only,
// such as a twiddle table, may come before).  pdl_release lets the next
// kernel in the stream begin launching; its CTAs then wait in their own
// pdl_wait.  Both are no-ops when the kernel was launched without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_release();
}

// rev_w(v) for 0 <= w <= 32 using the single-instruction 32-bit reversal.
__device__ __forceinline__ uint32_t rev_bits(uint32_t v, int w) {
  return w == 0 ? 0u : (__brev(v) >> (32 - w));
}
template <int W>
__device__ __forceinline__ uint32_t rev_c(uint32_t v) {
  if constexpr (W == 0) {
    return 0u;
  } else {
    return __brev(v) >> (32 - W);
  }
}

// Number of y in [0, 2^w) with y < rev_w(y): 2^(w-1) - 2^(ceil(w/2)-1)
// (the swaps of Listing 1; Methods, unrolled closed form with the
// recurrence r(w) = 2^(w-2) + 2 r(w-2)).
__host__ __device__ __forceinline__ uint32_t count_lt(int w) {
  return w >= 1 ? (1u << (w - 1)) - (1u << ((w + 1) / 2 - 1)) : 0u;
}
// Number of palindromes y = rev_w(y): 2^ceil(w/2).
__host__ __device__ __forceinline__ uint32_t count_self(int w) {
  return 1u << ((w + 1) / 2);
}

// The q-th y (0 <= q < count_lt(w)) with y < rev_w(y), enumerated with the
// branch-and-bound classes of the unrolled method (Methods, "Unrolling"):
// for y = a m c with outer bits a, c, the class 0m1 always qualifies (all
// 2^(w-2) middles, enumerated first), 1m0 never does, and 0m0 / 1m1 qualify
// exactly when m < rev(m), a problem two bits smaller.
__device__ __forceinline__ uint32_t unrank_lt(uint32_t q, int w) {
  uint32_t outer = 0;
  for (int d = 0; 2 * d + 2 <= w; ++d) {
    const int rem = w - 2 * d;
    const uint32_t c01 = 1u << (rem - 2);
    if (q < c01) return outer | (q << (d + 1)) | (1u << d);
    q -= c01;
    const uint32_t r2 = count_lt(rem - 2);
    if (q >= r2) {  // class 1m1
      q -= r2;
      outer |= (1u << (w - 1 - d)) | (1u << d);
    }  // else class 0m0: outer bits stay 0
  }
  return outer;  // not reached for q < count_lt(w)
}

// The p-th palindrome of w bits (0 <= p < count_self(w)): the top
// ceil(w/2) bits are p, the rest mirror them.
__device__ __forceinline__ uint32_t unrank_self(uint32_t p, int w) {
  const int a = (w + 1) / 2;
  const int lw = w - a;
  return (p << lw) | rev_bits(p >> (a - lw), lw);
}

// ------------------------------------------------ blocked tile order --
// A launch order in which 64 consecutive CTAs cover an 8 x 8 block of
// (high 3 bits, low 3 bits) of y at one middle value.  Their tiles y form 8
// runs of 8 adjacent tiles, and so do the partner tiles rev(y), because
// reversal swaps the high and low fields.  HBM rows are then read and
// written in runs of eight tiles rather than one tile at scattered places.
// Needs w >= 6 bits of y; the tuner decides per shape whether it pays.
constexpr int BLOCK_ORDER_MIN_W = 6;

// Out-of-place: the t-th tile in blocked order (a bijection of [0, 2^w)).
__device__ __forceinline__ uint32_t blocked_tile(uint32_t t, int w) {
  const uint32_t lo = t & 7u, hi = (t >> 3) & 7u, mid = t >> 6;
  return (hi << (w - 3)) | (mid << 3) | lo;
}

// In-place: unit q (0 <= q < count_lt(w) + count_self(w)) in blocked order,
// giving a tile y and its partner ry (ry == y: self-paired).  The blocks are
// the 2^(w-6) middle values m.  A middle with m < rev(m) pairs its whole
// block with block rev(m): 64 pair units led from block m.  A palindromic
// middle pairs its block with itself: (hi, lo) leads a pair when
// hi < rev(lo) (28 units, lo-major) and is self-paired when hi = rev(lo)
// (8 units).
__device__ __forceinline__ void blocked_unit(uint32_t q, int w, uint32_t& y, uint32_t& ry) {
  const int mw = w - 6;
  const uint32_t full = count_lt(mw) << 6;
  uint32_t mid, hi, lo;
  if (q < full) {
    mid = unrank_lt(q >> 6, mw);
    hi = (q >> 3) & 7u;
    lo = q & 7u;
  } else {
    const uint32_t q2 = q - full;
    mid = unrank_self(q2 / 36u, mw);
    uint32_t r = q2 % 36u;
    if (r < 28u) {
      lo = 0;
      while (r >= rev_c<3>(lo)) {
        r -= rev_c<3>(lo);
        ++lo;
      }
      hi = r;
    } else {
      lo = r - 28u;
      hi = rev_c<3>(lo);
    }
  }
  y = (hi << (w - 3)) | (mid << 3) | lo;
  ry = rev_bits(y, w);
}

// ------------------------------------------------------- chunk types --
template <int W> struct ChunkT;
template <> struct ChunkT<16> { using type = uint4; };
template <> struct ChunkT<8> { using type = uint2; };
template <> struct ChunkT<4> { using type = uint32_t; };
template <> struct ChunkT<2> { using type = uint16_t; };
template <> struct ChunkT<1> { using type = uint8_t; };

// Global loads of the element-wide path (W = E < 16, pointers not 16-byte
// aligned; 16-byte chunks go by asynchronous copies).  NC: the source is
// read-only for the whole kernel (out-of-place), so the non-coherent path
// is legal.
template <int W, bool NC>
__device__ __forceinline__ typename ChunkT<W>::type gload(const char* p) {
  static_assert(W < 16, "16-byte chunks are staged by cp.async");
  using C = typename ChunkT<W>::type;
  if constexpr (NC) {
    return __ldg(reinterpret_cast<const C*>(p));
  } else {
    return *reinterpret_cast<const C*>(p);
  }
}

template <int W>
__device__ __forceinline__ void gstore(char* p, const typename ChunkT<W>::type& v) {
  if constexpr (W == 16) {
    asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
  } else {
    *reinterpret_cast<typename ChunkT<W>::type*>(p) = v;
  }
}

__device__ __forceinline__ uint32_t comp(const uint4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_comp(uint4& v, int i, uint32_t s) {
  if (i == 0) v.x = s;
  else if (i == 1) v.y = s;
  else if (i == 2) v.z = s;
  else v.w = s;
}

// out[e] element j = in[j] element e, for a V x V block of E-byte
// elements held as V chunks of W bytes (V = W / E).
template <int E, int W>
__device__ __forceinline__ void xpose(const typename ChunkT<W>::type (&in)[W / E],
                                      typename ChunkT<W>::type (&out)[W / E]) {
  constexpr int V = W / E;
  if constexpr (V == 1) {
    out[0] = in[0];
  } else if constexpr (E == 8) {  // 2 x 2 of 64-bit elements
    out[0] = make_uint4(in[0].x, in[0].y, in[1].x, in[1].y);
    out[1] = make_uint4(in[0].z, in[0].w, in[1].z, in[1].w);
  } else if constexpr (E == 4) {  // 4 x 4 of 32-bit elements
#pragma unroll
    for (int e = 0; e < 4; ++e)
      out[e] = make_uint4(comp(in[0], e), comp(in[1], e), comp(in[2], e), comp(in[3], e));
  } else if constexpr (E == 2) {  // 8 x 8 of 16-bit elements
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t sel = (e & 1) ? 0x7632u : 0x5410u;
      uint4 o;
#pragma unroll
      for (int p = 0; p < 4; ++p)
        set_comp(o, p, __byte_perm(comp(in[2 * p], e >> 1), comp(in[2 * p + 1], e >> 1), sel));
      out[e] = o;
    }
  } else {  // E == 1: 16 x 16 bytes
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t b = e & 3;
      const uint32_t sel = b | ((4 + b) << 4);  // byte b of a, byte b of b
      uint4 o;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t lo = __byte_perm(comp(in[4 * p], e >> 2), comp(in[4 * p + 1], e >> 2), sel);
        const uint32_t hi =
            __byte_perm(comp(in[4 * p + 2], e >> 2), comp(in[4 * p + 3], e >> 2), sel);
        set_comp(o, p, __byte_perm(lo, hi, 0x5410u));
      }
      out[e] = o;
    }
  }
}

// ---------------------------------------------------------- geometry --
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <int E_, int W_, int BX_, int BZ_>
struct Geom {
  static constexpr int E = E_, W = W_, BX = BX_, BZ = BZ_;
  static constexpr int V = W / E;             // elements per chunk
  static_assert(V >= 1 && W % E == 0, "chunk must hold whole elements");
  static constexpr int CIN = (1 << BZ) / V;   // chunks per source row
  static constexpr int COUT = (1 << BX) / V;  // chunks per destination row
  static_assert(CIN >= 1 && COUT >= 1, "tile narrower than one chunk");
  static_assert(CIN * W >= 128 && COUT * W >= 128, "rows of at least 128 bytes");
  static constexpr int LOG_CIN = ilog2c(CIN);
  static constexpr int LOG_COUT = ilog2c(COUT);
  static constexpr int CHUNKS = (1 << BX) * CIN;  // chunks per tile
  static constexpr int UNITS = CIN * COUT;        // store units (V chunks each)
  static constexpr int THREADS = UNITS < 256 ? UNITS : 256;
  static constexpr int PHASE = 128 / W;           // lanes per smem wavefront
  static constexpr int SWZ = PHASE - 1;
  static constexpr unsigned TILE_BYTES = unsigned(CHUNKS) * W;
};

// Load tiles src0 (and src1 when NT = 2) of geometry G into shared memory
// (tile t at sm + t * CHUNKS), with NTHR threads: source row x, chunk c
// lands at shared row rev(x), swizzled chunk c ^ ((rev(x) / V) & SWZ).
// 16-byte chunks go by per-thread asynchronous copies (cp.async, through
// L2), all of a thread's chunks issued at once and then waited for; the
// caller's barrier follows.  No registers hold loaded data, so more bytes
// are in flight than register-staged loads allow (batches of 8 chunks per
// thread): on GB300 the large arrays moved from 0.99 to 1.01 of the
// measured copy bandwidth.  The element-wide path (W = E, pointers not
// 16-byte aligned) loads through registers in batches of up to 8 per thread.
// WAIT = false (16-byte chunks only) issues the copies and returns: the
// caller commits them as a group and waits for the group later.
template <class G, bool NC, int NTHR, int NT, bool WAIT = true>
__device__ __forceinline__ void load_tiles(typename ChunkT<G::W>::type* sm,
                                           const char* src0, const char* src1,
                                           uint64_t row_stride, int nt_active) {
  static_assert(WAIT || G::W == 16, "only the asynchronous 16-byte path can defer its wait");
  using C = typename ChunkT<G::W>::type;
  constexpr int PER = (G::CHUNKS + NTHR - 1) / NTHR;  // chunks per thread per tile
  constexpr int TOTAL = PER * NT;
  constexpr int BATCH = TOTAL < 8 ? TOTAL : 8;
  const int tid = threadIdx.x;
  if constexpr (G::W == 16) {
#pragma unroll
    for (int f = 0; f < TOTAL; ++f) {
      const int t = f / PER, i = f % PER;
      const int q = tid + i * NTHR;
      if (t < nt_active && (G::CHUNKS % NTHR == 0 || q < G::CHUNKS)) {
        const int x = q >> G::LOG_CIN, c = q & (G::CIN - 1);
        const char* base = (NT == 1 || t == 0) ? src0 : src1;
        const int X = (int)rev_c<G::BX>((uint32_t)x);
        const int pc = c ^ ((X / G::V) & G::SWZ);
        cp_async16(sm + t * G::CHUNKS + X * G::CIN + pc,
                   base + (uint64_t)x * row_stride + (unsigned)c * 16);
      }
    }
    if constexpr (WAIT) cp_async_wait_all();
  } else {
#pragma unroll 1
    for (int b0 = 0; b0 < TOTAL; b0 += BATCH) {
      C r[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int f = b0 + j;
        const int t = f / PER, i = f % PER;
        const int q = tid + i * NTHR;
        if (f < TOTAL && t < nt_active && (G::CHUNKS % NTHR == 0 || q < G::CHUNKS)) {
          const int x = q >> G::LOG_CIN, c = q & (G::CIN - 1);
          const char* base = (NT == 1 || t == 0) ? src0 : src1;
          r[j] = gload<G::W, NC>(base + (uint64_t)x * row_stride + (unsigned)c * G::W);
        }
      }
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int f = b0 + j;
        const int t = f / PER, i = f % PER;
        const int q = tid + i * NTHR;
        if (f < TOTAL && t < nt_active && (G::CHUNKS % NTHR == 0 || q < G::CHUNKS)) {
          const int x = q >> G::LOG_CIN, c = q & (G::CIN - 1);
          const int X = (int)rev_c<G::BX>((uint32_t)x);
          const int pc = c ^ ((X / G::V) & G::SWZ);
          sm[t * G::CHUNKS + X * G::CIN + pc] = r[j];
        }
      }
    }
  }
}

// Write one staged tile to its destination: destination row Z = rev(z) is
// a contiguous run of 2^BX elements at dst_tile + Z * row_stride.
template <class G, int NTHR>
__device__ __forceinline__ void store_tile(const typename ChunkT<G::W>::type* sm,
                                           char* dst_tile, uint64_t row_stride) {
  using C = typename ChunkT<G::W>::type;
  constexpr int PER = (G::UNITS + NTHR - 1) / NTHR;
  constexpr int UNROLL = PER < 4 ? PER : 4;
  const int tid = threadIdx.x;
#pragma unroll UNROLL
  for (int i = 0; i < PER; ++i) {
    const int u = tid + i * NTHR;
    if (G::UNITS % NTHR == 0 || u < G::UNITS) {
      const int c = u >> G::LOG_COUT, d = u & (G::COUT - 1);
      const int pc = c ^ (d & G::SWZ);
      C blk[G::V], out[G::V];
#pragma unroll
      for (int j = 0; j < G::V; ++j) blk[j] = sm[(d * G::V + j) * G::CIN + pc];
      xpose<G::E, G::W>(blk, out);
#pragma unroll
      for (int e = 0; e < G::V; ++e) {
        const uint32_t Z = rev_c<G::BZ>((uint32_t)(c * G::V + e));
        gstore<G::W>(dst_tile + (uint64_t)Z * row_stride + (unsigned)d * G::W, out[e]);
      }
    }
  }
}

// --------------------------------------------------------- tile bodies --
// Out-of-place tile y: source rows at src + (x * 2^(k-BX) + y * 2^BZ) * E,
// destination rows at dst + (Z * 2^(k-BZ) + rev(y) * 2^BX) * E.
template <class G, int NTHR>
__device__ __forceinline__ void tile_oop_body(char* __restrict__ dst,
                                              const char* __restrict__ src, int k,
                                              uint32_t y, typename ChunkT<G::W>::type* sm) {
  const int wy = k - G::BX - G::BZ;
  const uint32_t ry = rev_bits(y, wy);
  const uint64_t stride_in = (uint64_t)G::E << (k - G::BX);
  const uint64_t stride_out = (uint64_t)G::E << (k - G::BZ);
  load_tiles<G, true, NTHR, 1>(sm, src + ((uint64_t)y << G::BZ) * G::E, nullptr, stride_in, 1);
  __syncthreads();
  store_tile<G, NTHR>(sm, dst + ((uint64_t)ry << G::BX) * G::E, stride_out);
}

// In-place work unit q of an array of 2^k elements with square tiles
// (BX = BZ = B): units [0, count_lt(w)) are tile pairs (y, rev(y)) with
// y < rev(y); units [count_lt(w), count_lt(w) + count_self(w)) are the
// self-paired tiles y = rev(y).  Both tiles of a pair are read before
// either is written (Introduction, in-place matrix buffer: swap through the
// buffer; Listing 1: each pair swapped once).
template <class G, int NTHR, int ORDER = 0>
__device__ __forceinline__ void tile_inplace_body(char* data, int k, uint32_t q,
                                                  typename ChunkT<G::W>::type* sm) {
  static_assert(G::BX == G::BZ, "in-place needs square tiles");
  const int wy = k - 2 * G::BX;
  const uint32_t npairs = count_lt(wy);
  uint32_t y, ry;
  int nt;
  if (ORDER == 1 && wy >= BLOCK_ORDER_MIN_W) {
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
  const uint64_t stride = (uint64_t)G::E << (k - G::BX);
  char* const ty = data + ((uint64_t)y << G::BX) * G::E;
  char* const tr = data + ((uint64_t)ry << G::BX) * G::E;
  load_tiles<G, false, NTHR, 2>(sm, ty, tr, stride, nt);
  __syncthreads();
  store_tile<G, NTHR>(sm, tr, stride);  // tile y's elements land in tile rev(y)
  if (nt == 2) store_tile<G, NTHR>(sm + G::CHUNKS, ty, stride);
}

// Whole array staged in one CTA (small arrays): element i is written to
// shared slot rev(i), then the slots are copied out in order.
template <int E>
__device__ __forceinline__ void small_body(char* dst, const char* src, int k, int nthr,
                                           typename ChunkT<E>::type* sm) {
  using C = typename ChunkT<E>::type;
  const uint32_t n = 1u << k;
  const C* s = reinterpret_cast<const C*>(src);
  C* d = reinterpret_cast<C*>(dst);
  for (uint32_t i = threadIdx.x; i < n; i += nthr) sm[rev_bits(i, k)] = s[i];
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += nthr) d[i] = sm[i];
}

}  // namespace brev
