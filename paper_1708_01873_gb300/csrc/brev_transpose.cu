// Power-of-two matrix transpositions on the tile machinery, the even-odd
// (Stockham) step and the perfect shuffle as special cases, segmented
// bit reversal, and the paper's recursive method as a multi-pass ablation.
//
// Transposition of a row-major 2^a x 2^c matrix: dst[j 2^a + i] = src[i 2^c + j]
// (Introduction: the even-odd step is the n/2 x 2 transposition, the perfect
// shuffle its inverse).  Tile (tr, tc) holds rows [tr 2^bx, ...) and columns
// [tc 2^bz, ...); its 2^bx source rows are contiguous runs of 2^bz elements
// and its 2^bz destination rows contiguous runs of 2^bx elements, so the same
// staged load / swizzle / register transpose / store as the bit-reversal
// tiles applies with identity index maps.
#include <algorithm>
#include <cmath>

#include "brev_device.cuh"
#include "brev_device_rt.cuh"
#include "brev_internal.h"
#include "brev_trace.h"
#include "brev_transpose_units.cuh"

namespace brev {

constexpr int TR_THREADS = 256;

// Out-of-place: CTA t handles tile (t >> (c - bz), t & (2^(c-bz) - 1)).
template <int E, int W>
__global__ void __launch_bounds__(TR_THREADS)
    k_transpose(char* __restrict__ dst, const char* __restrict__ src, int a, int c, int bx,
                int bz) {
  extern __shared__ uint4 smem_u4[];
  auto* sm = reinterpret_cast<typename ChunkT<W>::type*>(smem_u4);
  pdl_enter();
  const int lc = c - bz;
  const uint64_t t = blockIdx.x;
  const uint64_t tr = t >> lc, tc = t & ((1ull << lc) - 1);
  const char* s = src + ((tr << (bx + c)) + (tc << bz)) * E;
  char* d = dst + ((tc << (bz + a)) + (tr << bx)) * E;
  load_tiles_g<E, W, TR_THREADS, true, false>(sm, s, nullptr, (uint64_t)E << c, 1, bx, bz);
  __syncthreads();
  store_tile_g<E, W, TR_THREADS, false>(sm, d, (uint64_t)E << a, bx, bz);
}

// Out-of-place transposition of a 2^bx x 2^c matrix (one tile row spans
// every row) whose source row x becomes destination column rev_bx(x):
// dst[j 2^bx + rev(x)] = src[x 2^c + j].  The last local pass of the
// permutation spread over 2^bx ranks (brev_dist_finish).
template <int E, int W>
__global__ void __launch_bounds__(TR_THREADS)
    k_transpose_rowrev(char* __restrict__ dst, const char* __restrict__ src, int c, int bx,
                       int bz) {
  extern __shared__ uint4 smem_u4[];
  auto* sm = reinterpret_cast<typename ChunkT<W>::type*>(smem_u4);
  pdl_enter();
  const uint64_t tc = blockIdx.x;
  const char* s = src + (tc << bz) * E;
  char* d = dst + (tc << (bz + bx)) * E;
  load_tiles_g<E, W, TR_THREADS, true, true>(sm, s, nullptr, (uint64_t)E << c, 1, bx, bz);
  __syncthreads();
  store_tile_g<E, W, TR_THREADS, false>(sm, d, (uint64_t)E << bx, bx, bz);
}

template <int E, int W>
__global__ void __launch_bounds__(TR_THREADS) k_transpose_inplace(char* data, int a, int b) {
  extern __shared__ uint4 smem_u4[];
  auto* sm = reinterpret_cast<typename ChunkT<W>::type*>(smem_u4);
  pdl_enter();
  const uint64_t T = 1ull << (a - b);
  const uint64_t npairs = T * (T - 1) / 2;
  const uint32_t q = blockIdx.x;
  uint32_t tr, tc;
  int nt;
  if (T >= 8) {
    nt = blocked_upper(q, (uint32_t)T, tr, tc);
  } else if (q < npairs) {
    unrank_upper(q, tr, tc);
    nt = 2;
  } else {
    tr = tc = (uint32_t)(q - npairs);
    nt = 1;
  }
  const uint64_t stride = (uint64_t)E << a;
  char* const A = data + (((uint64_t)tr << (b + a)) + ((uint64_t)tc << b)) * E;
  char* const B = data + (((uint64_t)tc << (b + a)) + ((uint64_t)tr << b)) * E;
  load_tiles_g<E, W, TR_THREADS, false, false>(sm, A, B, stride, nt, b, b);
  __syncthreads();
  store_tile_g<E, W, TR_THREADS, false>(sm, B, stride, b, b);  // tile (tr,tc) -> (tc,tr)
  constexpr int LOG_V = ilog2c(W / E);
  if (nt == 2) store_tile_g<E, W, TR_THREADS, false>(sm + (1 << (2 * b - LOG_V)), A, stride, b, b);
}

// Segmented in-place bit reversal: 2^s contiguous segments of 2^m elements,
// each permuted on its own.  CTA q runs unit q % units of segment q / units
// (square tiles of exponent b), or, with b = 0, stages segment q whole.
template <int E, int W>
__global__ void __launch_bounds__(TR_THREADS)
    k_segments(char* data, int m, int b, unsigned units) {
  extern __shared__ uint4 smem_u4[];
  auto* sm = reinterpret_cast<typename ChunkT<W>::type*>(smem_u4);
  pdl_enter();
  if (b == 0) {
    char* seg = data + ((uint64_t)blockIdx.x << m) * E;
    small_body<E>(seg, seg, m, TR_THREADS, reinterpret_cast<typename ChunkT<E>::type*>(sm));
    return;
  }
  const uint32_t seg_i = blockIdx.x / units, u = blockIdx.x - seg_i * units;
  char* seg = data + ((uint64_t)seg_i << m) * E;
  tile_inplace_body_rt<E, W, TR_THREADS>(seg, m, b, u, sm);
}

// ------------------------------------------------------------------ host --

struct TrKernels {
  const void* oop;
  const void* inplace;
  const void* seg;
  const void* rowrev;
};

template <int E, int W>
static TrKernels tr_kernels() {
  return {(const void*)&k_transpose<E, W>, (const void*)&k_transpose_inplace<E, W>,
          (const void*)&k_segments<E, W>, (const void*)&k_transpose_rowrev<E, W>};
}

static bool tr_lookup(int E, int W, TrKernels* out) {
  switch (E * 100 + W) {
    case 16 * 100 + 16: *out = tr_kernels<16, 16>(); return true;
    case 8 * 100 + 16: *out = tr_kernels<8, 16>(); return true;
    case 8 * 100 + 8: *out = tr_kernels<8, 8>(); return true;
    case 4 * 100 + 16: *out = tr_kernels<4, 16>(); return true;
    case 4 * 100 + 4: *out = tr_kernels<4, 4>(); return true;
    case 2 * 100 + 16: *out = tr_kernels<2, 16>(); return true;
    case 2 * 100 + 2: *out = tr_kernels<2, 2>(); return true;
    case 1 * 100 + 16: *out = tr_kernels<1, 16>(); return true;
    case 1 * 100 + 1: *out = tr_kernels<1, 1>(); return true;
  }
  return false;
}

static bool valid_E(int E) { return E == 1 || E == 2 || E == 4 || E == 8 || E == 16; }
static int ilog2i(int v) {
  int r = 0;
  while ((1 << (r + 1)) <= v) ++r;
  return r;
}
// Square tile exponent targeted per element size (tiles of 16-64 KiB).
static int target_b(int E) { return E == 16 ? 5 : E == 8 ? 5 : E == 4 ? 6 : E == 2 ? 7 : 8; }

static brev_status check_args(void* dst, const void* src, int log2_total, int E) {
  if (!valid_E(E)) return set_error(BREV_ERR_INVALID_ARG, "elem_bytes=%d", E);
  if (log2_total < 0 || log2_total > BREV_MAX_LOG2N)
    return set_error(BREV_ERR_INVALID_ARG, "log2 of the element count %d outside [0, %d]",
                     log2_total, BREV_MAX_LOG2N);
  if (!dst || !src) return set_error(BREV_ERR_INVALID_ARG, "NULL data pointer");
  if ((uintptr_t)dst % E || (uintptr_t)src % E)
    return set_error(BREV_ERR_ALIGNMENT, "pointers must be aligned to elem_bytes=%d", E);
  const uint64_t bytes = (uint64_t)E << log2_total;
  if (dst != src) {
    const uint64_t d = (uintptr_t)dst, s = (uintptr_t)src;
    if (d < s + bytes && s < d + bytes)
      return set_error(BREV_ERR_OVERLAP, "source and destination overlap partially");
  }
  brev_status st = check_device_range(src, bytes, "source");
  if (st == BREV_OK && dst != src) st = check_device_range(dst, bytes, "destination");
  return st;
}

static brev_status launch(const void* kern, unsigned long long grid, unsigned smem, void** args,
                          cudaStream_t stream, const char* what) {
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return cuda_error(e, "shared-memory limit");
  e = launch_pdl(kern, (unsigned)grid, TR_THREADS, args, smem, stream);
  if (e != cudaSuccess) return cuda_error(e, what);
  note_launch();
  return BREV_OK;
}

// Transposition without argument checks.
static brev_status transpose_launch(void* dst, const void* src, int a, int c, int E,
                                    cudaStream_t stream) {
  const bool vec16 = (((uintptr_t)dst | (uintptr_t)src) % 16) == 0;
  const int V = 16 / E, lv = ilog2i(V);
  const int B = target_b(E), T = 2 * B;
  TrKernels K;
  if (dst == src) {  // square, in place
    const int pb = transpose_pipelined_b(E);
    if (vec16 && pb > 0 && a >= pb) return transpose_inplace_pipelined(dst, a, E, stream);
    const int b = std::min(a, B);
    const int W = (vec16 && b >= lv) ? 16 : E;
    if (!tr_lookup(E, W, &K)) return set_error(BREV_ERR_UNSUPPORTED, "no kernel");
    if (a == 0) return BREV_OK;
    const unsigned long long Tn = 1ull << (a - b);
    const unsigned long long grid = Tn * (Tn - 1) / 2 + Tn;
    const unsigned smem = 2u * ((unsigned)E << (2 * b));
    char* p = (char*)dst;
    void* args[] = {(void*)&p, (void*)&a, (void*)&b};
    return launch(K.inplace, grid, smem, args, stream, "in-place transposition launch");
  }
  // tiles of about 2^T elements; narrow matrices get long thin tiles
  const int bz0 = std::min(c, B);
  int bx = std::min(a, T - bz0);
  int bz = std::min(c, T - bx);
  const int W = (vec16 && bx >= lv && bz >= lv) ? 16 : E;
  if (!tr_lookup(E, W, &K)) return set_error(BREV_ERR_UNSUPPORTED, "no kernel");
  const unsigned long long grid = 1ull << ((a - bx) + (c - bz));
  const unsigned smem = (unsigned)E << (bx + bz);
  char* d = (char*)dst;
  const char* s = (const char*)src;
  void* args[] = {(void*)&d, (void*)&s, (void*)&a, (void*)&c, (void*)&bx, (void*)&bz};
  return launch(K.oop, grid, smem, args, stream, "transposition launch");
}

// Transposition of a 2^g x 2^c matrix with source row x written to
// destination column rev_g(x), without argument checks; g <= the tile's
// row exponent (every tile spans all rows).
brev_status transpose_rowrev_launch(void* dst, const void* src, int g, int c, int E,
                                    cudaStream_t stream) {
  const bool vec16 = (((uintptr_t)dst | (uintptr_t)src) % 16) == 0;
  const int V = 16 / E, lv = ilog2i(V);
  const int B = target_b(E), T = 2 * B;
  if (g > B) return set_error(BREV_ERR_UNSUPPORTED, "2^%d rows exceed one tile", g);
  const int bz = std::min(c, T - g);
  const int W = (vec16 && g >= lv && bz >= lv) ? 16 : E;
  TrKernels K;
  if (!tr_lookup(E, W, &K)) return set_error(BREV_ERR_UNSUPPORTED, "no kernel");
  const unsigned long long grid = 1ull << (c - bz);
  const unsigned smem = (unsigned)E << (g + bz);
  char* d = (char*)dst;
  const char* s = (const char*)src;
  int gg = g;
  void* args[] = {(void*)&d, (void*)&s, (void*)&c, (void*)&gg, (void*)&bz};
  return launch(K.rowrev, grid, smem, args, stream, "row-reversed transposition launch");
}

int transpose_rowrev_max_g(int E) { return target_b(E); }

// Segmented bit reversal without argument checks: 2^s segments of 2^m.
static brev_status segments_launch(void* data, int s_log, int m, int E, cudaStream_t stream) {
  if (m <= 1) return BREV_OK;  // identity
  const bool vec16 = ((uintptr_t)data % 16) == 0;
  const int bmin = b_min_for(E);
  int b = m < 2 * bmin ? 0 : std::min(target_b(E) - (E <= 2 ? 1 : 0), m / 2);
  const int W = vec16 ? 16 : E;
  TrKernels K;
  if (!tr_lookup(E, W, &K)) return set_error(BREV_ERR_UNSUPPORTED, "no kernel");
  unsigned units = 1;
  unsigned smem;
  if (b == 0) {
    smem = (unsigned)E << m;
  } else {
    const int w = m - 2 * b;
    units = count_lt(w) + count_self(w);
    smem = 2u * ((unsigned)E << (2 * b));
  }
  const unsigned long long grid = (unsigned long long)units << s_log;
  if (grid > 0x7FFFFFFFull)
    return set_error(BREV_ERR_UNSUPPORTED, "too many work units for one launch");
  char* p = (char*)data;
  void* args[] = {(void*)&p, (void*)&m, (void*)&b, (void*)&units};
  return launch(K.seg, grid, smem, args, stream, "segmented bit-reversal launch");
}

}  // namespace brev

using namespace brev;

extern "C" {

brev_status brev_transpose(void* dst, const void* src, int log2_rows, int log2_cols,
                           int elem_bytes, void* stream) {
  BREV_TRACE("brev_transpose");
  if (log2_rows < 0 || log2_cols < 0)
    return set_error(BREV_ERR_INVALID_ARG, "log2_rows=%d log2_cols=%d", log2_rows, log2_cols);
  brev_status s = check_args(dst, src, log2_rows + log2_cols, elem_bytes);
  if (s != BREV_OK) return s;
  if (dst == src && log2_rows != log2_cols)
    return set_error(BREV_ERR_UNSUPPORTED,
                     "in-place transposition is supported for square matrices only");
  return transpose_launch(dst, src, log2_rows, log2_cols, elem_bytes, (cudaStream_t)stream);
}

brev_status brev_even_odd(void* dst, const void* src, int log2n, int elem_bytes, void* stream) {
  BREV_TRACE("brev_even_odd");
  if (log2n < 1) return brev_transpose(dst, src, 0, 0, elem_bytes, stream);
  return brev_transpose(dst, src, log2n - 1, 1, elem_bytes, stream);
}

brev_status brev_perfect_shuffle(void* dst, const void* src, int log2n, int elem_bytes,
                                 void* stream) {
  BREV_TRACE("brev_perfect_shuffle");
  if (log2n < 1) return brev_transpose(dst, src, 0, 0, elem_bytes, stream);
  return brev_transpose(dst, src, 1, log2n - 1, elem_bytes, stream);
}

brev_status brev_permute_segments(void* data, int log2_segments, int log2_seglen, int elem_bytes,
                                  void* stream) {
  BREV_TRACE("brev_permute_segments");
  if (log2_segments < 0 || log2_seglen < 0)
    return set_error(BREV_ERR_INVALID_ARG, "log2_segments=%d log2_seglen=%d", log2_segments,
                     log2_seglen);
  brev_status s = check_args(data, data, log2_segments + log2_seglen, elem_bytes);
  if (s != BREV_OK) return s;
  return segments_launch(data, log2_segments, log2_seglen, elem_bytes, (cudaStream_t)stream);
}

brev_status brev_permute_recursive(void* data, int log2n, int elem_bytes, void* stream) {
  BREV_TRACE("brev_permute_recursive");
  brev_status s = check_args(data, data, log2n, elem_bytes);
  if (s != BREV_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int k = log2n, E = elem_bytes;
  if (k <= 1) return BREV_OK;
  if (k % 2 == 0) {
    // x y -> x rev(y) -> rev(y) x -> rev(y) rev(x)
    const int h = k / 2;
    s = segments_launch(data, h, h, E, st);
    if (s == BREV_OK) s = transpose_launch(data, data, h, h, E, st);
    if (s == BREV_OK) s = segments_launch(data, h, h, E, st);
    return s;
  }
  // odd k: index x y z with z one bit; the even-odd step gives z x y, then
  // each half takes the (k-1)-bit permutation (x y -> rev(y) rev(x))
  const uint64_t bytes = (uint64_t)E << k;
  void* ws = nullptr;
  cudaError_t e = ws_alloc(&ws, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "even-odd workspace: %s", cudaGetErrorString(e));
  }
  s = transpose_launch(ws, data, k - 1, 1, E, st);
  const int h = (k - 1) / 2;
  for (int half = 0; half < 2 && s == BREV_OK; ++half) {
    char* p = (char*)ws + (uint64_t)half * (bytes / 2);
    s = segments_launch(p, h, h, E, st);
    if (s == BREV_OK) s = transpose_launch(p, p, h, h, E, st);
    if (s == BREV_OK) s = segments_launch(p, h, h, E, st);
  }
  if (s == BREV_OK) {
    e = cudaMemcpyAsync(data, ws, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = cuda_error(e, "copy back");
  }
  ws_free(ws, st);
  return s;
}

}  // extern "C"
