// Bit-reversed permutation fused with the first S radix-2 decimation-in-time
// FFT stages, for complex<float> (E = 8, float arithmetic) and
// complex<double> (E = 16, double arithmetic).
//
// The paper's motivation (Introduction): once the bit-reversed permutation
// has been applied, each level of the Cooley-Tukey recursion finds its
// even-odd split done, so the FFT proper is a sequence of butterfly stages
// over contiguous blocks.  Stage s combines, in every block of m = 2^s
// consecutive elements, a[j] and a[j + m/2] with w = exp(-2 pi i j / m).
// The tile kernel's output rows are contiguous runs of 2^B elements aligned
// to 2^B, so the first S <= B stages act inside one output row: after the
// tile is staged and transposed in shared memory (output row rev(z) is
// shared-memory column z), the butterflies run there and the tile is stored
// once -- the permutation and S stages in a single HBM round trip instead of
// one pass for the permutation and another for the stages.
#include <algorithm>

#include "brev_device.cuh"
#include "brev_internal.h"
#include "brev_trace.h"

namespace brev {

#ifndef BREV_FFT_IP_THREADS_MULT
#define BREV_FFT_IP_THREADS_MULT 1  // in-place CTA threads vs the out-of-place CTA (x2 spilled)
#endif
#ifndef BREV_FFT_MIN_CTAS
#define BREV_FFT_MIN_CTAS 6  // register budget for 6 resident CTAs per SM (measured best)
#endif

template <int E> struct Cplx;
template <> struct Cplx<8> { using T = float2; using R = float; };
template <> struct Cplx<16> { using T = double2; using R = double; };

// Element (X, z) of a staged tile (row X = rev(x), column z).
template <class G>
__device__ __forceinline__ typename Cplx<G::E>::T* tile_elem(uint4* sm, int X, int z) {
  constexpr int LOG_V = ilog2c(G::V);
  const int chunk = X * G::CIN + ((z >> LOG_V) ^ ((X >> LOG_V) & G::SWZ));
  return reinterpret_cast<typename Cplx<G::E>::T*>(sm + chunk) + (z & (G::V - 1));
}

// Twiddles w_{2^B}^i = exp(-2 pi i i / 2^B), i < 2^(B-1), into shared memory.
template <int E, int B>
__device__ __forceinline__ void fill_twiddles(typename Cplx<E>::T* tw) {
  using R = typename Cplx<E>::R;
  for (int i = threadIdx.x; i < (1 << (B - 1)); i += blockDim.x) {
    double sn, cs;
    sincospi((double)i / (double)(1 << (B - 1)), &sn, &cs);
    tw[i].x = (R)cs;
    tw[i].y = (R)(-sn);
  }
}

__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }

// x with its sign bit XORed with bit 31 of m (m = 0 or 0x80000000): an
// integer operation, so that conjugating costs no floating-point issue slot.
__device__ __forceinline__ float flip_sign(float x, uint32_t m) {
  return __uint_as_float(__float_as_uint(x) ^ m);
}
__device__ __forceinline__ double flip_sign(double x, uint32_t m) {
  return __hiloint2double(__double2hiint(x) ^ (int)m, __double2loint(x));
}

// a' = a + w b, b' = a - w b.  In double precision a' takes two fused
// multiply-adds per component (a.x - b.y w.y + b.x w.x, a.y + b.y w.x +
// b.x w.y) and b' one more, as 2a - a': six operations, against eight for
// the complex product followed by a sum and a difference.  This is the
// standard rewrite of the radix-2 butterfly for multiply-add units.  The FP64
// issue rate bounds the complex<double> stages, so the operation count is
// the time.  Each component of a' is rounded twice (at most about 1 ulp of
// |a| + |b|) and b' once more, so the per-stage error stays within that of
// the plain form.  complex<float> keeps the plain form: its stages are
// latency-bound, not FP32-bound, and the plain form holds the 5-CTA
// register budget without spilling.
template <class T>
__device__ __forceinline__ void butterfly(T& a, T& b, T w) {
  using R = decltype(a.x);
  if constexpr (sizeof(R) == 8) {
    const R px = fmad(b.x, w.x, fmad(-b.y, w.y, a.x));
    const R py = fmad(b.x, w.y, fmad(b.y, w.x, a.y));
    b.x = fmad(R(2), a.x, -px);
    b.y = fmad(R(2), a.y, -py);
    a.x = px;
    a.y = py;
  } else {
    T t;
    t.x = b.x * w.x - b.y * w.y;
    t.y = b.x * w.y + b.y * w.x;
    b.x = a.x - t.x;
    b.y = a.y - t.y;
    a.x = a.x + t.x;
    a.y = a.y + t.y;
  }
}

// The forward butterfly of stage S with twiddle w = exp(-2 pi i JJ / 2^S)
// known at compile time (S <= 3): w = 1 and the quarter turn w = -i need
// only a sum and a difference; the eighth turns of stage 3 (JJ = 1, 3) are
// (+-1 - i)/sqrt 2, i.e. w b = sqrt(1/2) (s, d) or sqrt(1/2) (d, -s) with
// s = b.x + b.y, d = b.y - b.x, which two additions and the multiply-add
// form above finish.
template <class T, int S, int JJ>
__device__ __forceinline__ void butterfly_const(T& a, T& b) {
  using R = decltype(a.x);
  static_assert(S >= 1 && S <= 3 && JJ >= 0 && 2 * JJ < (1 << S), "first-pass twiddle");
  if constexpr (JJ == 0) {
    const T t = b;
    b.x = a.x - t.x;
    b.y = a.y - t.y;
    a.x = a.x + t.x;
    a.y = a.y + t.y;
  } else if constexpr (2 * JJ == (1 << (S - 1))) {  // a quarter turn: -i b = (b.y, -b.x)
    const T t = b;
    b.x = a.x - t.y;
    b.y = a.y + t.x;
    a.x = a.x + t.y;
    a.y = a.y - t.x;
  } else {  // an eighth turn (S == 3, JJ odd)
    const R c = R(0.70710678118654752440);  // sqrt(1/2)
    const R s = b.x + b.y, d = b.y - b.x;
    const R re = JJ == 1 ? s : d, im = JJ == 1 ? d : -s;  // (w b) / sqrt(1/2)
    const R px = fmad(c, re, a.x);
    const R py = fmad(c, im, a.y);
    b.x = fmad(R(2), a.x, -px);
    b.y = fmad(R(2), a.y, -py);
    a.x = px;
    a.y = py;
  }
}

// Stages 1..R (R <= 3) of every output row, in registers, with the
// twiddles resolved at compile time (groups are 2^R consecutive elements).
// Imaginary parts have their sign flipped by conj_in on loading and by
// conj_out on storing.
template <class G, int NTHR, int R>
__device__ __forceinline__ void dit_first_pass(uint4* sm0, int nt, uint32_t conj_in,
                                               uint32_t conj_out) {
  using T = typename Cplx<G::E>::T;
  constexpr int GN = 1 << R;
  constexpr int LOG_GROUPS = G::BX + G::BZ - R;  // groups per tile
  for (int gt = threadIdx.x; gt < (nt << LOG_GROUPS); gt += NTHR) {
    uint4* sm = sm0 + (gt >> LOG_GROUPS) * G::CHUNKS;  // the nt staged tiles, one after another
    const int g = gt & ((1 << LOG_GROUPS) - 1);
    const int z = g & ((1 << G::BZ) - 1);
    const int base = (g >> G::BZ) << R;
    T v[GN];
#pragma unroll
    for (int t = 0; t < GN; ++t) {
      v[t] = *tile_elem<G>(sm, base + t, z);
      v[t].y = flip_sign(v[t].y, conj_in);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int t = 0; t < GN; ++t) {
        if (t & (1 << r)) continue;
        T& a = v[t];
        T& b = v[t + (1 << r)];
        // stage s = r + 1: jj = t mod 2^r
        if (r == 0) butterfly_const<T, 1, 0>(a, b);
        else if (r == 1) {
          if ((t & 1) == 0) butterfly_const<T, 2, 0>(a, b);
          else butterfly_const<T, 2, 1>(a, b);
        } else {
          switch (t & 3) {
            case 0: butterfly_const<T, 3, 0>(a, b); break;
            case 1: butterfly_const<T, 3, 1>(a, b); break;
            case 2: butterfly_const<T, 3, 2>(a, b); break;
            default: butterfly_const<T, 3, 3>(a, b); break;
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < GN; ++t) {
      v[t].y = flip_sign(v[t].y, conj_out);
      *tile_elem<G>(sm, base + t, z) = v[t];
    }
  }
}

// The butterflies of one group of the second pass, v holding the elements
// X = base + j + t 2^S0 (t < 2^R) of one output row: stage s = S0 + r + 1
// pairs t and t + 2^r with w = exp(-2 pi i jj / 2^s), jj = (j + t 2^S0) mod
// 2^(s-1).  For a group whose j is known at compile time (J >= 0) every
// twiddle that is a whole number of eighth turns (8 jj divisible by 2^s)
// takes butterfly_const's form -- w = 1 and -i need no product -- and the
// others the table; J = -1 reads every twiddle from the table.
template <class G, int R, int S0, int J, class T>
__device__ __forceinline__ void dit_group(T* v, int j, const T* tw) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int s = S0 + r + 1;
    const int hmask = (1 << (s - 1)) - 1;
#pragma unroll
    for (int t = 0; t < (1 << R); ++t) {
      if (t & (1 << r)) continue;
      T& a = v[t];
      T& b = v[t + (1 << r)];
      if constexpr (J >= 0) {
        const int jc = (J + (t << S0)) & hmask;  // folds to a constant once unrolled
        if (((jc << 3) & ((1 << s) - 1)) == 0) {
          switch ((jc << 3) >> s) {  // eighth turns
            case 0: butterfly_const<T, 3, 0>(a, b); break;
            case 1: butterfly_const<T, 3, 1>(a, b); break;
            case 2: butterfly_const<T, 3, 2>(a, b); break;
            default: butterfly_const<T, 3, 3>(a, b); break;
          }
          continue;
        }
      }
      const int jj = (j + (t << S0)) & hmask;
      butterfly(a, b, tw[jj << (G::BX - s)]);
    }
  }
}

// Stages 4 and 5 of a complex<double> group v[t] = X(base + j + 8 t),
// t < 4, j in {1, 2, 3, 5, 6, 7}, in 22 fused multiply-adds instead of the
// 24 of four multiply-add butterflies.  With w = exp(-2 pi i j / 32), stage
// 4 pairs (v0, v1) and (v2, v3) with w^2 and stage 5 pairs the results
// (A, C) with w and (B, D) with -i w, so
//   A, B = v0 +- w^2 v1,   w C, w D = w v2 +- w^3 v3,
//   out0, out2 = A +- w C,   out1, out3 = B -+ i w D.
// Writing w^m = c_m (1 + i t_m) (t_m = tan, c_m = cos of the angle m j pi / 16):
// u = (1 + i t2) v1 and p2 = (1 + i t1) v2, p3 = (1 + i t3) v3 take two
// operations each; A, B = v0 +- c2 u, q+- = p2 +- (c3 / c1) p3 and the
// outputs A +- c1 q+, B -+ i c1 q- two each, the factor c1 of w C = c1 q+ and
// w D = c1 q- folding into the last multiply-adds (the multiply-add form of
// the radix-4 butterfly).  Every c_m is nonzero for these j.  A tangent
// product is rounded relative to a value at most (1 + |t|) times its input
// and is then scaled by |c| = 1 / sqrt(1 + t^2), so each error stays within
// about sqrt(2) ulp of the inputs' magnitude, as in the plain butterfly.
// kRadix4Fma[j] = {t1, t2, t3, c1, c2, c3 / c1}, each the double nearest the
// exact value (rows 0 and 4 are unused: those groups take compile-time
// twiddles).  The index j is the same for a warp's 32 lanes, so the table is
// read by broadcast.
__constant__ double kRadix4Fma[8][6] = {
    {0, 0, 0, 0, 0, 0},
    {-0.198912367379658, -0.41421356237309503, -0.6681786379192989, 0.9807852804032304,
     0.9238795325112867, 0.8477590650225735},
    {-0.41421356237309503, -1.0, -2.414213562373095, 0.9238795325112867, 0.7071067811865476,
     0.41421356237309503},
    {-0.6681786379192989, -2.414213562373095, 5.027339492125848, 0.8314696123025452,
     0.3826834323650898, -0.23463313526982046},
    {0, 0, 0, 0, 0, 0},
    {-1.496605762665489, 2.414213562373095, 0.198912367379658, 0.5555702330196022,
     -0.3826834323650898, -1.7653668647301795},
    {-2.414213562373095, 1.0, -0.41421356237309503, 0.3826834323650898, -0.7071067811865476,
     -2.414213562373095},
    {-5.027339492125848, 0.41421356237309503, -1.496605762665489, 0.19509032201612828,
     -0.9238795325112867, -2.8477590650225735},
};

__device__ __forceinline__ void radix4_fma(double2* v, int j) {
  const double t1 = kRadix4Fma[j][0], t2 = kRadix4Fma[j][1], t3 = kRadix4Fma[j][2];
  const double c1 = kRadix4Fma[j][3], c2 = kRadix4Fma[j][4], r = kRadix4Fma[j][5];
  const double ux = fmad(-t2, v[1].y, v[1].x), uy = fmad(t2, v[1].x, v[1].y);
  const double ax = fmad(c2, ux, v[0].x), ay = fmad(c2, uy, v[0].y);
  const double bx = fmad(-c2, ux, v[0].x), by = fmad(-c2, uy, v[0].y);
  const double p2x = fmad(-t1, v[2].y, v[2].x), p2y = fmad(t1, v[2].x, v[2].y);
  const double p3x = fmad(-t3, v[3].y, v[3].x), p3y = fmad(t3, v[3].x, v[3].y);
  const double qpx = fmad(r, p3x, p2x), qpy = fmad(r, p3y, p2y);
  const double qmx = fmad(-r, p3x, p2x), qmy = fmad(-r, p3y, p2y);
  v[0].x = fmad(c1, qpx, ax);
  v[0].y = fmad(c1, qpy, ay);
  v[2].x = fmad(-c1, qpx, ax);
  v[2].y = fmad(-c1, qpy, ay);
  v[1].x = fmad(c1, qmy, bx);   // B - i c1 q-
  v[1].y = fmad(-c1, qmx, by);
  v[3].x = fmad(-c1, qmy, bx);  // B + i c1 q-
  v[3].y = fmad(c1, qmx, by);
}

// Stages 4 .. 3 + R (R <= 3) on every output row of a staged tile, in
// registers, after the first pass took stages 1..3 (rows hold at most 2^6
// elements, so this is the last pass): each thread takes groups of 2^R
// elements of one shared-memory column, X = base + j + t 2^3 (t < 2^R),
// which those R stages combine only among themselves (the radix-2^R view of
// R consecutive radix-2 stages).  j is the same for the 32 lanes of a warp
// (they take consecutive columns z of one group row when BZ >= 5), so the
// branch to the groups with j = 0 and j = 4 -- whose twiddles are all or
// mostly 1, -i and eighth turns -- does not diverge.  Forward twiddles;
// imaginary parts have their sign flipped by conj_out on storing.
template <class G, int NTHR, int R>
__device__ __forceinline__ void dit_pass(uint4* sm0, int nt, uint32_t conj_out,
                                         const typename Cplx<G::E>::T* tw) {
  static_assert(G::BX <= 6, "at most two passes: rows of at most 2^6 elements");
  using T = typename Cplx<G::E>::T;
  constexpr int S0 = 3;
  constexpr int GN = 1 << R;
  constexpr int LOG_GROUPS = G::BX + G::BZ - R;
  for (int gt = threadIdx.x; gt < (nt << LOG_GROUPS); gt += NTHR) {
    uint4* sm = sm0 + (gt >> LOG_GROUPS) * G::CHUNKS;
    const int g = gt & ((1 << LOG_GROUPS) - 1);
    const int z = g & ((1 << G::BZ) - 1);
    const int q = g >> G::BZ;
    const int j = q & ((1 << S0) - 1);
    const int base = (q >> S0) << (S0 + R);
    T v[GN];
#pragma unroll
    for (int t = 0; t < GN; ++t) v[t] = *tile_elem<G>(sm, base + j + (t << S0), z);
    if (j == 0) dit_group<G, R, S0, 0>(v, j, tw);
    else if (j == 4) dit_group<G, R, S0, 4>(v, j, tw);
    else if constexpr (R == 2 && sizeof(typename Cplx<G::E>::R) == 8) radix4_fma(v, j);
    else dit_group<G, R, S0, -1>(v, j, tw);
#pragma unroll
    for (int t = 0; t < GN; ++t) {
      v[t].y = flip_sign(v[t].y, conj_out);
      *tile_elem<G>(sm, base + j + (t << S0), z) = v[t];
    }
  }
}

// Stages 1..S on every output row of a staged tile (columns of sm): the
// first pass takes stages 1..3 with compile-time twiddles, the second
// stages 4..S (S <= 6), from the table except where they are whole eighth
// turns.  The butterflies are always the forward ones.  The inverse stages
// (conjugate twiddles) are conj(forward(conj(x))) exactly -- every operation
// of the butterflies is odd in the imaginary parts and rounding to nearest
// is symmetric -- so the first pass flips the sign of the imaginary parts it
// loads and the last pass those it stores.
template <class G, int NTHR>
__device__ __forceinline__ void dit_stages(uint4* sm, int nt, int S, int inverse,
                                           const typename Cplx<G::E>::T* tw) {
  if (S <= 0) return;
  const uint32_t conj = inverse ? 0x80000000u : 0u;
  const int R0 = S >= 3 ? 3 : S;
  const uint32_t conj_out0 = S == R0 ? conj : 0u;
  if (R0 == 3) dit_first_pass<G, NTHR, 3>(sm, nt, conj, conj_out0);
  else if (R0 == 2) dit_first_pass<G, NTHR, 2>(sm, nt, conj, conj_out0);
  else dit_first_pass<G, NTHR, 1>(sm, nt, conj, conj_out0);
  __syncthreads();
  if (S > 3) {  // S <= BX <= 6: the second pass takes the rest, stages 4..S
    const int R = S - 3;
    if (R == 3) dit_pass<G, NTHR, 3>(sm, nt, conj, tw);
    else if (R == 2) dit_pass<G, NTHR, 2>(sm, nt, conj, tw);
    else dit_pass<G, NTHR, 1>(sm, nt, conj, tw);
    __syncthreads();
  }
}

#ifndef BREV_FFT_OOP_THREADS_MULT
#define BREV_FFT_OOP_THREADS_MULT 1
#endif
template <int E, int B>
__host__ __device__ constexpr int fft_oop_threads() {
  return Geom<E, 16, B, B>::THREADS * BREV_FFT_OOP_THREADS_MULT;
}

template <int E, int B>
__global__ void __launch_bounds__(fft_oop_threads<E, B>(), BREV_FFT_MIN_CTAS)
    k_fft_oop(char* __restrict__ dst, const char* __restrict__ src, int k, int S,
              int inverse) {
  using G = Geom<E, 16, B, B>;
  constexpr int NTHR = fft_oop_threads<E, B>();
  using T = typename Cplx<E>::T;
  extern __shared__ uint4 smem_u4[];
  T* tw = reinterpret_cast<T*>(smem_u4 + G::CHUNKS);
  pdl_release();
  fill_twiddles<E, B>(tw);  // shared memory only: overlaps the previous kernel's tail
  pdl_wait();
  const int wy = k - 2 * B;
  const uint32_t y = blockIdx.x;
  const uint32_t ry = rev_bits(y, wy);
  const uint64_t stride = (uint64_t)E << (k - B);
  load_tiles<G, true, NTHR, 1>(smem_u4, src + ((uint64_t)y << B) * E, nullptr, stride, 1);
  __syncthreads();
  dit_stages<G, NTHR>(smem_u4, 1, S, inverse, tw);
  store_tile<G, NTHR>(smem_u4, dst + ((uint64_t)ry << B) * E, stride);
}

// In place: NTHR threads; each FFT pass takes the groups of both staged
// tiles of the pair at once (one barrier per pass for the pair).
template <int E, int B>
__host__ __device__ constexpr int fft_ip_threads() {
  return Geom<E, 16, B, B>::THREADS * BREV_FFT_IP_THREADS_MULT > 1024
             ? 1024
             : Geom<E, 16, B, B>::THREADS * BREV_FFT_IP_THREADS_MULT;
}

// In-place register budget: complex<float> pairs of 2^6 x 2^6 tiles fill
// shared memory at 3 CTAs per SM, so the budget is for 3 (a budget for 5
// measured slower); complex<double> pairs of 2^5 x 2^5 tiles take the
// out-of-place budget.
template <int E>
__host__ __device__ constexpr int fft_ip_min_ctas() {
  return E == 8 ? 3 : BREV_FFT_MIN_CTAS;
}

template <int E, int B>
__global__ void __launch_bounds__(fft_ip_threads<E, B>(), fft_ip_min_ctas<E>())
    k_fft_inplace(char* data, int k, int S, int inverse) {
  using G = Geom<E, 16, B, B>;
  constexpr int NTHR = fft_ip_threads<E, B>();
  using T = typename Cplx<E>::T;
  extern __shared__ uint4 smem_u4[];
  T* tw = reinterpret_cast<T*>(smem_u4 + 2 * G::CHUNKS);
  pdl_release();
  fill_twiddles<E, B>(tw);  // shared memory only: overlaps the previous kernel's tail
  pdl_wait();
  const int wy = k - 2 * B;
  const uint32_t npairs = count_lt(wy);
  const uint32_t q = blockIdx.x;
  uint32_t y, ry;
  int nt;
  if (q < npairs) {
    y = unrank_lt(q, wy);
    ry = rev_bits(y, wy);
    nt = 2;
  } else {
    y = unrank_self(q - npairs, wy);
    ry = y;
    nt = 1;
  }
  const uint64_t stride = (uint64_t)E << (k - B);
  char* const ty = data + ((uint64_t)y << B) * E;
  char* const tr = data + ((uint64_t)ry << B) * E;
  load_tiles<G, false, NTHR, 2>(smem_u4, ty, tr, stride, nt);
  __syncthreads();
  dit_stages<G, NTHR>(smem_u4, nt, S, inverse, tw);  // both tiles in each pass
  store_tile<G, NTHR>(smem_u4, tr, stride);
  if (nt == 2) store_tile<G, NTHR>(smem_u4 + G::CHUNKS, ty, stride);
}

// complex<double> out of place: the FP64 pipe, not HBM, bounds the stages
// (GB300 issues 2 FP64 operations per SM per cycle), so FP64 work outside
// the butterflies costs time.  In the one-tile-per-CTA kernel above every
// CTA spends 2^(B-1) double-precision sincospi on its twiddles (about 0.4
// FP64 operations per element at B = 5).  The streaming kernel runs one CTA
// per resident slot: it computes the twiddles once, and the next tile is in
// flight (cp.async, one commit group per tile, two buffers) while the
// current tile's stages run and it is stored.  The CTAs of an SM share its
// FP64 pipe and progress at different speeds, so tiles are claimed from a
// counter (zeroed in stream order before the launch) rather than dealt out
// by a fixed stride: CTA c takes tile c first, then gridDim.x + the
// counter's old value, one claim ahead so that the atomic's round trip
// overlaps a tile's work.  It is used for 2^5 x 2^5 tiles (the tile of every
// stage count up to 5 once k >= 10) when there are more tiles than resident
// slots; two buffers still fit 6 CTAs per SM.  At B = 6 (one CTA per SM) it
// measured slower, and so did an in-place form with two buffers of tile
// pairs (3 CTAs per SM).
template <int B>
__global__ void __launch_bounds__(fft_oop_threads<16, B>(), BREV_FFT_MIN_CTAS)
    k_fft_oop_stream(char* __restrict__ dst, const char* __restrict__ src, int k, int S,
                     int inverse, unsigned* __restrict__ ticket) {
  constexpr int E = 16;
  using G = Geom<E, 16, B, B>;
  constexpr int NTHR = fft_oop_threads<E, B>();
  using T = typename Cplx<E>::T;
  extern __shared__ uint4 smem_u4[];
  __shared__ uint32_t s_claim;
  T* tw = reinterpret_cast<T*>(smem_u4 + 2 * G::CHUNKS);
  pdl_release();
  fill_twiddles<E, B>(tw);
  pdl_wait();
  const int wy = k - 2 * B;
  const uint32_t ntiles = 1u << wy;
  const uint64_t stride = (uint64_t)E << (k - B);
  uint32_t y = blockIdx.x;  // the grid is smaller than the tile count
  if (threadIdx.x == 0) s_claim = gridDim.x + atomicAdd(ticket, 1u);
  load_tiles<G, true, NTHR, 1, false>(smem_u4, src + ((uint64_t)y << B) * E, nullptr, stride,
                                      1);
  cp_async_commit();
  __syncthreads();
  uint32_t yn = s_claim;
  for (int buf = 0; y < ntiles; buf ^= 1) {
    uint4* const cur = smem_u4 + buf * G::CHUNKS;
    uint32_t claim = 0;
    if (yn < ntiles) {  // the other buffer was released by the barrier ending the last tile
      load_tiles<G, true, NTHR, 1, false>(smem_u4 + (buf ^ 1) * G::CHUNKS,
                                          src + ((uint64_t)yn << B) * E, nullptr, stride, 1);
      if (threadIdx.x == 0) claim = atomicAdd(ticket, 1u);  // the tile after yn
    }
    cp_async_commit();
    cp_async_wait_group<1>();  // this tile's group has landed; the next one may be in flight
    __syncthreads();
    dit_stages<G, NTHR>(cur, 1, S, inverse, tw);
    store_tile<G, NTHR>(cur, dst + ((uint64_t)rev_bits(y, wy) << B) * E, stride);
    if (threadIdx.x == 0) s_claim = yn < ntiles ? gridDim.x + claim : ntiles;
    __syncthreads();  // every thread has read cur before it is refilled, and sees s_claim
    y = yn;
    yn = s_claim;
  }
}

// Tiles (y, rev(y)) of in-place unit q (pairs first, then self-paired tiles).
__device__ __forceinline__ int fft_unit(uint32_t q, int wy, uint32_t npairs, uint32_t& y,
                                        uint32_t& ry) {
  if (q < npairs) {
    y = unrank_lt(q, wy);
    ry = rev_bits(y, wy);
    return 2;
  }
  y = ry = unrank_self(q - npairs, wy);
  return 1;
}

// complex<double> in place, the same way: one CTA per resident slot,
// twiddles once per CTA, units (tile pairs, then self-paired tiles) claimed
// from a counter.  A unit's two tiles are both staged before either is
// written (the swap through the buffer), and units are disjoint.  One
// buffer of a pair per CTA keeps 6 CTAs per SM, whose loads and stores
// overlap each other's stages; two buffers (3 CTAs per SM) measured slower
// (6.06 against 6.01 ms at k = 28, S = 5).
template <int B>
__global__ void __launch_bounds__(fft_ip_threads<16, B>(), BREV_FFT_MIN_CTAS)
    k_fft_inplace_stream(char* data, int k, int S, int inverse, unsigned* __restrict__ ticket) {
  constexpr int E = 16;
  using G = Geom<E, 16, B, B>;
  constexpr int NTHR = fft_ip_threads<E, B>();
  using T = typename Cplx<E>::T;
  extern __shared__ uint4 smem_u4[];
  __shared__ uint32_t s_claim;
  T* tw = reinterpret_cast<T*>(smem_u4 + 2 * G::CHUNKS);
  pdl_release();
  fill_twiddles<E, B>(tw);
  pdl_wait();
  const int wy = k - 2 * B;
  const uint32_t npairs = count_lt(wy);
  const uint32_t units = npairs + count_self(wy);
  const uint64_t stride = (uint64_t)E << (k - B);
  uint32_t q = blockIdx.x;  // the grid is smaller than the unit count
  if (threadIdx.x == 0) s_claim = gridDim.x + atomicAdd(ticket, 1u);
  uint32_t y, ry;
  int nt = fft_unit(q, wy, npairs, y, ry);
  load_tiles<G, false, NTHR, 2, false>(smem_u4, data + ((uint64_t)y << B) * E,
                                       data + ((uint64_t)ry << B) * E, stride, nt);
  __syncthreads();
  uint32_t qn = s_claim;
  while (q < units) {
    uint32_t claim = 0;
    if (qn < units && threadIdx.x == 0) claim = atomicAdd(ticket, 1u);  // the unit after qn
    cp_async_wait_all();
    __syncthreads();
    dit_stages<G, NTHR>(smem_u4, nt, S, inverse, tw);
    store_tile<G, NTHR>(smem_u4, data + ((uint64_t)ry << B) * E, stride);
    if (nt == 2) store_tile<G, NTHR>(smem_u4 + G::CHUNKS, data + ((uint64_t)y << B) * E, stride);
    if (threadIdx.x == 0) s_claim = qn < units ? gridDim.x + claim : units;
    __syncthreads();  // every thread has read the buffer, and sees s_claim
    q = qn;
    if (q < units) {
      nt = fft_unit(q, wy, npairs, y, ry);
      load_tiles<G, false, NTHR, 2, false>(smem_u4, data + ((uint64_t)y << B) * E,
                                           data + ((uint64_t)ry << B) * E, stride, nt);
    }
    qn = s_claim;
  }
}

// Small arrays (and any array that fits): one CTA stages the permuted array
// in shared memory, runs the stages, and stores it.
template <int E>
__global__ void __launch_bounds__(256) k_fft_small(char* dst, const char* src, int k, int S,
                                                 int inverse) {
  using T = typename Cplx<E>::T;
  extern __shared__ uint4 smem_u4[];
  T* a = reinterpret_cast<T*>(smem_u4);
  pdl_enter();
  const uint32_t n = 1u << k;
  const T* s = reinterpret_cast<const T*>(src);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) a[rev_bits(i, k)] = s[i];
  __syncthreads();
  for (int st = 1; st <= S; ++st) {
    const uint32_t h = 1u << (st - 1);
    for (uint32_t p = threadIdx.x; p < n / 2; p += blockDim.x) {
      const uint32_t j = p & (h - 1);
      const uint32_t i0 = ((p >> (st - 1)) << st) + j;
      double sn, cs;
      sincospi((double)j / (double)h, &sn, &cs);
      T w;
      w.x = (typename Cplx<E>::R)cs;
      w.y = (typename Cplx<E>::R)(inverse ? sn : -sn);
      const T x0 = a[i0], x1 = a[i0 + h];
      T t;
      t.x = x1.x * w.x - x1.y * w.y;
      t.y = x1.x * w.y + x1.y * w.x;
      a[i0].x = x0.x + t.x;
      a[i0].y = x0.y + t.y;
      a[i0 + h].x = x0.x - t.x;
      a[i0 + h].y = x0.y - t.y;
    }
    __syncthreads();
  }
  T* d = reinterpret_cast<T*>(dst);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) d[i] = a[i];
}

// ------------------------------------------------------------------ host --

struct FftKernel {
  const void* oop;
  const void* inplace;
  const void* oop_stream;      // complex<double> with B = 5: the streaming forms
  const void* inplace_stream;  // (else nullptr)
  int B, threads, ip_threads;
  unsigned tile_bytes;
};

template <int E, int B>
static FftKernel fft_k() {
  using G = Geom<E, 16, B, B>;
  FftKernel K{(const void*)&k_fft_oop<E, B>, (const void*)&k_fft_inplace<E, B>, nullptr, nullptr,
              B, fft_oop_threads<E, B>(), fft_ip_threads<E, B>(), G::TILE_BYTES};
  if constexpr (E == 16 && B == 5) {
    K.oop_stream = (const void*)&k_fft_oop_stream<B>;
    K.inplace_stream = (const void*)&k_fft_inplace_stream<B>;
  }
  return K;
}

// Grid of a streaming kernel: every resident slot of the device, at most
// one CTA per unit.
static cudaError_t stream_grid(const void* kern, unsigned threads, unsigned smem,
                               unsigned long long units, unsigned* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads,
                                                                smem);
  if (e != cudaSuccess) return e;
  const unsigned long long slots =
      (unsigned long long)std::max(per_sm, 1) * (unsigned long long)current_device_sm_count();
  *grid = (unsigned)std::min(slots, units);
  return cudaSuccess;
}

static bool fft_lookup(int E, int B, FftKernel* out) {
  switch (E * 16 + B) {
    case 16 * 16 + 3: *out = fft_k<16, 3>(); return true;
    case 16 * 16 + 4: *out = fft_k<16, 4>(); return true;
    case 16 * 16 + 5: *out = fft_k<16, 5>(); return true;
    case 16 * 16 + 6: *out = fft_k<16, 6>(); return true;
    case 8 * 16 + 4: *out = fft_k<8, 4>(); return true;
    case 8 * 16 + 5: *out = fft_k<8, 5>(); return true;
    case 8 * 16 + 6: *out = fft_k<8, 6>(); return true;
  }
  return false;
}

}  // namespace brev

using namespace brev;

extern "C" brev_status brev_fft_stages(void* dst, const void* src, int log2n, int elem_bytes,
                                       int stages, int inverse, void* stream) {
  BREV_TRACE("brev_fft_stages");
  const int E = elem_bytes, k = log2n, S = stages;
  if (E != 8 && E != 16)
    return set_error(BREV_ERR_INVALID_ARG, "elem_bytes=%d (complex<float> 8 or complex<double> 16)",
                     E);
  if (k < 0 || k > 31) return set_error(BREV_ERR_INVALID_ARG, "log2n=%d", k);
  if (S < 0 || S > k) return set_error(BREV_ERR_INVALID_ARG, "stages=%d for log2n=%d", S, k);
  if (!dst || !src) return set_error(BREV_ERR_INVALID_ARG, "NULL data pointer");
  if ((uintptr_t)dst % 16 || (uintptr_t)src % 16)
    return set_error(BREV_ERR_ALIGNMENT, "complex arrays must be 16-byte aligned");
  const uint64_t bytes = (uint64_t)E << k;
  if (dst != src) {
    const uint64_t d = (uintptr_t)dst, s = (uintptr_t)src;
    if (d < s + bytes && s < d + bytes)
      return set_error(BREV_ERR_OVERLAP, "source and destination overlap partially");
  }
  brev_status st = check_device_range(src, bytes, "source");
  if (st == BREV_OK && dst != src) st = check_device_range(dst, bytes, "destination");
  if (st != BREV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool inplace = dst == src;
  const int pref = E == 16 ? 5 : 6;
  int B = std::max(S, std::min(pref, k / 2));
  FftKernel K{};
  const bool tiles = 2 * B <= k && B >= b_min_for(E) && fft_lookup(E, B, &K);
  cudaError_t e;
  if (!tiles) {
    // whole array in one CTA when it fits in shared memory
    const unsigned smem = (unsigned)E << k;
    if (smem > 96 * 1024)
      return set_error(BREV_ERR_UNSUPPORTED,
                       "%d stages need tile rows of 2^%d elements, not compiled for k=%d E=%d", S,
                       B, k, E);
    const void* kern = E == 16 ? (const void*)&k_fft_small<16> : (const void*)&k_fft_small<8>;
    e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return cuda_error(e, "shared-memory limit");
    char* d = (char*)dst;
    const char* sr = (const char*)src;
    int kk = k, SS = S, inv = inverse ? 1 : 0;
    void* args[] = {(void*)&d, (void*)&sr, (void*)&kk, (void*)&SS, (void*)&inv};
    e = launch_pdl(kern, 1, 256, args, smem, s);
    if (e != cudaSuccess) return cuda_error(e, "fused FFT launch");
    note_launch();
    return BREV_OK;
  }
  const unsigned tw_bytes = (unsigned)E << (K.B - 1);
  int kk = k, SS = S, inv = inverse ? 1 : 0;
  if (inplace) {
    const int w = k - 2 * K.B;
    const unsigned long long grid = (unsigned long long)count_lt(w) + count_self(w);
    if (K.inplace_stream) {
      const unsigned smem = 2 * K.tile_bytes + tw_bytes;
      unsigned g = 0;
      e = ensure_smem(K.inplace_stream, smem);
      if (e == cudaSuccess) e = stream_grid(K.inplace_stream, K.ip_threads, smem, grid, &g);
      if (e != cudaSuccess) return cuda_error(e, "streaming kernel shape");
      if (g < grid) {
        void* ticket = nullptr;
        e = ws_alloc(&ticket, 16, s);
        if (e != cudaSuccess) {
          cudaGetLastError();
          return set_error(BREV_ERR_OOM, "unit counter: %s", cudaGetErrorString(e));
        }
        e = cudaMemsetAsync(ticket, 0, 16, s);
        if (e == cudaSuccess) {
          char* d = (char*)dst;
          unsigned* t = (unsigned*)ticket;
          void* args[] = {(void*)&d, (void*)&kk, (void*)&SS, (void*)&inv, (void*)&t};
          e = launch_pdl(K.inplace_stream, g, K.ip_threads, args, smem, s);
        }
        ws_free(ticket, s);
        if (e != cudaSuccess) return cuda_error(e, "fused FFT launch");
        note_launch();
        return BREV_OK;
      }
    }
    const unsigned smem = 2 * K.tile_bytes + tw_bytes;
    e = ensure_smem(K.inplace, smem);
    if (e != cudaSuccess) return cuda_error(e, "shared-memory limit");
    char* d = (char*)dst;
    void* args[] = {(void*)&d, (void*)&kk, (void*)&SS, (void*)&inv};
    e = launch_pdl(K.inplace, (unsigned)grid, K.ip_threads, args, smem, s);
  } else {
    const unsigned long long units = 1ull << (k - 2 * K.B);
    char* d = (char*)dst;
    const char* sr = (const char*)src;
    unsigned grid = (unsigned)units;
    if (K.oop_stream) {
      const unsigned smem = 2 * K.tile_bytes + tw_bytes;
      e = ensure_smem(K.oop_stream, smem);
      if (e == cudaSuccess) e = stream_grid(K.oop_stream, K.threads, smem, units, &grid);
      if (e != cudaSuccess) return cuda_error(e, "streaming kernel shape");
      if (grid < units) {  // more tiles than resident slots: stream them
        void* ticket = nullptr;
        e = ws_alloc(&ticket, 16, s);
        if (e != cudaSuccess) {
          cudaGetLastError();
          return set_error(BREV_ERR_OOM, "tile counter: %s", cudaGetErrorString(e));
        }
        e = cudaMemsetAsync(ticket, 0, 16, s);
        if (e == cudaSuccess) {
          unsigned* t = (unsigned*)ticket;
          void* args[] = {(void*)&d, (void*)&sr, (void*)&kk, (void*)&SS, (void*)&inv, (void*)&t};
          e = launch_pdl(K.oop_stream, grid, K.threads, args, smem, s);
        }
        ws_free(ticket, s);
        if (e != cudaSuccess) return cuda_error(e, "fused FFT launch");
        note_launch();
        return BREV_OK;
      }
    }
    const unsigned smem = K.tile_bytes + tw_bytes;
    e = ensure_smem(K.oop, smem);
    if (e != cudaSuccess) return cuda_error(e, "shared-memory limit");
    void* args[] = {(void*)&d, (void*)&sr, (void*)&kk, (void*)&SS, (void*)&inv};
    e = launch_pdl(K.oop, (unsigned)grid, K.threads, args, smem, s);
  }
  if (e != cudaSuccess) return cuda_error(e, "fused FFT launch");
  note_launch();
  return BREV_OK;
}
