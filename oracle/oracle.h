/*
 * CPU oracle for the bit-reversed permutation: TEST INFRASTRUCTURE ONLY.
 *
 * This header and oracle.c are the plain, slow, obviously correct statement
 * of what the GPU library computes.  Only the test-suite, the smoke check in
 * __graft_entry__.py and the CPU-baseline / reference legs of bench.py may
 * load or call it.  The product path (the CUDA library and its Python
 * binding) never includes, links or calls anything here, and this file
 * includes nothing from the product.
 *
 * Definition followed (Introduction, the bit-reversed permutation and the
 * n = 8 worked example): for an array of n = 2^k elements, the element at
 * index i moves to index rev_k(i), where rev_k reverses the k-bit binary
 * representation of i.  Elements are opaque blobs of E bytes; nothing is
 * computed on them, only moved.
 */
#ifndef BREV_ORACLE_H
#define BREV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* rev_k(i): reverse the low k bits of i one bit at a time (the naive
 * bitwise rev of the Introduction, Theta(k) per index).  Bits of i above
 * bit k-1 are ignored.  k in [0, 63]; k = 0 gives 0. */
uint64_t oracle_rev_bits(uint64_t i, int k);

/* Out-of-place permutation: dst[rev_k(i)] = src[i] for every i < 2^k,
 * element size elem_bytes.  dst and src must not overlap.
 * Returns 0, or -1 on a bad argument. */
int oracle_brev_oop(void *dst, const void *src, int k, int elem_bytes);

/* In-place permutation: the definition (v[rev_k(i)] = old v[i]) applied to
 * a copy of the input.  Returns 0, or -1 on a bad argument or when the copy
 * cannot be allocated. */
int oracle_brev_inplace(void *v, int k, int elem_bytes);

/* The out-of-place definition again with the index range split over
 * `threads` POSIX threads: only for timing on many host cores.  Same result
 * as oracle_brev_oop.  Returns the number of threads used, or -1. */
int oracle_brev_oop_mt(void *dst, const void *src, int k, int elem_bytes,
                       int threads);

/* Expected output at sampled positions: out[s] = src[rev_k(idx[s])] for
 * s < count, where src holds the whole 2^k-element input.  Used to check
 * full-size GPU runs at a sample of output indices. */
int oracle_brev_gather(void *out, const void *src, const uint64_t *idx,
                       int64_t count, int k, int elem_bytes);

/* Transposition of a row-major 2^a x 2^c matrix of elem_bytes elements:
 * dst[j * 2^a + i] = src[i * 2^c + j] (Introduction: the even-odd step as a
 * matrix transposition).  dst and src must not overlap.  Returns 0 or -1. */
int oracle_transpose(void *dst, const void *src, int log2_rows, int log2_cols,
                     int elem_bytes);

/* Even-odd step of the Stockham auto-sort (Introduction): the elements at
 * even indices, in order, followed by those at odd indices.  n = 2^k, k >= 1
 * (k = 0 copies the single element).  Returns 0 or -1. */
int oracle_even_odd(void *dst, const void *src, int k, int elem_bytes);

/* Perfect (faro) shuffle, the inverse of the even-odd step (Introduction):
 * the two halves interleaved, dst[2i] = src[i], dst[2i+1] = src[n/2 + i].
 * Returns 0 or -1. */
int oracle_perfect_shuffle(void *dst, const void *src, int k, int elem_bytes);

/* The first `stages` stages of the iterative radix-2 decimation-in-time FFT
 * applied after the bit-reversed permutation (Introduction: once the
 * permutation has been applied, every level of the Cooley-Tukey recursion
 * finds its even-odd split already done).  in and out hold n = 2^k complex
 * numbers as interleaved (re, im) doubles; out = stages of rev-permuted in,
 * all arithmetic in double.  Stage s (1-based) combines, in every block of
 * m = 2^s consecutive elements, a[j] and a[j + m/2] (j < m/2) with the twiddle
 * w = exp(-2 pi i j / m) (exp(+...) when inverse != 0):
 *   (a[j], a[j + m/2]) <- (a[j] + w a[j + m/2], a[j] - w a[j + m/2]).
 * stages = k gives the full (unnormalised) DFT.  Returns 0 or -1. */
int oracle_fft_dit_stages(double *out, const double *in, int k, int stages, int inverse);

#ifdef __cplusplus
}
#endif

#endif /* BREV_ORACLE_H */
