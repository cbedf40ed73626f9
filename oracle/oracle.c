/*
 * CPU oracle for the bit-reversed permutation: TEST INFRASTRUCTURE ONLY.
 * See oracle.h for who may use it.  Plain C99 + POSIX threads, no compiler
 * builtins, no tables, nothing shared with the GPU library.
 *
 * Every function is the plain definition from the Introduction of the paper
 * (element i moves to rev_k(i), worked example for n = 8).  No blocking,
 * tiling or reordering is done here.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* Largest element we accept: the library's own limit is 16 bytes; the
 * oracle is more permissive so that tests can use wider fingerprints. */
#define ORACLE_MAX_ELEM 64

static int bad_args(int k, int elem_bytes)
{
    return k < 0 || k > 40 || elem_bytes <= 0 || elem_bytes > ORACLE_MAX_ELEM;
}

/* Naive bitwise rev (Introduction, "Theta(b)" per index): take the bits of
 * i from least to most significant and push each one onto the result from
 * the right, so the first bit taken ends up most significant. */
uint64_t oracle_rev_bits(uint64_t i, int k)
{
    uint64_t r = 0;
    int j;
    for (j = 0; j < k; ++j) {
        r = (r << 1) | (i & 1u);
        i >>= 1;
    }
    return r;
}

/* Definition of the permutation (Introduction): dst[rev(i)] <- src[i]. */
int oracle_brev_oop(void *dst, const void *src, int k, int elem_bytes)
{
    uint64_t n, i;
    unsigned char *d = (unsigned char *)dst;
    const unsigned char *s = (const unsigned char *)src;
    if (bad_args(k, elem_bytes) || (!dst || !src))
        return -1;
    n = (uint64_t)1 << k;
    for (i = 0; i < n; ++i)
        memcpy(d + oracle_rev_bits(i, k) * (uint64_t)elem_bytes,
               s + i * (uint64_t)elem_bytes, (size_t)elem_bytes);
    return 0;
}

/* In place (Introduction: the same map, with the result in the input's
 * buffer): the definition applied to a copy of the input.  k = 0 and k = 1
 * are identities like every other size, with no special case. */
int oracle_brev_inplace(void *v, int k, int elem_bytes)
{
    uint64_t bytes;
    void *copy;
    int rc;
    if (bad_args(k, elem_bytes) || !v)
        return -1;
    bytes = ((uint64_t)1 << k) * (uint64_t)elem_bytes;
    copy = malloc((size_t)bytes);
    if (!copy)
        return -1;
    memcpy(copy, v, (size_t)bytes);
    rc = oracle_brev_oop(v, copy, k, elem_bytes);
    free(copy);
    return rc;
}

struct oop_slice {
    unsigned char *dst;
    const unsigned char *src;
    uint64_t begin, end;
    int k, elem_bytes;
};

static void *oop_slice_run(void *arg)
{
    struct oop_slice *s = (struct oop_slice *)arg;
    uint64_t i;
    for (i = s->begin; i < s->end; ++i)
        memcpy(s->dst + oracle_rev_bits(i, s->k) * (uint64_t)s->elem_bytes,
               s->src + i * (uint64_t)s->elem_bytes, (size_t)s->elem_bytes);
    return NULL;
}

/* The same definition as oracle_brev_oop, each thread taking one
 * contiguous range of source indices.  Destinations of different i never
 * coincide (rev is a bijection), so the threads never write the same
 * element. */
int oracle_brev_oop_mt(void *dst, const void *src, int k, int elem_bytes,
                       int threads)
{
    uint64_t n, per;
    int t, started = 0;
    pthread_t *tid;
    struct oop_slice *sl;
    if (bad_args(k, elem_bytes) || !dst || !src || threads < 1)
        return -1;
    n = (uint64_t)1 << k;
    if ((uint64_t)threads > n)
        threads = (int)n;
    tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    sl = (struct oop_slice *)calloc((size_t)threads, sizeof(struct oop_slice));
    if (!tid || !sl) {
        free(tid);
        free(sl);
        return -1;
    }
    per = (n + (uint64_t)threads - 1) / (uint64_t)threads;
    for (t = 0; t < threads; ++t) {
        sl[t].dst = (unsigned char *)dst;
        sl[t].src = (const unsigned char *)src;
        sl[t].begin = per * (uint64_t)t < n ? per * (uint64_t)t : n;
        sl[t].end = per * (uint64_t)(t + 1) < n ? per * (uint64_t)(t + 1) : n;
        sl[t].k = k;
        sl[t].elem_bytes = elem_bytes;
    }
    for (t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, oop_slice_run, &sl[t]) != 0)
            break;
        ++started;
    }
    oop_slice_run(&sl[0]);
    /* a slice whose thread could not start runs on this thread */
    for (t = 1 + started; t < threads; ++t)
        oop_slice_run(&sl[t]);
    for (t = 1; t <= started; ++t)
        pthread_join(tid[t], NULL);
    free(tid);
    free(sl);
    return started + 1;
}

/* out[s] = src[rev(idx[s])]: the definition read at one output index at a
 * time (the permutation is an involution, so the element landing at j is
 * the one that started at rev(j)). */
int oracle_brev_gather(void *out, const void *src, const uint64_t *idx,
                       int64_t count, int k, int elem_bytes)
{
    int64_t s;
    uint64_t n;
    unsigned char *o = (unsigned char *)out;
    const unsigned char *p = (const unsigned char *)src;
    if (bad_args(k, elem_bytes) || count < 0 || (count && (!out || !src || !idx)))
        return -1;
    n = (uint64_t)1 << k;
    for (s = 0; s < count; ++s) {
        if (idx[s] >= n)
            return -1;
        memcpy(o + (uint64_t)s * (uint64_t)elem_bytes,
               p + oracle_rev_bits(idx[s], k) * (uint64_t)elem_bytes,
               (size_t)elem_bytes);
    }
    return 0;
}

/* Matrix transposition, element by element, from its definition. */
int oracle_transpose(void *dst, const void *src, int log2_rows, int log2_cols,
                     int elem_bytes)
{
    uint64_t R, C, i, j;
    unsigned char *d = (unsigned char *)dst;
    const unsigned char *s = (const unsigned char *)src;
    if (log2_rows < 0 || log2_cols < 0 || bad_args(log2_rows + log2_cols, elem_bytes) ||
        !dst || !src)
        return -1;
    R = (uint64_t)1 << log2_rows;
    C = (uint64_t)1 << log2_cols;
    for (i = 0; i < R; ++i)
        for (j = 0; j < C; ++j)
            memcpy(d + (j * R + i) * (uint64_t)elem_bytes,
                   s + (i * C + j) * (uint64_t)elem_bytes, (size_t)elem_bytes);
    return 0;
}

/* Even indices first, then odd ones (the Stockham even-odd step). */
int oracle_even_odd(void *dst, const void *src, int k, int elem_bytes)
{
    uint64_t n, i, out = 0;
    unsigned char *d = (unsigned char *)dst;
    const unsigned char *s = (const unsigned char *)src;
    if (bad_args(k, elem_bytes) || !dst || !src)
        return -1;
    n = (uint64_t)1 << k;
    for (i = 0; i < n; i += 2)
        memcpy(d + (out++) * (uint64_t)elem_bytes, s + i * (uint64_t)elem_bytes,
               (size_t)elem_bytes);
    for (i = 1; i < n; i += 2)
        memcpy(d + (out++) * (uint64_t)elem_bytes, s + i * (uint64_t)elem_bytes,
               (size_t)elem_bytes);
    return 0;
}

/* A deck cut in half and the halves interleaved (faro shuffle). */
int oracle_perfect_shuffle(void *dst, const void *src, int k, int elem_bytes)
{
    uint64_t n, h, i;
    unsigned char *d = (unsigned char *)dst;
    const unsigned char *s = (const unsigned char *)src;
    if (bad_args(k, elem_bytes) || !dst || !src)
        return -1;
    n = (uint64_t)1 << k;
    if (n == 1) {
        memcpy(d, s, (size_t)elem_bytes);
        return 0;
    }
    h = n / 2;
    for (i = 0; i < h; ++i) {
        memcpy(d + (2 * i) * (uint64_t)elem_bytes, s + i * (uint64_t)elem_bytes,
               (size_t)elem_bytes);
        memcpy(d + (2 * i + 1) * (uint64_t)elem_bytes, s + (h + i) * (uint64_t)elem_bytes,
               (size_t)elem_bytes);
    }
    return 0;
}

/* Bit-reversed permutation, then the textbook radix-2 DIT butterflies stage
 * by stage, twiddles from cos/sin of the exact angle. */
int oracle_fft_dit_stages(double *out, const double *in, int k, int stages, int inverse)
{
    uint64_t n, m, h, base, j;
    int s;
    const double two_pi = 6.283185307179586476925286766559;
    if (k < 0 || k > 30 || stages < 0 || stages > k || !out || !in)
        return -1;
    if (oracle_brev_oop(out, in, k, 2 * (int)sizeof(double)) != 0)
        return -1;
    n = (uint64_t)1 << k;
    for (s = 1; s <= stages; ++s) {
        m = (uint64_t)1 << s;
        h = m / 2;
        for (base = 0; base < n; base += m) {
            for (j = 0; j < h; ++j) {
                const double ang = two_pi * (double)j / (double)m;
                const double wr = cos(ang), wi = inverse ? sin(ang) : -sin(ang);
                double *a = out + 2 * (base + j);
                double *b = out + 2 * (base + j + h);
                const double tr = b[0] * wr - b[1] * wi;
                const double ti = b[0] * wi + b[1] * wr;
                const double ar = a[0], ai = a[1];
                a[0] = ar + tr;
                a[1] = ai + ti;
                b[0] = ar - tr;
                b[1] = ai - ti;
            }
        }
    }
    return 0;
}
