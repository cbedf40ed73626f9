/* A C program using the library through include/brev.h alone (no Python,
 * no PyTorch): device buffers from the CUDA runtime, results checked
 * against the CPU oracle's C library (test infrastructure).  Exit status 0
 * and the line "c client ok" on success. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "brev.h"
#include "oracle.h"

#define CHECK_CUDA(x)                                                         \
    do {                                                                      \
        cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) {                                              \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));          \
            return 1;                                                         \
        }                                                                     \
    } while (0)
#define CHECK_BREV(x)                                                         \
    do {                                                                      \
        brev_status s_ = (x);                                                 \
        if (s_ != BREV_OK) {                                                  \
            fprintf(stderr, "%s: %s: %s\n", #x, brev_status_string(s_),       \
                    brev_last_error());                                       \
            return 1;                                                         \
        }                                                                     \
    } while (0)

static void fill(unsigned char *p, size_t bytes, uint64_t seed) {
    uint64_t x = seed;
    for (size_t i = 0; i < bytes; ++i) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        p[i] = (unsigned char)(x >> 56);
    }
}

int main(void) {
    const int k = 18, E = 16;
    const size_t bytes = (size_t)E << k;
    unsigned char *h = malloc(bytes), *want = malloc(bytes), *got = malloc(bytes);
    if (!h || !want || !got) return 1;
    fill(h, bytes, 7);
    if (oracle_brev_oop(want, h, k, E) != 0) return 1;

    void *d_src = NULL, *d_dst = NULL;
    CHECK_CUDA(cudaMalloc(&d_src, bytes));
    CHECK_CUDA(cudaMalloc(&d_dst, bytes));
    CHECK_CUDA(cudaMemcpy(d_src, h, bytes, cudaMemcpyHostToDevice));

    /* out of place, on the default stream */
    CHECK_BREV(brev_permute_to(d_dst, d_src, k, E, NULL));
    CHECK_CUDA(cudaMemcpy(got, d_dst, bytes, cudaMemcpyDeviceToHost));
    if (memcmp(got, want, bytes) != 0) { fprintf(stderr, "out-of-place mismatch\n"); return 1; }

    /* in place, on a stream of our own */
    cudaStream_t st;
    CHECK_CUDA(cudaStreamCreate(&st));
    CHECK_BREV(brev_permute(d_src, k, E, 1, st));
    CHECK_CUDA(cudaStreamSynchronize(st));
    CHECK_CUDA(cudaMemcpy(got, d_src, bytes, cudaMemcpyDeviceToHost));
    if (memcmp(got, want, bytes) != 0) { fprintf(stderr, "in-place mismatch\n"); return 1; }

    /* a batch of two arrays of different sizes and element sizes */
    const int k2 = 11, E2 = 8;
    const size_t bytes2 = (size_t)E2 << k2;
    unsigned char *h2 = malloc(bytes2), *want2 = malloc(bytes2), *got2 = malloc(bytes2);
    if (!h2 || !want2 || !got2) return 1;
    fill(h2, bytes2, 11);
    if (oracle_brev_oop(want2, h2, k2, E2) != 0) return 1;
    void *d2 = NULL;
    CHECK_CUDA(cudaMalloc(&d2, bytes2));
    CHECK_CUDA(cudaMemcpy(d2, h2, bytes2, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d_src, h, bytes, cudaMemcpyHostToDevice));
    void *ptrs[2] = {d_src, d2};
    int ks[2] = {k, k2}, es[2] = {E, E2};
    CHECK_BREV(brev_permute_batched_mixed(ptrs, ks, es, 2, st));
    CHECK_CUDA(cudaStreamSynchronize(st));
    CHECK_CUDA(cudaMemcpy(got, d_src, bytes, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(got2, d2, bytes2, cudaMemcpyDeviceToHost));
    if (memcmp(got, want, bytes) != 0 || memcmp(got2, want2, bytes2) != 0) {
        fprintf(stderr, "batched mismatch\n");
        return 1;
    }

    /* an error status, with its message, and nothing launched */
    const uint64_t launches = brev_launch_count();
    brev_status s = brev_permute_to((char *)d_dst + 8, (char *)d_src + 8, k, E, NULL);
    if (s != BREV_ERR_ALIGNMENT || brev_launch_count() != launches || !brev_last_error()[0]) {
        fprintf(stderr, "misaligned call: %s\n", brev_status_string(s));
        return 1;
    }

    cudaStreamDestroy(st);
    cudaFree(d_src);
    cudaFree(d_dst);
    cudaFree(d2);
    free(h); free(want); free(got); free(h2); free(want2); free(got2);
    printf("c client ok (library version %d)\n", brev_version());
    return 0;
}
