// Device ceilings measured by the library itself (no counterpart in the
// paper): the FP64 fused multiply-add rate that bounds the complex<double>
// FFT stages fused into the permutation, and the rate at which the SMs
// copy page-locked host memory to page-locked host memory, which bounds the
// host-buffer path (brev_permute_host).  A roofline against this number is
// against the GPU the code runs on, not against a figure derived from
// datasheet unit counts and clocks.
#include <algorithm>

#include "brev_internal.h"
#include "brev_trace.h"

namespace brev {

constexpr int FMA_CHAINS = 8;     // independent chains per thread (hides the FMA latency)
constexpr int FMA_THREADS = 256;

// Every thread runs FMA_CHAINS independent chains x <- x * a + c for
// `iters` rounds (a slightly below 1 keeps the values bounded), then
// stores one sum only if it equals an impossible value, so the compiler
// keeps every FMA and the kernel writes nothing in practice.
__global__ void __launch_bounds__(FMA_THREADS) k_fp64_fma(double* sink, int iters, double a,
                                                           double c) {
  double x[FMA_CHAINS];
#pragma unroll
  for (int j = 0; j < FMA_CHAINS; ++j) x[j] = 1e-3 * (threadIdx.x + 1) + j;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; ++j) x[j] = fma(x[j], a, c);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < FMA_CHAINS; ++j) s += x[j];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace brev

using namespace brev;

extern "C" brev_status brev_fp64_fma_tflops(double* tflops) {
  BREV_TRACE("brev_fp64_fma_tflops");
  if (!tflops) return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  *tflops = 0;
  int sms = current_device_sm_count(), per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma,
                                                                FMA_THREADS, 0);
  if (e != cudaSuccess || per_sm < 1) return cuda_error(e, "FMA kernel occupancy");
  const unsigned grid = (unsigned)(sms * per_sm);
  cudaStream_t st = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "FMA stream");
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMallocAsync((void**)&sink, grid * sizeof(double), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0;
  // about 10 ms per launch at 1.2 TFLOP/s: 2 * grid * 256 * 8 * iters flops
  const int iters = (int)std::max(64.0, 1.2e12 * 1e-2 /
                                            (2.0 * grid * FMA_THREADS * FMA_CHAINS));
  const double a = 0.999999999, c = 1e-9;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    k_fp64_fma<<<grid, FMA_THREADS, 0, st>>>(sink, iters, a, c);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0)  // the first launch warms up
      best = std::max(best, 2.0 * grid * FMA_THREADS * FMA_CHAINS * (double)iters /
                                (ms * 1e-3) / 1e12);
    note_launch();
  }
  const cudaError_t err = e;
  if (sink) cudaFreeAsync(sink, st);
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (err != cudaSuccess) return cuda_error(err, "FMA rate measurement");
  *tflops = best;
  return BREV_OK;
}

// ------------------------------------------- host link, SM-driven copy --
namespace brev {

constexpr int LINK_THREADS = 256;
constexpr int LINK_UNROLL = 4;

// dst[i] = src[i] for n 16-byte chunks, grid-stride, LINK_UNROLL loads in
// flight per thread before their stores.
__global__ void __launch_bounds__(LINK_THREADS) k_link_copy(uint4* __restrict__ dst,
                                                            const uint4* __restrict__ src,
                                                            uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * LINK_THREADS;
  uint64_t i = (uint64_t)blockIdx.x * LINK_THREADS + threadIdx.x;
  for (; i + (LINK_UNROLL - 1) * stride < n; i += LINK_UNROLL * stride) {
    uint4 v[LINK_UNROLL];
#pragma unroll
    for (int j = 0; j < LINK_UNROLL; ++j) v[j] = src[i + j * stride];
#pragma unroll
    for (int j = 0; j < LINK_UNROLL; ++j) dst[i + j * stride] = v[j];
  }
  for (; i < n; i += stride) dst[i] = src[i];
}

// Device address of a page-locked host range [p, p + bytes), or nullptr.
static void* mapped_host(const void* p, uint64_t bytes) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  (void)bytes;
  return a.devicePointer;
}

}  // namespace brev

extern "C" brev_status brev_host_link_gbs(void* dst_host, const void* src_host, uint64_t bytes,
                                          double* gbs) {
  BREV_TRACE("brev_host_link_gbs");
  if (!gbs || !dst_host || !src_host) return set_error(BREV_ERR_INVALID_ARG, "NULL argument");
  *gbs = 0;
  if (bytes == 0 || bytes % 16 || (uintptr_t)dst_host % 16 || (uintptr_t)src_host % 16)
    return set_error(BREV_ERR_ALIGNMENT, "16-byte aligned pointers and a multiple of 16 bytes");
  const uint64_t d = (uintptr_t)dst_host, s = (uintptr_t)src_host;
  if (d < s + bytes && s < d + bytes) return set_error(BREV_ERR_OVERLAP, "buffers overlap");
  void* dd = mapped_host(dst_host, bytes);
  void* ds = mapped_host(src_host, bytes);
  if (!dd || !ds)
    return set_error(BREV_ERR_INVALID_ARG, "both buffers must be page-locked host memory");
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "link stream");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const unsigned grid = (unsigned)current_device_sm_count() * 8;
  double best = 0;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    k_link_copy<<<grid, LINK_THREADS, 0, st>>>((uint4*)dd, (const uint4*)ds, bytes / 16);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0)  // the first copy warms up
      best = std::max(best, 2.0 * (double)bytes / (ms * 1e-3) / 1e9);
    note_launch();
  }
  const cudaError_t err = e;
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (err != cudaSuccess) return cuda_error(err, "host link copy");
  *gbs = best;
  return BREV_OK;
}
