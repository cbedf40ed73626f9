// Device ceilings measured by the library itself (no counterpart in the
// paper): the FP64 fused multiply-add rate that bounds the complex<double>
// FFT stages fused into the permutation.  A roofline against this number is
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
