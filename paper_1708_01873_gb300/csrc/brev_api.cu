// C ABI of the library: argument checks, tile-shape choice (built-in
// defaults or a tuned table), single-array launches, the host-buffer path,
// the autotuner and its JSON cache, device queries and error reporting.
#include <algorithm>
#include <atomic>
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "brev_device.cuh"
#include "brev_internal.h"
#include "brev_trace.h"

namespace brev {

// ------------------------------------------------------------- errors --
static thread_local std::string t_last_error;
static std::atomic<uint64_t> g_launches{0};

void note_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void note_launch_adjust(int64_t delta) {
  g_launches.fetch_add((uint64_t)delta, std::memory_order_relaxed);
}

brev_status set_error(brev_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return s;
}

brev_status cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free launch error so the next call starts clean
  return set_error(BREV_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static bool valid_E(int E) { return E == 1 || E == 2 || E == 4 || E == 8 || E == 16; }
static int e_index(int E) {
  switch (E) {
    case 16: return 0;
    case 8: return 1;
    case 4: return 2;
    case 2: return 3;
    case 1: return 4;
  }
  return -1;
}

// ------------------------------------------------------- device state --
static std::mutex g_mu;
static std::set<std::pair<const void*, int>> g_smem_done;

// Workspace pool.  Descriptor tables, ticket counters and staging buffers
// are stream-ordered allocations from a pool the library owns (one per
// device) that keeps up to BREV_WS_POOL_KEEP_BYTES reserved across
// synchronisations.  The device's default pool returns its memory at every
// synchronisation (release threshold 0), so the first stream-ordered
// allocation after one maps memory again on the calling thread -- about
// 0.1 ms on GB300, paid by every call made right after a synchronise while
// the GPU waits.  Beyond the kept amount (the host path's staging buffer of
// a large array) memory still goes back at synchronisation.  The caller's
// default pool is left as it is.
#ifndef BREV_WS_POOL_KEEP_BYTES
#define BREV_WS_POOL_KEEP_BYTES (32ull << 20)
#endif
static std::vector<cudaMemPool_t> g_ws_pools;  // per device, created on first use

static cudaError_t workspace_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_ws_pools.size() <= dev) g_ws_pools.resize(dev + 1, nullptr);
  if (!g_ws_pools[dev]) {
    // the first stream-ordered allocation may come inside a stream capture:
    // creating the pool is not a stream operation, so it may run there
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaThreadExchangeStreamCaptureMode(&mode);
    struct Restore {
      cudaStreamCaptureMode m;
      ~Restore() { cudaThreadExchangeStreamCaptureMode(&m); }
    } restore{mode};
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = BREV_WS_POOL_KEEP_BYTES;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_ws_pools[dev] = pool;
  }
  *out = g_ws_pools[dev];
  return cudaSuccess;
}

cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t stream) {
  cudaMemPool_t pool = nullptr;
  const cudaError_t e = workspace_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

void ws_free(void* p, cudaStream_t stream) {
  if (p) cudaFreeAsync(p, stream);
}

cudaError_t ensure_smem(const void* kernel, unsigned smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_smem_done.count({kernel, dev})) return cudaSuccess;
  // the largest size any launch of this kernel may ask for
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    // raise to the device maximum once so later, larger requests need no update
    int mx = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) {
      mx -= (int)fa.sharedSizeBytes;
      if (mx >= (int)smem &&
          cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) ==
              cudaSuccess)
        g_smem_done.insert({kernel, dev});
    }
    cudaGetLastError();
  }
  return e;
}

int current_device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

// cuMemGetAddressRange through the runtime's driver entry-point query, so
// the library needs no link-time dependency on the driver library.
typedef int (*AddrRangeFn)(unsigned long long* base, size_t* size, unsigned long long ptr);
static AddrRangeFn address_range_fn() {
  static AddrRangeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (AddrRangeFn)p;
    cudaGetLastError();
  });
  return fn;
}

// cuPointerGetAttribute, looked up the same way.
typedef int (*PtrAttrFn)(void* data, int attribute, unsigned long long ptr);
static PtrAttrFn pointer_attribute_fn() {
  static PtrAttrFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PtrAttrFn)p;
    cudaGetLastError();
  });
  return fn;
}

// [p, p + bytes) lies inside one page-locked host allocation that the
// current device can address; *dev receives the device-side address of p.
static bool pinned_host_range(const void* p, uint64_t bytes, void** dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
  PtrAttrFn f = pointer_attribute_fn();
  if (!f) return false;
  unsigned long long start = 0;
  size_t size = 0;
  const int kRangeStart = 11, kRangeSize = 12;  // CU_POINTER_ATTRIBUTE_RANGE_{START_ADDR,SIZE}
  if (f(&start, kRangeStart, (unsigned long long)(uintptr_t)p) != 0 ||
      f(&size, kRangeSize, (unsigned long long)(uintptr_t)p) != 0)
    return false;
  if ((unsigned long long)(uintptr_t)p < start ||
      (unsigned long long)(uintptr_t)p + bytes > start + size)
    return false;
  *dev = a.devicePointer;
  return true;
}

brev_status check_device_range(const void* p, uint64_t bytes, const char* what) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_INVALID_ARG, "%s (%p) is not known to CUDA: %s", what, p,
                     cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return set_error(BREV_ERR_INVALID_ARG, "%s (%p) is not device memory", what, p);
  int dev = 0;
  cudaGetDevice(&dev);
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return set_error(BREV_ERR_INVALID_ARG, "%s (%p) belongs to device %d, current device is %d",
                     what, p, a.device, dev);
  if (AddrRangeFn fn = address_range_fn()) {
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, (unsigned long long)(uintptr_t)p) == 0) {
      const unsigned long long lo = (unsigned long long)(uintptr_t)p;
      if (lo + bytes > base + size)
        return set_error(BREV_ERR_INVALID_ARG,
                         "%s: %llu bytes at %p run past the end of its allocation "
                         "(%zu bytes at 0x%llx)",
                         what, (unsigned long long)bytes, p, size, base);
    }
  }
  return BREV_OK;
}

// -------------------------------------------------------- shape table --
static const ShapeEntry* table_for(int E, int* n) {
  switch (E) {
    case 16: *n = g_shapes_e16_n; return g_shapes_e16;
    case 8: *n = g_shapes_e8_n; return g_shapes_e8;
    case 4: *n = g_shapes_e4_n; return g_shapes_e4;
    case 2:
    case 1: *n = g_shapes_e21_n; return g_shapes_e21;
  }
  *n = 0;
  return nullptr;
}

static const ShapeEntry* find_shape(int E, int W, int bx, int bz, int kind, int order = 0) {
  int n = 0;
  const ShapeEntry* t = table_for(E, &n);
  for (int i = 0; i < n; ++i)
    if (t[i].E == E && t[i].W == W && t[i].bx == bx && t[i].bz == bz && t[i].kind == kind &&
        t[i].order == order)
      return &t[i];
  return nullptr;
}

// Built-in square tile exponents: tiles of 8-32 KiB whose rows are
// 256-512 bytes, chosen before any tuning.
static int default_b(int E, bool inplace) {
  switch (E) {
    case 16: return 5;              // 512 B rows, 16 KiB tile
    case 8: return inplace ? 5 : 6;  // 256 B / 512 B rows
    case 4: return 6;               // 256 B rows, 16 KiB tile
    case 2: return 7;
    case 1: return 8;
  }
  return 0;
}

// tuned (bx, bz, order) per element size, in-place flag and k; bx = 0: not tuned
static int8_t g_tuned[5][2][BREV_MAX_LOG2N + 1][3];
static double g_tuned_gbs[5][2][BREV_MAX_LOG2N + 1];
// tuned batched tile exponent + 1 per element size and k (0: not tuned);
// read without the lock on every array of a batched call
static std::atomic<int8_t> g_tuned_batched[5][BREV_MAX_LOG2N + 1];
// tuned stage count of a batch whose largest stage is an array (k, E) (0: not tuned)
static std::atomic<int8_t> g_tuned_batched_stages[5][BREV_MAX_LOG2N + 1];
// tuned staging of the array's tile rows + 1 (0: not tuned)
static std::atomic<int8_t> g_tuned_batched_copy[5][BREV_MAX_LOG2N + 1];
// tuned consumer warps per CTA (0: not tuned)
static std::atomic<int8_t> g_tuned_batched_warps[5][BREV_MAX_LOG2N + 1];
static double g_tuned_batched_gbs[5][BREV_MAX_LOG2N + 1];

int tuned_batched_b(int k, int E) {
  if (k < 0 || k > BREV_MAX_LOG2N || !valid_E(E)) return -1;
  return (int)g_tuned_batched[e_index(E)][k].load(std::memory_order_relaxed) - 1;
}

int tuned_batched_stages(int k, int E) {
  if (k < 0 || k > BREV_MAX_LOG2N || !valid_E(E)) return 0;
  return (int)g_tuned_batched_stages[e_index(E)][k].load(std::memory_order_relaxed);
}

int tuned_batched_warps(int k, int E) {
  if (k < 0 || k > BREV_MAX_LOG2N || !valid_E(E)) return 0;
  return (int)g_tuned_batched_warps[e_index(E)][k].load(std::memory_order_relaxed);
}

int tuned_batched_copy(int k, int E) {
  if (k < 0 || k > BREV_MAX_LOG2N || !valid_E(E)) return -1;
  return (int)g_tuned_batched_copy[e_index(E)][k].load(std::memory_order_relaxed) - 1;
}

struct Choice {
  bool small;
  const ShapeEntry* entry;
  int pipe_b = 0;  // > 0: in place on the TMA pipeline with 2^b x 2^b tiles (order 2)
};

static Choice choose_default(int k, int E, bool inplace, bool vec16);

static Choice choose(int k, int E, bool inplace, bool vec16) {
  const int bmin = b_min_for(E);
  if (k < 2 * bmin) return {true, nullptr};
  const int kind = inplace ? 1 : 0;
  if (vec16) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int8_t* t = g_tuned[e_index(E)][kind][k];
    if (t[2] == 2 && inplace && t[0] == t[1] && pipeline_shape_ok(k, E, t[0]))
      return {false, nullptr, t[0]};
    if (t[0] > 0 && t[1] > 0 && t[0] + t[1] <= k)
      if (const ShapeEntry* s = find_shape(E, 16, t[0], t[1], kind, t[2])) return {false, s};
  }
  return choose_default(k, E, inplace, vec16);
}

// The built-in shape, ignoring the tuned table.
static Choice choose_default(int k, int E, bool inplace, bool vec16) {
  const int bmin = b_min_for(E);
  if (k < 2 * bmin) return {true, nullptr};
  const int kind = inplace ? 1 : 0;
  const int W = vec16 ? 16 : E;
  for (int b = std::min(default_b(E, inplace), k / 2); b >= bmin; --b)
    if (const ShapeEntry* s = find_shape(E, W, b, b, kind)) return {false, s};
  // element-wide path compiles only the narrowest shapes
  for (int b = bmin; 2 * b <= k; ++b)
    if (const ShapeEntry* s = find_shape(E, W, b, b, kind)) return {false, s};
  return {false, nullptr};
}

// Launch with programmatic stream serialisation: the kernel's CTAs may
// start while the previous kernel in the stream finishes, and wait for it
// themselves (pdl_wait) before touching global memory.
cudaError_t launch_pdl(const void* kern, unsigned grid, unsigned threads, void** args,
                       unsigned smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, kern, args);
}

static brev_status launch_choice(const Choice& c, void* dst, const void* src, int k, int E,
                                 cudaStream_t stream) {
  if (c.pipe_b > 0) return bitrev_inplace_pipelined(dst, k, E, c.pipe_b, stream);
  cudaError_t e;
  if (c.small) {
    const void* kern = small_kernel(E);
    const unsigned smem = (unsigned)E << k;
    char* d = (char*)dst;
    const char* s = (const char*)src;
    void* args[] = {(void*)&d, (void*)&s, (void*)&k};
    e = launch_pdl(kern, 1, 256, args, smem, stream);
    if (e != cudaSuccess) return cuda_error(e, "small-array kernel launch");
    note_launch();
    return BREV_OK;
  }
  const ShapeEntry* t = c.entry;
  if (!t) return set_error(BREV_ERR_UNSUPPORTED, "no compiled tile shape for k=%d E=%d", k, E);
  e = ensure_smem(t->kernel, t->smem);
  if (e != cudaSuccess) return cuda_error(e, "shared-memory limit");
  if (t->kind == 0) {
    const unsigned long long grid = 1ull << (k - t->bx - t->bz);
    char* d = (char*)dst;
    const char* s = (const char*)src;
    void* args[] = {(void*)&d, (void*)&s, (void*)&k};
    e = launch_pdl(t->kernel, (unsigned)grid, t->threads, args, t->smem, stream);
  } else {
    const int w = k - 2 * t->bx;
    const unsigned long long grid = (unsigned long long)count_lt(w) + count_self(w);
    char* d = (char*)dst;
    void* args[] = {(void*)&d, (void*)&k};
    e = launch_pdl(t->kernel, (unsigned)grid, t->threads, args, t->smem, stream);
  }
  if (e != cudaSuccess) return cuda_error(e, "tile kernel launch");
  note_launch();
  return BREV_OK;
}

brev_status launch_single(void* dst, const void* src, int k, int E, cudaStream_t stream) {
  const bool inplace = dst == src;
  if (inplace && k <= 1) return BREV_OK;  // identity
  const bool vec16 = (((uintptr_t)dst | (uintptr_t)src) % 16) == 0;
  return launch_choice(choose(k, E, inplace, vec16), dst, src, k, E, stream);
}

void preload_single(int k, int E, bool inplace) {
  if (!valid_E(E) || k < 0 || k > BREV_MAX_LOG2N || (inplace && k <= 1)) return;
  const Choice c = choose(k, E, inplace, true);
  if (c.pipe_b > 0) {
    preload_batched();
    return;
  }
  const void* kern = c.small ? small_kernel(E) : (c.entry ? c.entry->kernel : nullptr);
  cudaFuncAttributes fa;
  if (kern && cudaFuncGetAttributes(&fa, kern) != cudaSuccess) cudaGetLastError();
}

static brev_status check_common(int k, int E) {
  if (!valid_E(E))
    return set_error(BREV_ERR_INVALID_ARG, "elem_bytes=%d (must be 1, 2, 4, 8 or 16)", E);
  if (k < 0 || k > BREV_MAX_LOG2N)
    return set_error(BREV_ERR_INVALID_ARG, "log2n=%d outside [0, %d]", k, BREV_MAX_LOG2N);
  return BREV_OK;
}

static brev_status check_pair(void* dst, const void* src, int k, int E) {
  brev_status s = check_common(k, E);
  if (s != BREV_OK) return s;
  if (!dst || !src) return set_error(BREV_ERR_INVALID_ARG, "NULL data pointer");
  if ((uintptr_t)dst % E || (uintptr_t)src % E)
    return set_error(BREV_ERR_ALIGNMENT, "pointers must be aligned to elem_bytes=%d", E);
  const uint64_t bytes = (uint64_t)E << k;
  if (dst != src) {
    const uint64_t d = (uintptr_t)dst, sr = (uintptr_t)src;
    if (d < sr + bytes && sr < d + bytes)
      return set_error(BREV_ERR_OVERLAP, "source and destination overlap partially");
  }
  s = check_device_range(src, bytes, "source");
  if (s != BREV_OK) return s;
  if (dst != src) s = check_device_range(dst, bytes, "destination");
  return s;
}

brev_status validate_batch_items(const BatchItem* items, int count) {
  std::vector<std::pair<uint64_t, uint64_t>> ranges;
  ranges.reserve(count);
  for (int i = 0; i < count; ++i) {
    const BatchItem& it = items[i];
    brev_status s = check_common(it.k, it.E);
    if (s != BREV_OK) return set_error(s, "array %d: %s", i, t_last_error.c_str());
    if (!it.ptr) return set_error(BREV_ERR_INVALID_ARG, "array %d: NULL pointer", i);
    if ((uintptr_t)it.ptr % it.E)
      return set_error(BREV_ERR_ALIGNMENT, "array %d: pointer not aligned to %d bytes", i, it.E);
    const uint64_t bytes = (uint64_t)it.E << it.k;
    s = check_device_range(it.ptr, bytes, "array");
    if (s != BREV_OK) return set_error(s, "array %d: %s", i, t_last_error.c_str());
    ranges.push_back({(uint64_t)(uintptr_t)it.ptr, bytes});
  }
  std::sort(ranges.begin(), ranges.end());
  for (size_t i = 1; i < ranges.size(); ++i)
    if (ranges[i - 1].first + ranges[i - 1].second > ranges[i].first)
      return set_error(BREV_ERR_OVERLAP, "two arrays of the batch overlap");
  return BREV_OK;
}

}  // namespace brev

using namespace brev;

// ================================================================ C ABI ==
extern "C" {

brev_status brev_permute_to(void* dst, const void* src, int log2n, int elem_bytes, void* stream) {
  BREV_TRACE("brev_permute_to");
  brev_status s = check_pair(dst, src, log2n, elem_bytes);
  if (s != BREV_OK) return s;
  return launch_single(dst, src, log2n, elem_bytes, (cudaStream_t)stream);
}

brev_status brev_permute(void* data, int log2n, int elem_bytes, int in_place, void* stream) {
  BREV_TRACE("brev_permute");
  brev_status s = check_common(log2n, elem_bytes);
  if (s != BREV_OK) return s;
  if (!data) return set_error(BREV_ERR_INVALID_ARG, "NULL data pointer");
  if (in_place) return brev_permute_to(data, data, log2n, elem_bytes, stream);
  char* src = (char*)data;
  s = check_device_range(data, 2 * ((uint64_t)elem_bytes << log2n), "data ([src | dst])");
  if (s != BREV_OK) return s;
  return brev_permute_to(src + ((size_t)elem_bytes << log2n), src, log2n, elem_bytes, stream);
}

brev_status brev_permute_shape(void* dst, const void* src, int log2n, int elem_bytes, int bx,
                               int bz, int order, void* stream) {
  BREV_TRACE("brev_permute_shape");
  brev_status s = check_pair(dst, src, log2n, elem_bytes);
  if (s != BREV_OK) return s;
  const bool inplace = dst == src;
  const bool vec16 = (((uintptr_t)dst | (uintptr_t)src) % 16) == 0;
  Choice c{false, nullptr};
  if (bx == 0 && bz == 0) {
    if (log2n >= 2 * b_min_for(elem_bytes))
      return set_error(BREV_ERR_UNSUPPORTED, "whole-array staging only for k < %d",
                       2 * b_min_for(elem_bytes));
    c.small = true;
  } else {
    if (bx < 0 || bz < 0 || bx + bz > log2n)
      return set_error(BREV_ERR_INVALID_ARG, "tile %dx%d does not fit k=%d", bx, bz, log2n);
    if (inplace && bx != bz)
      return set_error(BREV_ERR_INVALID_ARG, "in-place needs a square tile");
    if (order < 0 || order > 2) return set_error(BREV_ERR_INVALID_ARG, "order=%d", order);
    if (order == 2) {  // the TMA pipeline: in place, 16-byte aligned
      if (!inplace || !vec16 || !pipeline_shape_ok(log2n, elem_bytes, bx))
        return set_error(BREV_ERR_UNSUPPORTED,
                         "order 2 (TMA pipeline) needs in place, 16-byte alignment and a "
                         "pipeline tile (k=%d E=%d b=%d)",
                         log2n, elem_bytes, bx);
      return launch_choice(Choice{false, nullptr, bx}, dst, src, log2n, elem_bytes,
                           (cudaStream_t)stream);
    }
    c.entry = find_shape(elem_bytes, vec16 ? 16 : elem_bytes, bx, bz, inplace ? 1 : 0, order);
    if (!c.entry)
      return set_error(BREV_ERR_UNSUPPORTED, "tile %dx%d order %d not compiled for E=%d (%s path)",
                       bx, bz, order, elem_bytes, vec16 ? "16-byte" : "element-wide");
  }
  if (inplace && log2n <= 1) return BREV_OK;
  return launch_choice(c, dst, src, log2n, elem_bytes, (cudaStream_t)stream);
}

brev_status brev_permute_batched_mixed(void* const* ptr_array, const int* log2n_array,
                                       const int* elem_bytes_array, int count, void* stream) {
  BREV_TRACE("brev_permute_batched_mixed");
  if (count < 0) return set_error(BREV_ERR_INVALID_ARG, "count=%d", count);
  if (count == 0) return BREV_OK;
  if (!ptr_array || !log2n_array || !elem_bytes_array)
    return set_error(BREV_ERR_INVALID_ARG, "NULL host array");
  std::vector<BatchItem> items(count);
  for (int i = 0; i < count; ++i)
    items[i] = BatchItem{ptr_array[i], log2n_array[i], elem_bytes_array[i]};
  brev_status s = validate_batch_items(items.data(), count);
  if (s != BREV_OK) return s;
  return batched_launch(items.data(), count, (cudaStream_t)stream);
}

brev_status brev_permute_batched(void* const* ptr_array, const int* log2n_array, int count,
                                 int elem_bytes, void* stream) {
  BREV_TRACE("brev_permute_batched");
  if (count < 0) return set_error(BREV_ERR_INVALID_ARG, "count=%d", count);
  if (count == 0) return BREV_OK;
  std::vector<int> es(count, elem_bytes);
  return brev_permute_batched_mixed(ptr_array, log2n_array, es.data(), count, stream);
}

brev_status brev_permute_host(void* dst_host, const void* src_host, int log2n, int elem_bytes,
                              void* stream) {
  BREV_TRACE("brev_permute_host");
  brev_status s = check_common(log2n, elem_bytes);
  if (s != BREV_OK) return s;
  if (!dst_host || !src_host) return set_error(BREV_ERR_INVALID_ARG, "NULL host pointer");
  for (const void* p : {(const void*)dst_host, src_host}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return set_error(BREV_ERR_INVALID_ARG, "host pointer %p is not usable", p);
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
      return set_error(BREV_ERR_INVALID_ARG, "%p is device memory; use brev_permute_to", p);
  }
  const uint64_t bytes = (uint64_t)elem_bytes << log2n;
  if (dst_host != src_host) {
    const uint64_t d = (uintptr_t)dst_host, sr = (uintptr_t)src_host;
    if (d < sr + bytes && sr < d + bytes)
      return set_error(BREV_ERR_OVERLAP, "host source and destination overlap partially");
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Both buffers page-locked: the tile kernel reads the source and writes
  // the result in host memory directly (over the coherent CPU-GPU link on
  // Grace-Blackwell), both directions at once, with no device staging.
  void *dsrc = nullptr, *ddst = nullptr;
  if (pinned_host_range(src_host, bytes, &dsrc) && pinned_host_range(dst_host, bytes, &ddst)) {
    s = launch_single(ddst, dsrc, log2n, elem_bytes, st);
    if (s != BREV_OK) return s;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "host-path synchronize");
    return BREV_OK;
  }
  // Otherwise: copy in, permute in device memory, copy out.
  void* buf = nullptr;
  cudaError_t e = ws_alloc(&buf, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "device workspace of %llu bytes: %s",
                     (unsigned long long)bytes, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(buf, src_host, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    s = launch_single(buf, buf, log2n, elem_bytes, st);
    if (s == BREV_OK) {
      e = cudaMemcpyAsync(dst_host, buf, bytes, cudaMemcpyDeviceToHost, st);
    }
  }
  ws_free(buf, st);
  if (e != cudaSuccess) return cuda_error(e, "host-path copy");
  if (s != BREV_OK) return s;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "host-path synchronize");
  return BREV_OK;
}

brev_status brev_tile_shape(int log2n, int elem_bytes, int in_place, int* bx, int* bz,
                            int* order) {
  brev_status s = check_common(log2n, elem_bytes);
  if (s != BREV_OK) return s;
  if (!bx || !bz || !order) return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  Choice c = choose(log2n, elem_bytes, in_place != 0, true);
  if (c.small) {
    *bx = *bz = *order = 0;
    return BREV_OK;
  }
  if (c.pipe_b > 0) {
    *bx = *bz = c.pipe_b;
    *order = 2;
    return BREV_OK;
  }
  if (!c.entry) return set_error(BREV_ERR_UNSUPPORTED, "no tile shape");
  *bx = c.entry->bx;
  *bz = c.entry->bz;
  *order = c.entry->order;
  return BREV_OK;
}

int brev_shape_count(int elem_bytes, int in_place) {
  int n = 0, c = 0;
  const ShapeEntry* t = table_for(elem_bytes, &n);
  const int kind = in_place ? 1 : 0;
  for (int i = 0; i < n; ++i)
    if (t[i].E == elem_bytes && t[i].W == 16 && t[i].kind == kind) ++c;
  int pb[8];
  if (in_place) c += pipeline_shapes(elem_bytes, pb);  // order 2 (TMA pipeline)
  return c;
}

brev_status brev_shape_at(int elem_bytes, int in_place, int i, int* bx, int* bz, int* order) {
  int n = 0, c = 0;
  const ShapeEntry* t = table_for(elem_bytes, &n);
  const int kind = in_place ? 1 : 0;
  if (!bx || !bz || !order) return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  for (int j = 0; j < n; ++j)
    if (t[j].E == elem_bytes && t[j].W == 16 && t[j].kind == kind) {
      if (c == i) {
        *bx = t[j].bx;
        *bz = t[j].bz;
        *order = t[j].order;
        return BREV_OK;
      }
      ++c;
    }
  int pb[8];
  const int np = in_place ? pipeline_shapes(elem_bytes, pb) : 0;
  if (i >= c && i < c + np) {
    *bx = *bz = pb[i - c];
    *order = 2;
    return BREV_OK;
  }
  return set_error(BREV_ERR_INVALID_ARG, "shape index %d out of range", i);
}

void brev_reset_tuning(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  memset(g_tuned, 0, sizeof(g_tuned));
  memset(g_tuned_gbs, 0, sizeof(g_tuned_gbs));
  for (auto& row : g_tuned_batched)
    for (auto& v : row) v.store(0, std::memory_order_relaxed);
  for (auto& row : g_tuned_batched_stages)
    for (auto& v : row) v.store(0, std::memory_order_relaxed);
  for (auto& row : g_tuned_batched_copy)
    for (auto& v : row) v.store(0, std::memory_order_relaxed);
  for (auto& row : g_tuned_batched_warps)
    for (auto& v : row) v.store(0, std::memory_order_relaxed);
  memset(g_tuned_batched_gbs, 0, sizeof(g_tuned_batched_gbs));
}

static bool device_identity(std::string* name, int* sms) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *name = prop.name;
  *sms = prop.multiProcessorCount;
  return true;
}

static brev_status write_cache(const char* path) {
  std::string name;
  int sms = 0;
  if (!device_identity(&name, &sms)) return set_error(BREV_ERR_CUDA, "no device to tag the cache");
  FILE* f = fopen(path, "w");
  if (!f) return set_error(BREV_ERR_INVALID_ARG, "cannot write %s: %s", path, strerror(errno));
  fprintf(f, "{\"format\": \"brev-tune-1\", \"device\": \"%s\", \"sm_count\": %d, \"entries\": [",
          name.c_str(), sms);
  const int Es[5] = {16, 8, 4, 2, 1};
  bool first = true;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int ei = 0; ei < 5; ++ei)
    for (int ip = 0; ip < 2; ++ip)
      for (int k = 0; k <= BREV_MAX_LOG2N; ++k) {
        const int8_t* t = g_tuned[ei][ip][k];
        if (t[0] <= 0) continue;
        fprintf(f, "%s\n  {\"elem_bytes\": %d, \"log2n\": %d, \"in_place\": %d, \"bx\": %d, "
                   "\"bz\": %d, \"order\": %d, \"gbs\": %.1f}",
                first ? "" : ",", Es[ei], k, ip, t[0], t[1], t[2], g_tuned_gbs[ei][ip][k]);
        first = false;
      }
  for (int ei = 0; ei < 5; ++ei)
    for (int k = 0; k <= BREV_MAX_LOG2N; ++k) {
      const int v = g_tuned_batched[ei][k].load(std::memory_order_relaxed);
      if (v <= 0) continue;
      fprintf(f,
              "%s\n  {\"elem_bytes\": %d, \"log2n\": %d, \"batched_b\": %d, "
              "\"batched_stages\": %d, \"batched_copy\": %d, \"batched_warps\": %d, "
              "\"gbs\": %.1f}",
              first ? "" : ",", Es[ei], k, v - 1,
              (int)g_tuned_batched_stages[ei][k].load(std::memory_order_relaxed),
              (int)g_tuned_batched_copy[ei][k].load(std::memory_order_relaxed) - 1,
              (int)g_tuned_batched_warps[ei][k].load(std::memory_order_relaxed),
              g_tuned_batched_gbs[ei][k]);
      first = false;
    }
  fprintf(f, "\n]}\n");
  fclose(f);
  return BREV_OK;
}

// Integer value of "key": in [b, e); returns false if absent.
static bool json_int(const char* b, const char* e, const char* key, long* out) {
  std::string pat = std::string("\"") + key + "\"";
  const char* p = std::search(b, e, pat.begin(), pat.end());
  if (p == e) return false;
  p += pat.size();
  while (p < e && (*p == ' ' || *p == ':' || *p == '\t' || *p == '\n')) ++p;
  char* endp = nullptr;
  long v = strtol(p, &endp, 10);
  if (endp == p) return false;
  *out = v;
  return true;
}

static bool json_str(const char* b, const char* e, const char* key, std::string* out) {
  std::string pat = std::string("\"") + key + "\"";
  const char* p = std::search(b, e, pat.begin(), pat.end());
  if (p == e) return false;
  p += pat.size();
  while (p < e && *p != '"') ++p;
  if (p == e) return false;
  const char* q = ++p;
  while (q < e && *q != '"') ++q;
  *out = std::string(p, q);
  return true;
}

brev_status brev_load_tune_cache(const char* path) {
  if (!path) return set_error(BREV_ERR_INVALID_ARG, "NULL path");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(BREV_ERR_INVALID_ARG, "cannot read %s: %s", path, strerror(errno));
  std::string text;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
  fclose(f);
  const char* b = text.data();
  const char* e = b + text.size();
  const char* ent = strstr(b, "\"entries\"");
  if (!ent) return set_error(BREV_ERR_INVALID_ARG, "%s: no \"entries\"", path);
  std::string fname, dname;
  long fsms = 0;
  int dsms = 0;
  json_str(b, ent, "device", &fname);
  json_int(b, ent, "sm_count", &fsms);
  // without a device the entries are taken as they are (host-only use)
  if (device_identity(&dname, &dsms) && (fname != dname || fsms != dsms)) return BREV_OK;
  int loaded = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  for (const char* p = strchr(ent, '{'); p; p = strchr(p, '{')) {
    const char* q = strchr(p, '}');
    if (!q) break;
    long E = 0, k = -1, ip = -1, bx = 0, bz = 0, order = 0, bb = -1;
    if (json_int(p, q, "batched_b", &bb)) {  // batched tile exponent
      if (json_int(p, q, "elem_bytes", &E) && json_int(p, q, "log2n", &k) && valid_E((int)E) &&
          k >= 0 && k <= BREV_MAX_LOG2N && bb >= 0 && bb <= 7) {
        int cand[8], def = -1;
        const int nc = batched_candidates((int)k, (int)E, cand, &def);
        if (std::find(cand, cand + nc, (int)bb) != cand + nc) {
          g_tuned_batched[e_index((int)E)][k].store((int8_t)(bb + 1), std::memory_order_relaxed);
          long ns = 0;
          int sc[8];
          const int nsc = batched_stage_candidates((int)k, (int)E, (int)bb, sc);
          if (json_int(p, q, "batched_stages", &ns) &&
              std::find(sc, sc + nsc, (int)ns) != sc + nsc)
            g_tuned_batched_stages[e_index((int)E)][k].store((int8_t)ns,
                                                             std::memory_order_relaxed);
          long cp = -1;
          if (bb > 0 && json_int(p, q, "batched_copy", &cp) && (cp == 0 || cp == 1))
            g_tuned_batched_copy[e_index((int)E)][k].store((int8_t)(cp + 1),
                                                           std::memory_order_relaxed);
          long nw = 0;
          if (json_int(p, q, "batched_warps", &nw) && (nw == 4 || nw == 8))
            g_tuned_batched_warps[e_index((int)E)][k].store((int8_t)nw,
                                                            std::memory_order_relaxed);
          ++loaded;
        }
      }
      p = q + 1;
      continue;
    }
    if (!json_int(p, q, "order", &order)) order = 0;  // tables written before orders existed
    if (json_int(p, q, "elem_bytes", &E) && json_int(p, q, "log2n", &k) &&
        json_int(p, q, "in_place", &ip) && json_int(p, q, "bx", &bx) &&
        json_int(p, q, "bz", &bz) && valid_E((int)E) && k >= 0 && k <= BREV_MAX_LOG2N &&
        (ip == 0 || ip == 1) && bx > 0 && bz > 0 && bx + bz <= k && (ip == 0 || bx == bz) &&
        (((order == 0 || order == 1) &&
          find_shape((int)E, 16, (int)bx, (int)bz, (int)ip, (int)order)) ||
         (order == 2 && ip == 1 && pipeline_shape_ok((int)k, (int)E, (int)bx)))) {
      int8_t* t = g_tuned[e_index((int)E)][ip][k];
      t[0] = (int8_t)bx;
      t[1] = (int8_t)bz;
      t[2] = (int8_t)order;
      ++loaded;
    }
    p = q + 1;
  }
  return BREV_OK;
}

// Tuning runs print every candidate's time to stderr when BREV_TUNE_VERBOSE
// is set (the cache keeps only the winners).
static bool tune_verbose() {
  const char* v = getenv("BREV_TUNE_VERBOSE");
  return v && *v && strcmp(v, "0") != 0;
}

// Batched tile exponent and stage count per k: time every candidate
// (b, stages) on a batch of equal arrays of 2^k elements (up to 4096 of
// them, at most `budget` bytes in all), R launches back to back, and keep
// the fastest unless the built-in choice is within 3 %.  A batch larger
// than L2 is read from HBM at every launch; smaller batches (short arrays)
// run as they would in a caller's back-to-back use.
static brev_status autotune_batched(int k_min, int k_max, int E, cudaStream_t st,
                                    uint64_t budget, cudaEvent_t e0, cudaEvent_t e1) {
  constexpr int MAX_ARRAYS = 4096;
  constexpr int R = 4;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, budget);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "batched autotune buffer: %s", cudaGetErrorString(e));
  }
  cudaMemsetAsync(buf, 0x3C, budget, st);
  brev_status result = BREV_OK;
  std::vector<BatchItem> items;
  for (int k = std::max(k_min, 2); k <= k_max && result == BREV_OK; ++k) {
    int cand[8], def = -1;
    const int nc = batched_candidates(k, E, cand, &def);
    if (nc < 1 || def < 0) continue;
    const uint64_t bytes = (uint64_t)E << k;
    const int count = (int)std::min<uint64_t>(MAX_ARRAYS, budget / bytes);
    if (count < 1) continue;
    items.assign(count, BatchItem{});
    for (int i = 0; i < count; ++i) items[i] = BatchItem{(char*)buf + (uint64_t)i * bytes, k, E};
    double best = 1e30, def_ms = 0;
    int best_b = -1, best_s = 0, best_c = -1, best_w = 0;
    for (int c = 0; c < nc && result == BREV_OK; ++c) {
      int sc[8];
      const int ns = batched_stage_candidates(k, E, cand[c], sc);
      // (warps, stages, copy) candidates: the built-in choice (0, 0, -1)
      // first, then both CTA shapes with every stage count and either
      // staging (whole arrays: bulk only)
      const int ncopy = cand[c] > 0 ? 2 : 1;
      for (int si = -1; si < 2 * ns * ncopy && result == BREV_OK; ++si) {
        const int warps = si < 0 ? 0 : (si / (ns * ncopy) == 0 ? 4 : 8);
        const int rest = si < 0 ? 0 : si % (ns * ncopy);
        const int stages = si < 0 ? 0 : sc[rest / ncopy];
        const int copy = si < 0 ? -1 : (cand[c] > 0 ? rest % ncopy : 0);
        BatchForce f;
        f.b = cand[c];
        f.stages = stages;
        f.copy = copy;
        f.warps = warps;
        double ms_best = 1e30;
        for (int r = 0; r < 2 + 3 && result == BREV_OK; ++r) {
          if (r >= 2) cudaEventRecord(e0, st);
          for (int j = 0; j < (r >= 2 ? R : 1) && result == BREV_OK; ++j)
            result = batched_launch_forced(items.data(), count, f, st);
          if (result != BREV_OK) break;
          if (r < 2) continue;  // warm-up
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            result = cuda_error(cudaGetLastError(), "batched autotune timing");
            break;
          }
          float m = 0;
          cudaEventElapsedTime(&m, e0, e1);
          ms_best = std::min(ms_best, (double)m / R);
        }
        if (result != BREV_OK) break;
        if (tune_verbose())
          fprintf(stderr,
                  "brev tune batched E=%d k=%d count=%d b=%d warps=%d stages=%d copy=%d: "
                  "%.4f ms %.1f GB/s\n",
                  E, k, count, cand[c], warps, stages, copy, ms_best,
                  2.0 * (double)bytes * count / (ms_best * 1e-3) / 1e9);
        if (cand[c] == def && si < 0) def_ms = ms_best;
        if (ms_best < best) {
          best = ms_best;
          best_b = cand[c];
          best_s = stages;
          best_c = copy;
          best_w = warps;
        }
      }
    }
    if (result != BREV_OK) break;
    if (def_ms > 0 && best > 0.97 * def_ms) {
      best = def_ms;
      best_b = def;
      best_s = 0;
      best_c = -1;
      best_w = 0;
    }
    if (best_b >= 0) {
      g_tuned_batched[e_index(E)][k].store((int8_t)(best_b + 1), std::memory_order_relaxed);
      g_tuned_batched_stages[e_index(E)][k].store((int8_t)best_s, std::memory_order_relaxed);
      g_tuned_batched_copy[e_index(E)][k].store((int8_t)(best_c + 1), std::memory_order_relaxed);
      g_tuned_batched_warps[e_index(E)][k].store((int8_t)best_w, std::memory_order_relaxed);
      g_tuned_batched_gbs[e_index(E)][k] = 2.0 * (double)bytes * count / (best * 1e-3) / 1e9;
    }
  }
  cudaStreamSynchronize(st);
  cudaFree(buf);
  return result;
}

// Time one shape back to back: a CUDA graph of R launches over buffer sets
// carved from `pool` whose footprint together exceeds 3x L2 (each launch
// then reads its source from HBM, as in a caller's stream of permutations
// of different arrays), replayed three times after a warm-up; returns the
// best replay's time per launch in ms, or a negative value on error.
static double time_shape_b2b(const Choice& c, int k, int E, bool inplace, char* pool,
                             uint64_t pool_bytes, uint64_t l2, cudaStream_t st, cudaEvent_t e0,
                             cudaEvent_t e1, brev_status* result) {
  const uint64_t bytes = (uint64_t)E << k;
  const uint64_t foot = inplace ? bytes : 2 * bytes;
  const uint64_t M = std::max<uint64_t>(
      1, std::min<uint64_t>(pool_bytes / foot, (3 * l2 + foot - 1) / foot));
  const double est_s = 2.0 * (double)bytes / 6.5e12 + 1.5e-6;
  const int R = (int)std::max(4.0, std::min(256.0, std::ceil(1e-3 / est_s)));
  auto set = [&](int r, char** dst, char** src) {
    if (M == 1 && !inplace) {  // one set: ping-pong between its halves
      char* a = pool;
      char* b = pool + bytes;
      *src = (r & 1) ? b : a;
      *dst = (r & 1) ? a : b;
      return;
    }
    char* base = pool + (uint64_t)(r % M) * foot;
    *src = base;
    *dst = inplace ? base : base + bytes;
  };
  char *d0, *s0;
  set(0, &d0, &s0);
  *result = launch_choice(c, d0, s0, k, E, st);  // shared-memory limits and pools set up
  if (*result != BREV_OK) return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    *result = cuda_error(cudaGetLastError(), "autotune warm-up");
    return -1;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    *result = cuda_error(e, "autotune capture");
    return -1;
  }
  brev_status s = BREV_OK;
  for (int r = 0; r < R && s == BREV_OK; ++r) {
    char *d, *src;
    set(r, &d, &src);
    s = launch_choice(c, d, src, k, E, st);
  }
  e = cudaStreamEndCapture(st, &g);
  if (s != BREV_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    *result = s != BREV_OK ? s : cuda_error(e, "autotune capture");
    return -1;
  }
  note_launch_adjust(-(int64_t)R);  // counted at each replay below
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *result = cuda_error(e, "autotune graph");
    return -1;
  }
  double best = 1e30;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    e = cudaGraphLaunch(ge, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGraphExecDestroy(ge);
      *result = cuda_error(e != cudaSuccess ? e : cudaGetLastError(), "autotune replay");
      return -1;
    }
    note_launch(R);
    float m = 0;
    cudaEventElapsedTime(&m, e0, e1);
    if (rep > 0) best = std::min(best, (double)m / R);  // the first replay warms up
  }
  cudaGraphExecDestroy(ge);
  return best;
}

brev_status brev_autotune(int k_min, int k_max, int elem_bytes, const char* cache_path) {
  BREV_TRACE("brev_autotune");
  if (!valid_E(elem_bytes)) return set_error(BREV_ERR_INVALID_ARG, "elem_bytes=%d", elem_bytes);
  if (k_min < 0 || k_max > BREV_MAX_LOG2N || k_min > k_max)
    return set_error(BREV_ERR_INVALID_ARG, "k range [%d, %d]", k_min, k_max);
  const int E = elem_bytes;
  const uint64_t max_bytes = (uint64_t)E << k_max;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "autotune stream");
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  // one pool for the rotating buffer sets: the largest array out of place,
  // or 4x L2, whichever is larger
  const uint64_t pool_bytes = std::max<uint64_t>(2 * max_bytes, 4ull * (uint64_t)l2);
  void* pool = nullptr;
  e = cudaMalloc(&pool, pool_bytes);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  brev_status result = BREV_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    result = set_error(BREV_ERR_OOM, "autotune buffers: %s", cudaGetErrorString(e));
  }
  if (result == BREV_OK) {
    cudaMemsetAsync(pool, 0x5A, pool_bytes, st);
    for (int k = k_min; k <= k_max && result == BREV_OK; ++k) {
      if (k < 2 * b_min_for(E)) continue;
      const uint64_t bytes = (uint64_t)E << k;
      for (int ip = 0; ip < 2 && result == BREV_OK; ++ip) {
        int n = 0;
        const ShapeEntry* t = table_for(E, &n);
        double best = 1e30, def_ms = 0;
        int bbx = 0, bbz = 0, bord = 0;
        const ShapeEntry* def = choose_default(k, E, ip != 0, true).entry;
        // the tile kernels (orders 0 and 1), then in place the TMA pipeline
        // (order 2) for each of its tile exponents
        int pb[8];
        const int np = ip ? pipeline_shapes(E, pb) : 0;
        for (int i = 0; i < n + np && result == BREV_OK; ++i) {
          Choice c{false, nullptr};
          int cbx, cbz, cord;
          if (i < n) {
            if (t[i].E != E || t[i].W != 16 || t[i].kind != ip || t[i].bx + t[i].bz > k)
              continue;
            c.entry = &t[i];
            cbx = t[i].bx;
            cbz = t[i].bz;
            cord = t[i].order;
          } else {
            if (!pipeline_shape_ok(k, E, pb[i - n])) continue;
            c.pipe_b = pb[i - n];
            cbx = cbz = pb[i - n];
            cord = 2;
          }
          const double ms = time_shape_b2b(c, k, E, ip != 0, (char*)pool, pool_bytes,
                                           (uint64_t)l2, st, e0, e1, &result);
          if (result != BREV_OK) break;
          if (tune_verbose())
            fprintf(stderr, "brev tune E=%d k=%d %s %dx%d order %d: %.5f ms %.1f GB/s\n", E, k,
                    ip ? "in-place" : "out-of-place", cbx, cbz, cord, ms,
                    2.0 * (double)bytes / (ms * 1e-3) / 1e9);
          if (i < n && &t[i] == def) def_ms = ms;
          if (ms < best) {
            best = ms;
            bbx = cbx;
            bbz = cbz;
            bord = cord;
          }
        }
        if (result != BREV_OK) break;
        // keep the built-in shape unless another one is clearly faster:
        // small arrays are launch-bound and their timings differ by noise
        if (def && def_ms > 0 && best > 0.97 * def_ms) {
          best = def_ms;
          bbx = def->bx;
          bbz = def->bz;
          bord = def->order;
        }
        if (bbx > 0) {
          std::lock_guard<std::mutex> lk(g_mu);
          g_tuned[e_index(E)][ip][k][0] = (int8_t)bbx;
          g_tuned[e_index(E)][ip][k][1] = (int8_t)bbz;
          g_tuned[e_index(E)][ip][k][2] = (int8_t)bord;
          g_tuned_gbs[e_index(E)][ip][k] = 2.0 * (double)bytes / (best * 1e-3) / 1e9;
        }
      }
    }
  }
  if (result == BREV_OK && (E == 4 || E == 8 || E == 16)) {
    cudaStreamSynchronize(st);
    cudaFree(pool);
    pool = nullptr;
    result = autotune_batched(k_min, std::min(k_max, 24), E, st,
                              std::max<uint64_t>(512ull << 20, 4ull * (uint64_t)l2), e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  if (pool) cudaFree(pool);
  cudaStreamDestroy(st);
  if (result == BREV_OK && cache_path) result = write_cache(cache_path);
  return result;
}

brev_status brev_get_device_info(brev_device_info* out) {
  if (!out) return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  memset(out, 0, sizeof(*out));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  snprintf(out->name, sizeof(out->name), "%s", prop.name);
  cudaDeviceGetAttribute(&out->sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&out->l2_bytes, cudaDevAttrL2CacheSize, dev);
  cudaDeviceGetAttribute(&out->mem_clock_khz, cudaDevAttrMemoryClockRate, dev);
  cudaDeviceGetAttribute(&out->mem_bus_bits, cudaDevAttrGlobalMemoryBusWidth, dev);
  cudaDeviceGetAttribute(&out->max_smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  out->nominal_gbs = (double)out->mem_clock_khz * 1e3 * 2.0 * (out->mem_bus_bits / 8.0) / 1e9;
  return BREV_OK;
}

uint64_t brev_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

brev_status brev_workspace_bytes(uint64_t* reserved, uint64_t* used) {
  if (!reserved || !used) return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  *reserved = *used = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < (int)g_ws_pools.size()) pool = g_ws_pools[dev];
  }
  if (!pool) return BREV_OK;
  uint64_t r = 0, u = 0;  // the attributes are 64-bit byte counts
  e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
  if (e != cudaSuccess) return cuda_error(e, "workspace pool attributes");
  *reserved = (uint64_t)r;
  *used = (uint64_t)u;
  return BREV_OK;
}

const char* brev_status_string(brev_status s) {
  switch (s) {
    case BREV_OK: return "BREV_OK";
    case BREV_ERR_INVALID_ARG: return "BREV_ERR_INVALID_ARG";
    case BREV_ERR_ALIGNMENT: return "BREV_ERR_ALIGNMENT";
    case BREV_ERR_OVERLAP: return "BREV_ERR_OVERLAP";
    case BREV_ERR_OOM: return "BREV_ERR_OOM";
    case BREV_ERR_CUDA: return "BREV_ERR_CUDA";
    case BREV_ERR_UNSUPPORTED: return "BREV_ERR_UNSUPPORTED";
  }
  return "BREV_ERR_UNKNOWN";
}

const char* brev_last_error(void) { return t_last_error.c_str(); }

int brev_version(void) { return BREV_VERSION; }

}  // extern "C"
