// Batched in-place permutation of many independent arrays in one persistent
// launch (no counterpart in the paper, whose methods take one array).
//
// Work decomposition: every array contributes units -- its tile pairs and
// self-paired tiles (square tiles of exponent b), or one unit for a small
// array staged whole -- and consecutive units of one array are grouped into
// tickets of `grain` units.  Persistent CTAs (a full wave: SMs x resident
// CTAs) take tickets from a global counter with atomicAdd, find the owning
// array by a warp-parallel search over the descriptors' first-ticket
// indices, and run the units with the same device bodies as the
// single-array kernels.  The only cross-CTA interaction is the ticket
// counter; there are no spin waits.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "brev_device.cuh"
#include "brev_device_rt.cuh"
#include "brev_internal.h"

namespace brev {

struct BatchDesc {
  char* ptr;
  unsigned long long first_ticket;  // tickets [first_ticket, first_ticket + tickets)
  unsigned units;                   // work units of this array
  unsigned grain;                   // units per ticket
  int k;
  int E;
  int b;                            // square tile exponent; 0 = whole array in one CTA
  int pad_;
};

constexpr int BATCH_THREADS = 256;
#ifndef BREV_BATCHED_MIN_CTAS
#define BREV_BATCHED_MIN_CTAS 3  // register cap: 65536 / (256 * 3) = 85 per thread
#endif
#ifndef BREV_BATCHED_BODY_ATTR
#define BREV_BATCHED_BODY_ATTR __noinline__
#endif

// Last descriptor whose first_ticket <= t (descriptors sorted by
// first_ticket, strictly increasing, first one 0).  Run by one full warp:
// each round the 32 lanes probe evenly spaced descriptors and the window
// shrinks ~32x, so 4096 arrays need 3 rounds of one L2 load per lane.
__device__ __forceinline__ int find_array(const BatchDesc* __restrict__ d, int count,
                                          unsigned long long t) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int span = hi - lo;
    const int pos = lo + (int)(((long long)span * lane) >> 5);
    const bool ok = d[pos].first_ticket <= t;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const int last = 31 - __clz(m);
    const int nlo = __shfl_sync(0xffffffffu, pos, last);
    const int nhi = __shfl_sync(0xffffffffu, pos, last < 31 ? last + 1 : 31);
    lo = nlo;
    hi = last < 31 ? nhi : hi;
  }
  return lo;
}

// One body per element size with the tile exponent at run time, each a
// separate (not inlined) function: the kernel's register count is then that
// of the largest body, not of all bodies inlined side by side.
template <int E>
__device__ BREV_BATCHED_BODY_ATTR void run_tiles(char* ptr, int k, int b, unsigned u, uint4* sm) {
  tile_inplace_body_rt<E, 16, BATCH_THREADS>(ptr, k, b, u, sm);
}

template <int E>
__device__ BREV_BATCHED_BODY_ATTR void run_small(char* ptr, int k, uint4* sm) {
  small_body<E>(ptr, ptr, k, BATCH_THREADS, reinterpret_cast<typename ChunkT<E>::type*>(sm));
}

__device__ __forceinline__ void run_unit(const BatchDesc& d, unsigned u, uint4* sm) {
  if (d.b == 0) {
    switch (d.E) {
      case 16: run_small<16>(d.ptr, d.k, sm); break;
      case 8: run_small<8>(d.ptr, d.k, sm); break;
      case 4: run_small<4>(d.ptr, d.k, sm); break;
    }
    return;
  }
  switch (d.E) {
    case 16: run_tiles<16>(d.ptr, d.k, d.b, u, sm); break;
    case 8: run_tiles<8>(d.ptr, d.k, d.b, u, sm); break;
    case 4: run_tiles<4>(d.ptr, d.k, d.b, u, sm); break;
  }
}

__global__ void __launch_bounds__(BATCH_THREADS, BREV_BATCHED_MIN_CTAS)
    k_batched(const BatchDesc* __restrict__ desc, int count, unsigned long long tickets,
              unsigned long long* ticket_ctr) {
  extern __shared__ uint4 smem_u4[];
  __shared__ unsigned long long s_next;
  __shared__ int s_array;
  if (threadIdx.x == 0) s_next = atomicAdd(ticket_ctr, 1ull);
  __syncthreads();
  unsigned long long t = s_next;
  while (t < tickets) {
    if (threadIdx.x < 32) {
      const int a = find_array(desc, count, t);
      if (threadIdx.x == 0) s_array = a;
    }
    __syncthreads();  // s_array written; every thread has read s_next (= t)
    // take the next ticket now: the atomic's round trip overlaps this
    // ticket's units (its value is read after their barriers)
    if (threadIdx.x == 0) s_next = atomicAdd(ticket_ctr, 1ull);
    const BatchDesc d = desc[s_array];
    const unsigned first = (unsigned)(t - d.first_ticket) * d.grain;
    const unsigned last = min(first + d.grain, d.units);
    for (unsigned u = first; u < last; ++u) {
      run_unit(d, u, smem_u4);
      __syncthreads();  // the next unit reuses the shared-memory tiles
    }
    t = s_next;  // written before the barrier that ended the last unit
  }
}

// ------------------------------------------------------------------ host --

// Tile exponents with a body in run_unit (at most 16 KiB tiles, so the
// kernel keeps several CTAs per SM).
static bool batched_shape_ok(int E, int b) {
  switch (E) {
    case 16: return b == 0 || (b >= 3 && b <= 5);
    case 8: return b == 0 || (b >= 4 && b <= 5);
    case 4: return b == 0 || (b >= 5 && b <= 6);
  }
  return false;
}

// Tile exponent for an in-place array in the batched kernel.  Every body
// runs with 256 threads, so the tile should give each thread several
// 16-byte chunks: 16 KiB tiles with 256-512-byte rows (E=16: b=5, E=8:
// b=5, E=4: b=6), smaller only when the array is too short for them; 0
// stages the whole array in one CTA (k < 2 b_min).
static int batched_b(int k, int E) {
  const int bmin = b_min_for(E);
  if (k < 2 * bmin) return 0;
  const int pref = E == 16 ? 5 : (E == 8 ? 5 : 6);
  const int b = std::min(pref, k / 2);
  return batched_shape_ok(E, b) ? b : -1;
}

struct BatchPlanData {
  std::vector<BatchDesc> desc;
  unsigned long long tickets = 0;
  unsigned smem = 0;
  std::vector<BatchItem> fallback;  // arrays run with single-array launches
};

static brev_status build_batch(const BatchItem* items, int count, BatchPlanData* out) {
  struct Tmp {
    BatchDesc d;
    unsigned long long bytes;
  };
  std::vector<Tmp> tmp;
  tmp.reserve(count);
  for (int i = 0; i < count; ++i) {
    const BatchItem& it = items[i];
    if (it.k <= 1) continue;  // identity
    const bool vec = ((uintptr_t)it.ptr % 16) == 0;
    const int b = (it.E == 4 || it.E == 8 || it.E == 16) && vec ? batched_b(it.k, it.E) : -1;
    if (b < 0) {
      out->fallback.push_back(it);
      continue;
    }
    BatchDesc d{};
    d.ptr = (char*)it.ptr;
    d.k = it.k;
    d.E = it.E;
    d.b = b;
    unsigned long long unit_bytes;
    if (b == 0) {
      d.units = 1;
      unit_bytes = (unsigned long long)it.E << it.k;
      out->smem = std::max<unsigned>(out->smem, (unsigned)unit_bytes);
    } else {
      const int w = it.k - 2 * b;
      d.units = count_lt(w) + count_self(w);
      unit_bytes = 2ull * ((unsigned long long)it.E << (2 * b));
      out->smem = std::max<unsigned>(out->smem, (unsigned)unit_bytes);
    }
    // about 256 KiB of tile data per ticket
    const unsigned long long g = std::max<unsigned long long>(1, 262144ull / unit_bytes);
    d.grain = (unsigned)std::min<unsigned long long>(g, d.units);
    tmp.push_back({d, (unsigned long long)it.E << it.k});
  }
  // largest arrays first: the long-running tickets start early and the
  // small ones fill the tail
  std::stable_sort(tmp.begin(), tmp.end(),
                   [](const Tmp& a, const Tmp& b) { return a.bytes > b.bytes; });
  unsigned long long t = 0;
  out->desc.reserve(tmp.size());
  for (auto& x : tmp) {
    x.d.first_ticket = t;
    t += (x.d.units + x.d.grain - 1) / x.d.grain;
    out->desc.push_back(x.d);
  }
  out->tickets = t;
  return BREV_OK;
}

static int batched_grid(unsigned smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, BATCH_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * current_device_sm_count();
}

// Enqueue the ticket reset, the persistent kernel and the per-array
// fallbacks on `stream` (which may be capturing).
static brev_status enqueue_batch(const BatchPlanData& p, const BatchDesc* d_desc,
                                 unsigned long long* d_ticket, cudaStream_t stream) {
  if (!p.desc.empty()) {
    cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_error(e, "ticket reset");
    e = ensure_smem((const void*)k_batched, p.smem);
    if (e != cudaSuccess) return cuda_error(e, "shared-memory limit of the batched kernel");
    const int grid = (int)std::min<unsigned long long>(
        (unsigned long long)batched_grid(p.smem), p.tickets);
    int count = (int)p.desc.size();
    unsigned long long tickets = p.tickets;
    void* args[] = {(void*)&d_desc, (void*)&count, (void*)&tickets, (void*)&d_ticket};
    e = cudaLaunchKernel((const void*)k_batched, dim3(grid), dim3(BATCH_THREADS), args, p.smem,
                         stream);
    if (e != cudaSuccess) return cuda_error(e, "batched kernel launch");
    note_launch();
  }
  for (const BatchItem& it : p.fallback) {
    brev_status s = launch_single(it.ptr, it.ptr, it.k, it.E, stream);
    if (s != BREV_OK) return s;
  }
  return BREV_OK;
}

brev_status batched_launch(const BatchItem* items, int count, cudaStream_t stream) {
  BatchPlanData p;
  brev_status s = build_batch(items, count, &p);
  if (s != BREV_OK) return s;
  if (p.desc.empty()) return enqueue_batch(p, nullptr, nullptr, stream);
  // stream-ordered workspace: descriptors + ticket counter
  const size_t desc_bytes = p.desc.size() * sizeof(BatchDesc);
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, desc_bytes + 64, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "batched workspace of %zu bytes: %s", desc_bytes + 64,
                     cudaGetErrorString(e));
  }
  // pageable source: staged before the call returns
  e = cudaMemcpyAsync(ws, p.desc.data(), desc_bytes, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(ws, stream);
    return cuda_error(e, "descriptor upload");
  }
  auto* d_ticket = reinterpret_cast<unsigned long long*>((char*)ws + ((desc_bytes + 15) / 16) * 16);
  s = enqueue_batch(p, (const BatchDesc*)ws, d_ticket, stream);
  cudaFreeAsync(ws, stream);
  return s;
}

}  // namespace brev

// ------------------------------------------------------------------ plans --
struct brev_plan {
  brev::BatchPlanData data;
  void* d_ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches_per_replay = 0;
  int device = -1;
};

using namespace brev;

extern "C" brev_status brev_plan_create(void* const* ptr_array, const int* log2n_array,
                                        const int* elem_bytes_array, int elem_bytes, int count,
                                        brev_plan** out_plan) {
  if (!out_plan) return set_error(BREV_ERR_INVALID_ARG, "out_plan is NULL");
  *out_plan = nullptr;
  if (count < 0 || (count > 0 && (!ptr_array || !log2n_array)))
    return set_error(BREV_ERR_INVALID_ARG, "bad count or NULL arrays");
  std::vector<BatchItem> items(count);
  for (int i = 0; i < count; ++i) {
    const int E = elem_bytes_array ? elem_bytes_array[i] : elem_bytes;
    items[i] = BatchItem{ptr_array[i], log2n_array[i], E};
  }
  brev_status s = validate_batch_items(items.data(), count);
  if (s != BREV_OK) return s;
  brev_plan* p = new (std::nothrow) brev_plan();
  if (!p) return set_error(BREV_ERR_OOM, "plan allocation");
  cudaGetDevice(&p->device);
  s = build_batch(items.data(), count, &p->data);
  if (s != BREV_OK) {
    delete p;
    return s;
  }
  const size_t desc_bytes = p->data.desc.size() * sizeof(BatchDesc);
  const size_t ticket_off = ((desc_bytes + 15) / 16) * 16;
  cudaError_t e = cudaMalloc(&p->d_ws, ticket_off + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return set_error(BREV_ERR_OOM, "plan workspace: %s", cudaGetErrorString(e));
  }
  if (desc_bytes) {
    e = cudaMemcpy(p->d_ws, p->data.desc.data(), desc_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      brev_plan_destroy(p);
      return cuda_error(e, "plan descriptor upload");
    }
  }
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    brev_plan_destroy(p);
    return cuda_error(e, "capture stream");
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    brev_plan_destroy(p);
    return cuda_error(e, "begin capture");
  }
  const uint64_t before = brev_launch_count();
  s = enqueue_batch(p->data, (const BatchDesc*)p->d_ws,
                    (unsigned long long*)((char*)p->d_ws + ticket_off), cs);
  // captured launches run at each replay, not now
  p->launches_per_replay = brev_launch_count() - before;
  note_launch_adjust(-(int64_t)p->launches_per_replay);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (s != BREV_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    brev_plan_destroy(p);
    return s != BREV_OK ? s : cuda_error(e2, "end capture");
  }
  p->graph = g;
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) {
    brev_plan_destroy(p);
    return cuda_error(e, "graph instantiate");
  }
  *out_plan = p;
  return BREV_OK;
}

extern "C" brev_status brev_plan_launch(brev_plan* plan, void* stream) {
  if (!plan || !plan->exec) return set_error(BREV_ERR_INVALID_ARG, "invalid plan");
  cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "graph launch");
  note_launch(plan->launches_per_replay);
  return BREV_OK;
}

extern "C" void brev_plan_destroy(brev_plan* plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->d_ws) cudaFree(plan->d_ws);
  delete plan;
}

// ----------------------------------------------------- no-alloc variant --
// brev_permute_batched_noalloc: the batched launch above for callers that
// cannot allocate device memory.  Its scratch -- the ticket counter and the
// descriptor table that every other batched call places in stream-ordered
// workspace -- lives in the fixed device array below instead.  The array
// is part of the library's module, so every GPU that loads the library
// holds its NOALLOC_SCRATCH_BYTES until the process exits.
namespace brev {

constexpr int NOALLOC_MAX_ARRAYS = BREV_NOALLOC_MAX_ARRAYS;
constexpr size_t NOALLOC_DESC_OFFSET = 256;  // ticket counter in the first 256 bytes
constexpr size_t NOALLOC_SCRATCH_BYTES =
    NOALLOC_DESC_OFFSET + (size_t)NOALLOC_MAX_ARRAYS * sizeof(BatchDesc);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Host code cannot use g_noalloc_scratch as a device address (its name in
// host code is only a stand-in), so the address is looked up once per
// device with that device current and cached here.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];

static brev_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return set_error(BREV_ERR_UNSUPPORTED, "device %d beyond the no-alloc table", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress of the scratch array");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return BREV_OK;
}

// Host-side staging in one fixed static block (guarded by g_noalloc_mu for
// the whole call): nothing is allocated on the host either.
struct NoallocHost {
  BatchDesc desc[NOALLOC_MAX_ARRAYS];
  BatchItem fallback[NOALLOC_MAX_ARRAYS];
  unsigned long long bytes[NOALLOC_MAX_ARRAYS];
  int order[NOALLOC_MAX_ARRAYS];
  uint64_t lo[NOALLOC_MAX_ARRAYS], len[NOALLOC_MAX_ARRAYS];
  int range_order[NOALLOC_MAX_ARRAYS];
  BatchDesc sorted[NOALLOC_MAX_ARRAYS];
};
static NoallocHost g_noalloc_host;
static std::mutex g_noalloc_call_mu;

}  // namespace brev

extern "C" brev_status brev_permute_batched_noalloc(void* const* ptr_array,
                                                    const int* log2n_array,
                                                    const int* elem_bytes_array, int count,
                                                    void* stream) {
  if (count < 0) return set_error(BREV_ERR_INVALID_ARG, "count=%d", count);
  if (count > NOALLOC_MAX_ARRAYS)
    return set_error(BREV_ERR_INVALID_ARG,
                     "count=%d exceeds the %d arrays the fixed scratch of "
                     "brev_permute_batched_noalloc holds",
                     count, NOALLOC_MAX_ARRAYS);
  if (count == 0) return BREV_OK;
  if (!ptr_array || !log2n_array || !elem_bytes_array)
    return set_error(BREV_ERR_INVALID_ARG, "NULL host array");
  std::lock_guard<std::mutex> call_lock(g_noalloc_call_mu);
  NoallocHost& h = g_noalloc_host;
  cudaStream_t st = (cudaStream_t)stream;
  // argument checks, array by array, then pairwise overlap on sorted ranges
  for (int i = 0; i < count; ++i) {
    const BatchItem it{ptr_array[i], log2n_array[i], elem_bytes_array[i]};
    if (!(it.E == 1 || it.E == 2 || it.E == 4 || it.E == 8 || it.E == 16))
      return set_error(BREV_ERR_INVALID_ARG, "array %d: elem_bytes=%d", i, it.E);
    if (it.k < 0 || it.k > BREV_MAX_LOG2N)
      return set_error(BREV_ERR_INVALID_ARG, "array %d: log2n=%d", i, it.k);
    if (!it.ptr) return set_error(BREV_ERR_INVALID_ARG, "array %d: NULL pointer", i);
    if ((uintptr_t)it.ptr % it.E)
      return set_error(BREV_ERR_ALIGNMENT, "array %d: pointer not aligned to %d bytes", i, it.E);
    brev_status s = check_device_range(it.ptr, (uint64_t)it.E << it.k, "array");
    if (s != BREV_OK) return s;
    h.lo[i] = (uint64_t)(uintptr_t)it.ptr;
    h.len[i] = (uint64_t)it.E << it.k;
    h.range_order[i] = i;
  }
  std::sort(h.range_order, h.range_order + count,
            [&h](int a, int b) { return h.lo[a] < h.lo[b]; });
  for (int i = 1; i < count; ++i) {
    const int a = h.range_order[i - 1], b = h.range_order[i];
    if (h.lo[a] + h.len[a] > h.lo[b])
      return set_error(BREV_ERR_OVERLAP, "two arrays of the batch overlap");
  }
  // descriptors (the same decomposition as brev_permute_batched_mixed)
  int nd = 0, nf = 0;
  unsigned smem = 0;
  for (int i = 0; i < count; ++i) {
    const BatchItem it{ptr_array[i], log2n_array[i], elem_bytes_array[i]};
    if (it.k <= 1) continue;
    const bool vec = ((uintptr_t)it.ptr % 16) == 0;
    const int b = (it.E == 4 || it.E == 8 || it.E == 16) && vec ? batched_b(it.k, it.E) : -1;
    if (b < 0) {
      h.fallback[nf++] = it;
      continue;
    }
    BatchDesc d{};
    d.ptr = (char*)it.ptr;
    d.k = it.k;
    d.E = it.E;
    d.b = b;
    unsigned long long unit_bytes;
    if (b == 0) {
      d.units = 1;
      unit_bytes = (unsigned long long)it.E << it.k;
    } else {
      const int w = it.k - 2 * b;
      d.units = count_lt(w) + count_self(w);
      unit_bytes = 2ull * ((unsigned long long)it.E << (2 * b));
    }
    smem = std::max<unsigned>(smem, (unsigned)unit_bytes);
    const unsigned long long g = std::max<unsigned long long>(1, 262144ull / unit_bytes);
    d.grain = (unsigned)std::min<unsigned long long>(g, d.units);
    h.desc[nd] = d;
    h.bytes[nd] = (unsigned long long)it.E << it.k;
    h.order[nd] = nd;
    ++nd;
  }
  if (nd > 0) {
    std::sort(h.order, h.order + nd, [&h](int a, int b) {
      return h.bytes[a] != h.bytes[b] ? h.bytes[a] > h.bytes[b] : a < b;
    });
    unsigned long long tickets = 0;
    for (int i = 0; i < nd; ++i) {
      BatchDesc d = h.desc[h.order[i]];
      d.first_ticket = tickets;
      tickets += (d.units + d.grain - 1) / d.grain;
      h.sorted[i] = d;
    }
    void* scratch = nullptr;
    brev_status s = noalloc_scratch(&scratch);
    if (s != BREV_OK) return s;
    auto* d_ticket = reinterpret_cast<unsigned long long*>(scratch);
    auto* d_desc = reinterpret_cast<const BatchDesc*>((char*)scratch + NOALLOC_DESC_OFFSET);
    // the array keeps the previous call's contents: upload this call's
    // descriptors and zero the ticket counter, in stream order
    cudaError_t e = cudaMemcpyAsync((void*)d_desc, h.sorted, (size_t)nd * sizeof(BatchDesc),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "descriptor upload (no-alloc)");
    e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "ticket reset (no-alloc)");
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute((const void*)k_batched,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_error(e, "shared-memory limit (no-alloc)");
    }
    const int grid = (int)std::min<unsigned long long>((unsigned long long)batched_grid(smem),
                                                       tickets);
    int cnt = nd;
    void* args[] = {(void*)&d_desc, (void*)&cnt, (void*)&tickets, (void*)&d_ticket};
    e = cudaLaunchKernel((const void*)k_batched, dim3(grid), dim3(BATCH_THREADS), args, smem,
                         st);
    if (e != cudaSuccess) return cuda_error(e, "batched kernel launch (no-alloc)");
    note_launch();
  }
  for (int i = 0; i < nf; ++i) {
    brev_status s = launch_single(h.fallback[i].ptr, h.fallback[i].ptr, h.fallback[i].k,
                                  h.fallback[i].E, st);
    if (s != BREV_OK) return s;
  }
  return BREV_OK;
}
