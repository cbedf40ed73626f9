// Batched in-place permutation of many independent arrays in one persistent
// launch (no counterpart in the paper, whose methods take one array).
//
// Work decomposition: every array contributes units -- its tile pairs and
// self-paired tiles (square tiles of exponent b), or one unit for a small
// array staged whole -- and consecutive units of one array are grouped into
// tickets of `grain` units.  Persistent CTAs (a full wave: SMs x resident
// CTAs) take tickets from a global counter with atomicAdd and find the
// owning array by a warp-parallel search over the descriptors'
// first-ticket indices.  The only cross-CTA interaction is the ticket
// counter; inside a CTA, a producer warp and the consumer warps hand
// shared-memory stages to each other through mbarriers, every wait
// bounded (about a second, then counted in g_batched_wait_timeouts).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "brev_async.cuh"
#include "brev_device.cuh"
#include "brev_internal.h"
#include "brev_trace.h"
#include "brev_transpose_units.cuh"

namespace brev {

struct BatchDesc {
  char* ptr;
  unsigned long long first_ticket;  // tickets [first_ticket, first_ticket + tickets)
  unsigned units;                   // work units covered: [unit0, unit0 + units)
  unsigned grain;                   // units per ticket
  int k;                            // BATCH_BITREV: log2 n; BATCH_TRANSPOSE: log2 of the side
  int E;
  int b;                            // square tile exponent; 0 = whole array in one CTA
  int mode;                         // BATCH_BITREV or BATCH_TRANSPOSE
  unsigned unit0;                   // first unit of the array this descriptor covers
  int copy;                         // tile rows staged by BATCH_COPY_BULK or BATCH_COPY_CHUNKS
};
// An array's units may be spread over several consecutive descriptors with
// different grains (finer tickets near the end of a batch).
static_assert(sizeof(BatchDesc) == 48, "descriptor layout (the no-alloc scratch is sized by it)");
// Descriptor modes: in-place bit reversal of 2^k elements (units: tile
// pairs (y, rev y) then self-paired tiles), or in-place transposition of a
// 2^k x 2^k matrix (units: tile pairs (tr, tc), tr < tc, and diagonal
// tiles, in blocked order).  Both stage one tile or a pair of tiles per
// unit; they differ only in which tiles and in the row and column maps
// (reversal vs identity).
constexpr int BATCH_BITREV = 0;
constexpr int BATCH_TRANSPOSE = 1;
// How the producer warp stages a unit's tile rows: one bulk copy (TMA) per
// row, or the row's 16-byte chunks spread over the warp's lanes as
// per-thread asynchronous copies.  The bulk copy engine takes about one
// request per 30 SM cycles whatever its size, so rows of 256 bytes or less
// (4- and 8-byte elements) cap a batch at ~5.3-5.8 TB/s that way on GB300;
// chunks have no per-row cost.  Whole small arrays (b = 0) always go as one
// bulk copy.
constexpr int BATCH_COPY_BULK = 0;
constexpr int BATCH_COPY_CHUNKS = 1;

// Built-in staging of an array's tile rows: chunks for rows narrower than
// 512 bytes (where the bulk copy engine's per-request cost binds), bulk
// copies otherwise.
__host__ __device__ inline int batched_copy_default(int E, int b) {
  return b > 0 && (E << b) < 512 ? BATCH_COPY_CHUNKS : BATCH_COPY_BULK;
}


constexpr int BATCH_THREADS = 256;  // consumer threads of the resident serving kernel's CTA
#ifndef BREV_BATCHED_TICKET_BYTES
#define BREV_BATCHED_TICKET_BYTES 262144
#endif
constexpr unsigned long long BATCH_TICKET_BYTES = BREV_BATCHED_TICKET_BYTES;
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

// ----------------------------------------------- TMA-staged kernel --
// Each unit's tiles are brought into shared memory by bulk asynchronous
// copies (one per tile row of 2^b E contiguous bytes), issued by warp 0 and
// completed on an mbarrier, while all warps store the previous unit: a
// pipeline of BATCH_STAGES stages per CTA that keeps no loaded data in
// registers.
// Shared-memory rows are padded to 2^b E + 16 bytes, and row x of a tile
// lands at row rev_b(x), so the bit reversal of the high field costs
// nothing.  The store phase reads V = 16/E rows of one 16-byte column,
// transposes the V x V block in registers and writes V output rows
// rev_b(z); lanes are ordered so that each quarter-warp's 16-byte reads hit
// eight different bank groups (row pitch / 16 is odd) and each warp writes
// whole 128-byte lines.
#ifndef BREV_BATCHED_STORE_UNROLL
#define BREV_BATCHED_STORE_UNROLL 1
#endif
constexpr int BATCH_STORE_UNROLL = BREV_BATCHED_STORE_UNROLL;
// Pipeline stages per CTA.  The resident serving kernel uses BATCH_STAGES;
// the batched kernel takes its stage count at launch (2 .. BATCH_MAX_STAGES,
// chosen per batch from the stage size, or tuned).
#ifndef BREV_BATCHED_STAGES
#define BREV_BATCHED_STAGES 2
#endif
constexpr int BATCH_STAGES = BREV_BATCHED_STAGES;
constexpr int BATCH_MAX_STAGES = 6;

// Unit staged in one pipeline stage.  nt: 2 = tile pair, 1 = self-paired
// tile, 0 = small array staged whole, -1 = no unit.
struct StageInfo {
  char* a;                    // tile y, or (tr, tc) (the whole array when nt = 0)
  char* r;                    // its partner tile rev(y), or (tc, tr)
  unsigned long long stride;  // tile row stride in bytes
  int E, b, k, nt;
  int rev;                    // 1: bit-reversed row and column maps, 0: identity
  // resident serving only: ring slot of the unit's request (-1 in a batch),
  // the request's unit count and sequence number (completion accounting),
  // and the units this CTA completes for the request with this unit (its
  // ticket's units when this is the ticket's last unit, else 0)
  int slot;
  unsigned req_units;
  unsigned long long seq;
  unsigned count;
};

__host__ __device__ constexpr unsigned padded_row_bytes(int E, int b) {
  return ((unsigned)E << b) + 16u;
}

// Shared-memory bytes one stage needs for a unit of the array (k, E, b).
static __host__ unsigned stage_unit_bytes(int k, int E, int b) {
  const unsigned raw = b == 0 ? ((unsigned)E << k) : 2u * (1u << b) * padded_row_bytes(E, b);
  return (raw + 127u) & ~127u;
}

// Wait timeouts of the bulk-copy pipeline since the library loaded (each
// is one CTA that gave up on a copy after about a second).
__device__ unsigned g_batched_wait_timeouts;

// Producer warp: stage unit u of array d into `buf`.  Lane 0 publishes
// the unit's description in `info`, then arrives on `full` with the
// unit's byte count (the arrival releases the description to the
// consumers, who read it after the phase completes); all lanes then issue
// the row copies, which complete on `full`.
__device__ __forceinline__ void issue_unit(const BatchDesc& d, unsigned u, StageInfo* info,
                                           unsigned char* buf, uint64_t* full, int slot = -1,
                                           unsigned long long seq = 0, unsigned count = 0) {
  const int lane = threadIdx.x & 31;
  StageInfo s;
  s.E = d.E;
  s.b = d.b;
  s.k = d.k;
  s.rev = d.mode == BATCH_BITREV;
  s.slot = slot;
  s.req_units = d.units;
  s.seq = seq;
  s.count = count;
  if (d.b == 0) {
    const uint32_t bytes = (uint32_t)d.E << d.k;
    s.a = s.r = d.ptr;
    s.stride = 0;
    s.nt = 0;
    if (lane == 0) {
      *info = s;
      mbar_arrive_expect_tx(full, bytes);
      bulk_g2s(buf, d.ptr, bytes, full);
    }
    return;
  }
  const int b = d.b;
  if (d.mode == BATCH_BITREV) {
    const int wy = d.k - 2 * b;
    const uint32_t npairs = count_lt(wy);
    uint32_t y, ry;
    if (u < npairs) {
      y = unrank_lt(u, wy);
      ry = rev_bits(y, wy);
      s.nt = 2;
    } else {
      y = unrank_self(u - npairs, wy);
      ry = y;
      s.nt = 1;
    }
    s.stride = (unsigned long long)d.E << (d.k - b);
    s.a = d.ptr + ((uint64_t)y << b) * d.E;
    s.r = d.ptr + ((uint64_t)ry << b) * d.E;
  } else {  // transposition of a 2^k x 2^k matrix
    const uint32_t T = 1u << (d.k - b);
    const uint32_t npairs = T * (T - 1) / 2;
    uint32_t tr, tc;
    if (T >= 8) {
      s.nt = blocked_upper(u, T, tr, tc);
    } else if (u < npairs) {
      unrank_upper(u, tr, tc);
      s.nt = 2;
    } else {
      tr = tc = u - npairs;
      s.nt = 1;
    }
    s.stride = (unsigned long long)d.E << d.k;
    s.a = d.ptr + (((uint64_t)tr << (b + d.k)) + ((uint64_t)tc << b)) * d.E;
    s.r = d.ptr + (((uint64_t)tc << (b + d.k)) + ((uint64_t)tr << b)) * d.E;
  }
  const uint32_t rowb = (uint32_t)d.E << b;
  const uint32_t pitch = padded_row_bytes(d.E, b);
  const int rows = 1 << b;
  if (d.copy == BATCH_COPY_CHUNKS) {
    // chunk q: tile t, row x, 16-byte chunk c (consecutive lanes take
    // consecutive chunks of a row, so each warp instruction reads whole
    // rows); the lanes' copies complete on `full`, then lane 0's arrival
    // (which also publishes the unit's description) ends the phase's count
    const int log_cpr = __ffs((int)(rowb >> 4)) - 1;  // rowb / 16 is a power of two
    const int chunks = s.nt * (rows << log_cpr);
    for (int q = lane; q < chunks; q += 32) {
      const int c = q & ((1 << log_cpr) - 1);
      const int tx = q >> log_cpr;
      const int t = tx >> b, x = tx & (rows - 1);
      const uint32_t X = s.rev ? rev_bits((uint32_t)x, b) : (uint32_t)x;
      cp_async16(buf + (uint32_t)t * rows * pitch + X * pitch + (uint32_t)c * 16,
                 (t ? s.r : s.a) + (uint64_t)x * s.stride + (uint32_t)c * 16);
    }
    cp_async_mbar_arrive(full);
    __syncwarp();
    if (lane == 0) {
      *info = s;
      mbar_arrive(full);
    }
    return;
  }
  if (lane == 0) {
    *info = s;
    mbar_arrive_expect_tx(full, (uint32_t)s.nt * rows * rowb);
  }
  __syncwarp();
  for (int q = lane; q < s.nt * rows; q += 32) {
    const int t = q >> b, x = q & (rows - 1);
    const uint32_t X = s.rev ? rev_bits((uint32_t)x, b) : (uint32_t)x;
    bulk_g2s(buf + (uint32_t)t * rows * pitch + X * pitch,
             (t ? s.r : s.a) + (uint64_t)x * s.stride, rowb, full);
  }
}

// Store one staged 2^b x 2^b tile (rows at pitch P, row X = rev(x), or x
// when rev = 0) into the destination tile: output row rev(z) (or z),
// column X.
template <int E, int NTHR>
__device__ __forceinline__ void store_staged_tile(const unsigned char* sm, char* dst,
                                                  uint64_t stride, int b, uint32_t pitch,
                                                  int rev) {
  constexpr int V = 16 / E;
  constexpr int LOG_V = ilog2c(V);
  const int log_c = b - LOG_V;
  const int cmask = (1 << log_c) - 1;
  const int units = 1 << (2 * log_c);
#pragma unroll BATCH_STORE_UNROLL
  for (int q = threadIdx.x; q < units; q += NTHR) {
    const int cl = q & (V - 1);
    const int rest = q >> LOG_V;
    const int d = rest & cmask;
    const int c = ((rest >> log_c) << LOG_V) | cl;
    uint4 blk[V], out[V];
#pragma unroll
    for (int j = 0; j < V; ++j)
      blk[j] = *reinterpret_cast<const uint4*>(sm + (uint32_t)(d * V + j) * pitch + c * 16);
    xpose<E, 16>(blk, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const uint32_t z = (uint32_t)(c * V + e);
      const uint32_t Z = rev ? rev_bits(z, b) : z;
      gstore<16>(dst + (uint64_t)Z * stride + (unsigned)d * 16, out[e]);
    }
  }
}

template <int E, int NTHR>
__device__ BREV_BATCHED_BODY_ATTR void store_staged_unit(const unsigned char* sm, char* a,
                                                        char* r, uint64_t stride, int b, int k,
                                                        int nt, int rev) {
  using C = typename ChunkT<E>::type;
  if (nt == 0) {  // small array: out[j] = in[rev j], coalesced writes
    const uint32_t n = 1u << k;
    for (uint32_t j = threadIdx.x; j < n; j += NTHR)
      gstore<E>(a + (uint64_t)j * E,
                *reinterpret_cast<const C*>(sm + (size_t)rev_bits(j, k) * E));
    return;
  }
  const uint32_t pitch = padded_row_bytes(E, b);
  store_staged_tile<E, NTHR>(sm, r, stride, b, pitch, rev);  // tile a's data into tile r
  if (nt == 2) store_staged_tile<E, NTHR>(sm + ((uint32_t)pitch << b), a, stride, b, pitch, rev);
}

// CTA shape of the batched kernel: CW consumer warps (threads 0 .. 32 CW - 1)
// and one producer warp after them.  Stage p serves units p, p + S, p + 2S,
// ... (S = `stages`).  full[p] completes when the unit's copies have landed
// (one producer arrival plus the bytes); empty[p] completes when all CW
// consumer warps have read the stage.  No block-wide barrier after the
// set-up: each consumer warp moves on as soon as its own share of a unit
// is stored.  Two shapes are compiled: 8 consumer warps at up to 3 CTAs per
// SM and 4 at up to 6; the launch picks one (tuned per (k, E), else 4).
// On GB300 the 4-warp shape moved complex<float> batches from 5.9-6.3 to
// 6.6 TB/s and float32 ones by 3 %, and matched 8 warps on complex<double>.
constexpr int BATCH_CONSUMER_WARPS = BATCH_THREADS / 32;  // resident serving kernel
constexpr int BATCH_BLOCK = BATCH_THREADS + 32;
template <int CW> struct BatchShape {
  static constexpr int THREADS = 32 * CW;       // consumer threads
  static constexpr int BLOCK = THREADS + 32;    // + the producer warp
  static constexpr int MIN_CTAS = CW >= 8 ? BREV_BATCHED_MIN_CTAS : 2 * BREV_BATCHED_MIN_CTAS;
};

// count > 0: descriptors desc[0..count) in global memory; count = 0: the
// single descriptor `one`, passed by value.
template <int CW>
__global__ void __launch_bounds__(BatchShape<CW>::BLOCK, BatchShape<CW>::MIN_CTAS)
    k_batched(const BatchDesc* __restrict__ desc, int count, const BatchDesc one,
              unsigned long long tickets, unsigned long long* ticket_ctr,
              unsigned stage_bytes, int stages) {
  constexpr int NTHR = BatchShape<CW>::THREADS;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[BATCH_MAX_STAGES], empty[BATCH_MAX_STAGES];
  __shared__ StageInfo info[BATCH_MAX_STAGES];
  const int tid = threadIdx.x, lane = tid & 31;
  const unsigned S = (unsigned)stages;  // 2 .. BATCH_MAX_STAGES (checked by the host)
  if (tid == 0) {
    for (unsigned i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], CW);
    }
    mbar_init_fence();
  }
  __syncthreads();  // barriers initialised

  if (tid >= NTHR) {
    // ---- producer warp: tickets -> units -> bulk copies
    int a = -1;
    unsigned u = 0, ulast = 0;
    BatchDesc d{};
    // lane 0 holds the next ticket's number; its atomic is read only when
    // the current ticket runs out
    unsigned long long pending = 0;
    if (lane == 0) pending = atomicAdd(ticket_ctr, 1ull);
    unsigned i = 0, st = 0, round = 0;  // st = i mod S, round = i div S
    bool ok = true;
#pragma unroll 1
    for (;; ++i, st = st + 1 == S ? 0 : st + 1, round += st == 0) {
      if (i >= S) {  // wait until every consumer warp has read the stage
        ok = mbar_wait_bounded(&empty[st], (round - 1) & 1);
        if (!ok) break;
        fence_proxy_async_smem();
      }
      bool more = true;
      if (a >= 0 && u + 1 < ulast) {
        ++u;
      } else {
        const unsigned long long t = __shfl_sync(0xffffffffu, pending, 0);
        if (t >= tickets) {
          more = false;
        } else {
          if (count > 0) {
            a = find_array(desc, count, t);
            d = desc[a];
          } else {
            a = 0;
            d = one;
          }
          u = d.unit0 + (unsigned)(t - d.first_ticket) * d.grain;
          ulast = min(u + d.grain, d.unit0 + d.units);
          if (lane == 0) pending = atomicAdd(ticket_ctr, 1ull);
        }
      }
      if (!more) {  // end marker: a phase with no bytes
        if (lane == 0) {
          info[st].nt = -1;
          mbar_arrive(&full[st]);
        }
        break;
      }
      issue_unit(d, u, &info[st], smem + (size_t)st * stage_bytes, &full[st]);
    }
    if (!ok && lane == 0) atomicAdd(&g_batched_wait_timeouts, 1u);
    // the copies of the units still possibly in flight must land before the
    // CTA may exit: units i-S+1 .. i-1, and unit i-S too after a timeout
    // (after the end marker, unit i-S's stage was released and its barrier
    // has moved on to the marker's phase)
    const unsigned back = ok ? S - 1 : S;
    for (unsigned m = 1; m <= back && m <= i; ++m) {
      const unsigned j = i - m;
      mbar_wait_bounded(&full[j % S], (j / S) & 1);
    }
    return;
  }

  // ---- consumer warps
#pragma unroll 1
  for (unsigned i = 0, st = 0, round = 0;; ++i, st = st + 1 == S ? 0 : st + 1, round += st == 0) {
    if (!mbar_wait_bounded(&full[st], round & 1)) {
      if (lane == 0) atomicAdd(&g_batched_wait_timeouts, 1u);
      return;
    }
    const StageInfo s = info[st];
    if (s.nt < 0) return;
    const unsigned char* buf = smem + (size_t)st * stage_bytes;
    switch (s.E) {
      case 16: store_staged_unit<16, NTHR>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev); break;
      case 8: store_staged_unit<8, NTHR>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev); break;
      case 4: store_staged_unit<4, NTHR>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev); break;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

// ------------------------------------------------ resident serving --
// One kernel stays resident for a whole serving run and takes requests
// from page-locked host memory, so no request pays a kernel launch.
//   host:        writes request r into ring slot r % ring (ServeHostReq),
//                then release-stores the request count;
//   dispatcher:  (one warp, CTA 0) acquires the count, copies new requests
//                into the device ring, fills the ticket table (ticket ->
//                slot), then release-stores the published ticket count;
//   producers:   claim a ticket with atomicAdd, wait until it is
//                published, and run its units through the pipeline;
//   consumers:   after storing their share of a unit, count it on the
//                request's slot; the warp whose count completes the
//                request writes seq + 1 into the host's done word.
// Every wait is bounded (idle_ns of device time, then counted in
// g_batched_wait_timeouts); the host's stop word ends the run.
struct ServeDesc {  // device copy of a published request
  char* ptr;
  unsigned long long first_ticket;
  unsigned units, grain;
  int k, E, b, slot;
  unsigned long long seq;
};
struct ServeCtl {  // device memory (256 bytes), zeroed before each launch
  // the claimed counter (atomics) and the polled words sit on different
  // 128-byte lines
  unsigned long long ticket;     // next ticket to claim
  unsigned long long pad0_[15];
  unsigned long long published;  // tickets published by the dispatcher
  int stop;                      // the dispatcher saw the host's stop (or gave up)
  int pad1_;
};
static_assert(sizeof(ServeCtl) <= 256, "serving control block");
struct ServeArgs {
  ServeDesc* d_ring;
  unsigned* d_done;  // per slot: units completed, counted per ticket and CTA
  int* d_treq;       // ticket table: ticket & (ticket_table - 1) -> slot
  ServeCtl* ctl;
  const ServeHostReq* h_ring;
  const ServeHostCtl* h_ctl;
  unsigned long long* h_done;
  unsigned ring, ticket_table, stage_bytes;
  unsigned long long idle_ns;
};

constexpr int SERVE_BLOCK = BATCH_BLOCK + 32;  // consumers, producer, dispatcher

// Ticket sizing of the resident kernel and the producers' longest pause
// between polls of the published ticket count.
#ifndef BREV_SERVE_POLL_MAX_NS
#define BREV_SERVE_POLL_MAX_NS 2048
#endif
#ifndef BREV_SERVE_POLL_NS_PER_TICKET
#define BREV_SERVE_POLL_NS_PER_TICKET 8
#endif
#ifndef BREV_SERVE_TICKETS_PER_CTA
#define BREV_SERVE_TICKETS_PER_CTA 8
#endif
#ifndef BREV_SERVE_MAX_TICKET_BYTES
#define BREV_SERVE_MAX_TICKET_BYTES 65536
#endif
// Tickets of requests admitted while at least BREV_SERVE_BACKLOG_REQUESTS
// requests are in flight: queueing then sets their latency, and larger
// tickets (fewer claims and descriptor lookups per byte) raise the
// throughput the backlog drains at.  (Counting outstanding tickets instead
// switched on behind every single 512 MB request and coarsened its tail.)
#ifndef BREV_SERVE_BACKLOG_TICKET_BYTES
#define BREV_SERVE_BACKLOG_TICKET_BYTES 262144
#endif
#ifndef BREV_SERVE_BACKLOG_REQUESTS
#define BREV_SERVE_BACKLOG_REQUESTS 16
#endif


// Dispatcher warp: host ring -> device ring and ticket table.
__device__ void serve_dispatch(const ServeArgs& A) {
  const int lane = threadIdx.x & 31;
  unsigned long long seen = 0, last = global_ns();
  for (;;) {
    unsigned long long n = 0;
    if (lane == 0) n = ld_acquire_sys(&A.h_ctl->requests);
    n = __shfl_sync(0xffffffffu, n, 0);
    __syncwarp();  // orders the lanes' reads below after lane 0's acquire
    if (n > seen) {
      unsigned long long published = 0;
      for (unsigned long long r = seen; r < n; ++r) {
        const unsigned slot = (unsigned)(r & (A.ring - 1));
        const volatile ServeHostReq* hr = A.h_ring + slot;
        ServeDesc sd;
        sd.ptr = hr->ptr;
        sd.units = hr->units;
        sd.grain = hr->grain;
        sd.k = hr->k;
        sd.E = hr->E;
        sd.b = hr->b;
        sd.seq = hr->seq;
        sd.first_ticket = hr->first_ticket;
        sd.slot = (int)slot;
        const unsigned tickets = (sd.units + sd.grain - 1) / sd.grain;
        if (lane == 0) {
          A.d_ring[slot] = sd;
          A.d_done[slot] = 0;
        }
        for (unsigned t = lane; t < tickets; t += 32)
          A.d_treq[(sd.first_ticket + t) & (A.ticket_table - 1)] = (int)slot;
        published = sd.first_ticket + tickets;
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release_gpu(&A.ctl->published, published);
      seen = n;
      last = global_ns();
      continue;
    }
    int stop = 0;
    if (lane == 0) stop = ld_acquire_sys(&A.h_ctl->stop);
    stop = __shfl_sync(0xffffffffu, stop, 0);
    const bool idle = global_ns() - last > A.idle_ns;
    if (stop || idle) {
      if (lane == 0) {
        if (!stop) atomicAdd(&g_batched_wait_timeouts, 1u);
        st_release_gpu(&A.ctl->stop, 1);
      }
      return;
    }
  }
}

// A ticket taken by a producer, with its request's descriptor.
struct ServeTicket {
  BatchDesc d;
  unsigned u, ulast;  // units [u, ulast) of the request
  int slot;
  unsigned long long seq;
};

// Read ticket t's request (ticket table, then device ring) into `x`; the
// caller has acquired a published count above t.  Whole warp.
__device__ __forceinline__ void serve_read_ticket(const ServeArgs& A, unsigned long long t,
                                                  ServeTicket& x) {
  __syncwarp();  // the lanes' reads below come after lane 0's acquire
  // read through L2 (a slot's previous request may sit in this SM's L1)
  const int sl = __ldcg(A.d_treq + (t & (A.ticket_table - 1)));
  const ServeDesc* p = A.d_ring + sl;
  BatchDesc& d = x.d;
  d.ptr = (char*)__ldcg((const unsigned long long*)&p->ptr);
  d.first_ticket = __ldcg(&p->first_ticket);
  d.units = __ldcg(&p->units);
  d.grain = __ldcg(&p->grain);
  d.k = __ldcg(&p->k);
  d.E = __ldcg(&p->E);
  d.b = __ldcg(&p->b);
  d.mode = BATCH_BITREV;
  d.unit0 = 0;
  d.copy = batched_copy_default(d.E, d.b);
  x.seq = __ldcg(&p->seq);
  x.slot = sl;
  x.u = (unsigned)(t - d.first_ticket) * d.grain;
  x.ulast = min(x.u + d.grain, d.units);
  // the request's buffer may hold an earlier request's stores (generic
  // proxy), made visible through the acquire chain; the copies that read it
  // are async-proxy operations
  fence_proxy_async_global();
}

// Producer: claim the next ticket and wait until it is published.
// Returns 1 with `x` set, 0 at the end of the run, -1 after idle_ns
// without it being published or the run ending.
__device__ __forceinline__ int serve_next_ticket(const ServeArgs& A, ServeTicket& x) {
  const int lane = threadIdx.x & 31;
  unsigned long long t = 0;
  int status = 0;
  if (lane == 0) {
    t = atomicAdd(&A.ctl->ticket, 1ull);
    const unsigned long long t0 = global_ns();
    for (;;) {
      const unsigned long long p = ld_acquire_gpu(&A.ctl->published);
      if (p > t) {
        status = 1;
        break;
      }
      if (ld_acquire_gpu(&A.ctl->stop)) {  // published is final once stop is set
        status = ld_acquire_gpu(&A.ctl->published) > t ? 1 : 0;
        break;
      }
      if (global_ns() - t0 > A.idle_ns) {
        status = -1;
        break;
      }
      // the holders of the next few tickets poll often, later ones less
      // (hundreds of producers wait at once; their polls share two L2 lines)
      const unsigned long long dist = t - p;
      __nanosleep((unsigned)min(64ull + dist * BREV_SERVE_POLL_NS_PER_TICKET,
                                (unsigned long long)BREV_SERVE_POLL_MAX_NS));
    }
  }
  status = __shfl_sync(0xffffffffu, status, 0);
  if (status <= 0) return status;
  t = __shfl_sync(0xffffffffu, t, 0);
  serve_read_ticket(A, t, x);
  return 1;
}

__global__ void __launch_bounds__(SERVE_BLOCK, BREV_BATCHED_MIN_CTAS)
    k_serve(const ServeArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[BATCH_STAGES], empty[BATCH_STAGES];
  __shared__ StageInfo info[BATCH_STAGES];
  __shared__ unsigned stored[BATCH_STAGES];  // consumer warps done with each stage, counted up
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < BATCH_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], BATCH_CONSUMER_WARPS);
      stored[i] = 0;
    }
    mbar_init_fence();
  }
  __syncthreads();  // barriers initialised (every warp takes part before the roles split)

  if (warp == BATCH_CONSUMER_WARPS + 1) {  // dispatcher (CTA 0 only)
    if (blockIdx.x == 0) serve_dispatch(A);
    return;
  }
  if (warp == BATCH_CONSUMER_WARPS) {  // producer
    ServeTicket cur;  // the ticket being run
    cur.slot = -1;
    cur.u = cur.ulast = 0;
    unsigned i = 0, done_in_ticket = 0;
    bool ok = true, marker = false;
#pragma unroll 1
    for (;; ++i) {
      const int st = i % BATCH_STAGES;
      if (i >= BATCH_STAGES) {
        ok = mbar_wait_bounded(&empty[st], (i / BATCH_STAGES - 1) & 1);
        if (!ok) break;
        fence_proxy_async_smem();
      }
      int more = 1;
      if (cur.slot >= 0 && cur.u + 1 < cur.ulast) {
        ++cur.u;
      } else {
        more = serve_next_ticket(A, cur);
        if (more < 0) ok = false;
        done_in_ticket = 0;
      }
      if (more <= 0) {  // end marker: a phase with no bytes
        if (lane == 0) {
          info[st].nt = -1;
          mbar_arrive(&full[st]);
        }
        marker = true;
        break;
      }
      ++done_in_ticket;
      issue_unit(cur.d, cur.u, &info[st], smem + (size_t)st * A.stage_bytes, &full[st],
                 cur.slot, cur.seq, cur.u + 1 == cur.ulast ? done_in_ticket : 0u);
    }
    if (!ok && lane == 0) atomicAdd(&g_batched_wait_timeouts, 1u);
    // as in k_batched: the copies still in flight land before the CTA
    // exits; after an end marker, unit i-S's barrier has moved on to the
    // marker's phase and is not waited on
    const unsigned back = marker ? BATCH_STAGES - 1 : BATCH_STAGES;
    for (unsigned m = 1; m <= back && m <= i; ++m) {
      const unsigned j = i - m;
      mbar_wait_bounded(&full[j % BATCH_STAGES], (j / BATCH_STAGES) & 1);
    }
    return;
  }
  // consumers
#pragma unroll 1
  for (unsigned i = 0;; ++i) {
    const int st = i % BATCH_STAGES;
    if (!mbar_wait_bounded(&full[st], (i / BATCH_STAGES) & 1)) {
      if (lane == 0) atomicAdd(&g_batched_wait_timeouts, 1u);
      return;
    }
    const StageInfo s = info[st];
    if (s.nt < 0) return;
    const unsigned char* buf = smem + (size_t)st * A.stage_bytes;
    switch (s.E) {
      case 16:
        store_staged_unit<16, BATCH_THREADS>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev);
        break;
      case 8:
        store_staged_unit<8, BATCH_THREADS>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev);
        break;
      case 4:
        store_staged_unit<4, BATCH_THREADS>(buf, s.a, s.r, s.stride, s.b, s.k, s.nt, s.rev);
        break;
    }
    // Completion accounting, one global atomic per ticket and CTA: each
    // warp counts itself on the stage's shared counter (a release at CTA
    // scope: its stores, ordered before by the warp barrier); the last of
    // the 8 has acquired the others' and, on the ticket's last unit, adds
    // the ticket's units to the request's count with a release at GPU
    // scope, which covers every unit of the ticket (each warp stored them
    // before this one).  The warp that completes the request has acquired
    // all the others' and releases the lot to the host.  The stage is
    // released first, so that the producer refills it while the GPU-scope
    // release waits for the stores.  (One acquire-release atomic per warp
    // per unit on the request's one counter -- 16 k on the same word for a
    // 64 MiB request -- had held large requests near 5 TB/s.)
    __syncwarp();
    if (lane == 0) {
      const bool last =
          (atom_add_acq_rel_cta_shared(&stored[st], 1u) + 1u) % BATCH_CONSUMER_WARPS == 0;
      mbar_arrive(&empty[st]);
      if (last && s.count > 0 &&
          atom_add_acq_rel_gpu(&A.d_done[s.slot], s.count) + s.count == s.req_units)
        st_release_sys(&A.h_done[s.slot], s.seq + 1);
    }
  }
}

// ------------------------------------------------------------------ host --

// Tile exponents the batched kernel stages (at most 16 KiB tiles, so two
// stages of a tile pair leave room for three CTAs per SM).
static bool batched_shape_ok(int E, int b) {
  switch (E) {
    case 16: return b == 0 || (b >= 3 && b <= 5);
    case 8: return b == 0 || (b >= 4 && b <= 5);
    case 4: return b == 0 || (b >= 5 && b <= 6);
  }
  return false;
}

// Built-in tile exponent for an in-place array in the batched kernel.
// 256 consumer threads should each get several 16-byte chunks per tile:
// 16 KiB tiles with 256-512-byte rows (E=16: b=5, E=8: b=5, E=4: b=6),
// smaller only when the array is too short for them; 0 stages the whole
// array as one unit (k < 2 b_min).
static int batched_b_default(int k, int E) {
  const int bmin = b_min_for(E);
  if (k < 2 * bmin) return 0;
  const int pref = E == 16 ? 5 : (E == 8 ? 5 : 6);
  const int b = std::min(pref, k / 2);
  return batched_shape_ok(E, b) ? b : -1;
}

// Largest array staged whole (b = 0) at or above 2 b_min: no larger than
// the largest tile-pair stage, so it never raises the kernel's stage size.
constexpr unsigned long long BATCH_WHOLE_MAX_BYTES = 32768;

static bool batched_b_valid(int k, int E, int b) {
  if (!(E == 4 || E == 8 || E == 16) || k <= 1) return false;
  const int bmin = b_min_for(E);
  if (b == 0) return k < 2 * bmin || ((unsigned long long)E << k) <= BATCH_WHOLE_MAX_BYTES;
  return k >= 2 * bmin && b >= bmin && 2 * b <= k && batched_shape_ok(E, b);
}

int batched_candidates(int k, int E, int* out, int* def) {
  int n = 0;
  *def = -1;
  if (!(E == 4 || E == 8 || E == 16) || k <= 1) return 0;
  for (int b = 0; b <= 6; ++b)
    if (batched_b_valid(k, E, b)) out[n++] = b;
  *def = batched_b_default(k, E);
  return n;
}

// Tile exponent of an array in the batched kernel: the tuned one when
// present and valid, else the built-in one; -1 = single-array fallback.
static int batched_b(int k, int E) {
  const int t = tuned_batched_b(k, E);
  if (t >= 0 && batched_b_valid(k, E, t)) return t;
  return batched_b_default(k, E);
}

// Staging of an array (k, E) at tile exponent b: the tuned one for the
// array's usual tile exponent, else the built-in rule.
static int batched_copy(int k, int E, int b) {
  const int t = tuned_batched_copy(k, E);
  if (b > 0 && t >= 0 && b == batched_b(k, E)) return t;
  return batched_copy_default(E, b);
}

// Shared memory of one SM and the batched kernel's static shared memory,
// read once per process (the library serves one GPU model at a time).
static void batched_smem_limits(int* per_sm, int* per_block, int* static_bytes) {
  static int sm = 0, blk = 0, st = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void*)k_batched<8>) != cudaSuccess) {
      cudaGetLastError();
      sm = 228 * 1024;
      blk = 227 * 1024;
      st = 1024;
      return;
    }
    st = (int)fa.sharedSizeBytes;
  });
  *per_sm = sm;
  *per_block = blk;
  *static_bytes = st;
}

// Largest stage count whose shared memory fits one CTA (at least 2).
static int batched_stages_cap(unsigned stage_bytes) {
  int sm, blk, st;
  batched_smem_limits(&sm, &blk, &st);
  const int cap = stage_bytes ? (int)((unsigned)blk / stage_bytes) : BATCH_MAX_STAGES;
  return std::max(2, std::min(BATCH_MAX_STAGES, cap));
}

// CTA shapes of the batched kernel (consumer warps) and their properties.
constexpr int BATCH_WARPS_DEFAULT = 4;
static bool batched_warps_ok(int cw) { return cw == 4 || cw == 8; }
static const void* batched_kernel(int cw) {
  return cw == 8 ? (const void*)k_batched<8> : (const void*)k_batched<4>;
}
static int batched_block(int cw) { return cw == 8 ? BatchShape<8>::BLOCK : BatchShape<4>::BLOCK; }
static int batched_min_ctas(int cw) {
  return cw == 8 ? BatchShape<8>::MIN_CTAS : BatchShape<4>::MIN_CTAS;
}

// Built-in stage count: as many stages as fit while the shape's intended
// CTAs per SM share one SM's shared memory (each CTA also holds its static
// shared memory and the 1 KiB the hardware reserves per CTA),
// 2 .. BATCH_MAX_STAGES.  More stages keep more bytes in flight per CTA:
// one 16 KiB tile pair of 8-byte elements per CTA left the 8-warp kernel
// latency-bound (5.2 TB/s on equal arrays), two 32 KiB pairs do not.
static int batched_stages_default(unsigned stage_bytes, int cw) {
  int sm, blk, st;
  batched_smem_limits(&sm, &blk, &st);
  const int budget = sm / batched_min_ctas(cw) - 1024 - st;
  const int s = stage_bytes ? budget / (int)stage_bytes : BATCH_MAX_STAGES;
  return std::max(2, std::min(batched_stages_cap(stage_bytes), s));
}

int batched_stage_candidates(int k, int E, int b, int* out) {
  if (!batched_b_valid(k, E, b)) return 0;
  const int cap = batched_stages_cap(stage_unit_bytes(k, E, b));
  int n = 0;
  for (int s = 2; s <= cap; ++s) out[n++] = s;
  return n;
}

static int batched_grid(unsigned smem, int cw) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel(cw), batched_block(cw),
                                                    smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * current_device_sm_count();
}

struct BatchPlanData {
  std::vector<BatchDesc> desc;
  unsigned long long tickets = 0;
  unsigned stage_bytes = 0;  // shared memory of one pipeline stage
  int stages = 0;            // pipeline stages per CTA
  int warps = 0;             // consumer warps per CTA (the CTA shape)
  std::vector<BatchItem> fallback;  // arrays run with single-array launches
};

// Tickets shrink once the work left is below BATCH_GUIDE tickets per CTA
// (guided self-scheduling): a ticket of about 256 KiB keeps one CTA busy
// for ~17 us on GB300, so a batch whose last tickets all had that size
// ended on a tail of that length (14 us of a 1 GiB batch's 172 us).
constexpr unsigned long long BATCH_GUIDE = 4;
// Descriptors beyond one per array that the guided split may add.
constexpr int BATCH_EXTRA_DESC = 24;

// Descriptors and tickets of a batch; f.b >= 0 imposes that tile exponent
// on every array (which must accept it), f.stages > 0 the stage count,
// f.copy >= 0 the row staging and f.warps > 0 the CTA shape.
static brev_status build_batch(const BatchItem* items, int count, BatchPlanData* out,
                               const BatchForce& f = BatchForce{}) {
  const int force_b = f.b, force_stages = f.stages, force_copy = f.copy;
  struct Tmp {
    BatchDesc d;
    unsigned long long bytes, unit_bytes;
    unsigned stage;
  };
  std::vector<Tmp> tmp;
  tmp.reserve(count);
  for (int i = 0; i < count; ++i) {
    const BatchItem& it = items[i];
    if (it.k <= 1) continue;  // identity
    const bool vec = ((uintptr_t)it.ptr % 16) == 0;
    int b = (it.E == 4 || it.E == 8 || it.E == 16) && vec ? batched_b(it.k, it.E) : -1;
    if (force_b >= 0) {
      if (!vec || !batched_b_valid(it.k, it.E, force_b))
        return set_error(BREV_ERR_UNSUPPORTED, "array %d (k=%d, E=%d) cannot take b=%d", i,
                         it.k, it.E, force_b);
      b = force_b;
    }
    if (b < 0) {
      out->fallback.push_back(it);
      continue;
    }
    BatchDesc d{};
    d.ptr = (char*)it.ptr;
    d.k = it.k;
    d.E = it.E;
    d.b = b;
    d.copy = b == 0 ? BATCH_COPY_BULK : (force_copy >= 0 ? force_copy : batched_copy(it.k, it.E, b));
    unsigned long long unit_bytes;
    if (b == 0) {
      d.units = 1;
      unit_bytes = (unsigned long long)it.E << it.k;
    } else {
      const int w = it.k - 2 * b;
      d.units = count_lt(w) + count_self(w);
      unit_bytes = 2ull * ((unsigned long long)it.E << (2 * b));
    }
    const unsigned stage = stage_unit_bytes(it.k, it.E, b);
    // the array with the largest stage sets the CTA shape and the stage
    // count (tuned per (k, E), else the built-in ones)
    if (stage > out->stage_bytes) {
      out->stage_bytes = stage;
      const int ts = tuned_batched_stages(it.k, it.E);
      out->stages = ts > 0 ? ts : 0;
      const int tw = tuned_batched_warps(it.k, it.E);
      out->warps = batched_warps_ok(tw) ? tw : 0;
    }
    // about BATCH_TICKET_BYTES of tile data per ticket
    const unsigned long long g =
        std::max<unsigned long long>(1, BATCH_TICKET_BYTES / unit_bytes);
    d.grain = (unsigned)std::min<unsigned long long>(g, d.units);
    tmp.push_back({d, (unsigned long long)it.E << it.k, unit_bytes, stage});
  }
  if (f.warps > 0) out->warps = f.warps;
  if (!batched_warps_ok(out->warps)) out->warps = BATCH_WARPS_DEFAULT;
  if (force_stages > 0) out->stages = force_stages;
  if (out->stages <= 0) out->stages = batched_stages_default(out->stage_bytes, out->warps);
  out->stages = std::min(out->stages, batched_stages_cap(out->stage_bytes));
  // largest arrays first: the long-running tickets start early and the
  // small ones fill the tail
  std::stable_sort(tmp.begin(), tmp.end(),
                   [](const Tmp& a, const Tmp& b) { return a.bytes > b.bytes; });
  // guided ticket sizes: while the work left W exceeds BATCH_GUIDE x CTAs
  // x the ticket's bytes, keep the grain; below, halve it (down to one
  // unit), splitting an array across descriptors where its grain changes
  const unsigned long long P =
      tmp.empty() ? 1
                  : (unsigned long long)batched_grid(out->stages * out->stage_bytes, out->warps);
  unsigned long long left = 0;
  for (const auto& x : tmp) left += x.unit_bytes * x.d.units;
  unsigned long long t = 0;
  int extra = 0;
  out->desc.reserve(tmp.size() + BATCH_EXTRA_DESC);
  for (auto& x : tmp) {
    const unsigned long long ub = x.unit_bytes;
    unsigned u = 0;
    while (u < x.d.units) {
      const unsigned long long want = left / (BATCH_GUIDE * P * ub);
      unsigned long long g = x.d.grain;
      while (g > 1 && g > want) g = (g + 1) / 2;
      unsigned long long n = x.d.units - u;
      if (g > 1 && extra < BATCH_EXTRA_DESC) {
        // units at this grain until the work left falls below keep
        const unsigned long long keep = g * BATCH_GUIDE * P * ub;
        const unsigned long long m = (left - keep) / ub + 1;
        n = std::min(n, (m + g - 1) / g * g);
      } else if (g > 1) {
        g = x.d.grain;  // no descriptor left for a split: finish the array as it is
      }
      BatchDesc d = x.d;
      d.unit0 = u;
      d.units = (unsigned)n;
      d.grain = (unsigned)g;
      d.first_ticket = t;
      t += (n + g - 1) / g;
      out->desc.push_back(d);
      if (u > 0) ++extra;
      u += (unsigned)n;
      left -= n * ub;
    }
  }
  out->tickets = t;
  return BREV_OK;
}

// Launch the persistent kernel over `count` descriptors already on the
// device (ticket counter zeroed in stream order before it), with `warps`
// consumer warps per CTA (0: the built-in shape) and `stages` pipeline
// stages (0: the built-in count for the shape and stage size).
static brev_status launch_batched_kernel(const BatchDesc* d_desc, int count,
                                         unsigned long long tickets,
                                         unsigned long long* d_ticket, unsigned stage_bytes,
                                         int stages, int warps, cudaStream_t stream,
                                         const BatchDesc* one = nullptr) {
  BatchDesc one_v{};
  if (one) one_v = *one;
  if (warps <= 0) warps = BATCH_WARPS_DEFAULT;
  if (!batched_warps_ok(warps))
    return set_error(BREV_ERR_INVALID_ARG, "%d consumer warps per CTA", warps);
  if (stages <= 0) stages = batched_stages_default(stage_bytes, warps);
  if (stages < 2 || stages > BATCH_MAX_STAGES || stages > batched_stages_cap(stage_bytes))
    return set_error(BREV_ERR_INVALID_ARG, "stage count %d for stages of %u bytes", stages,
                     stage_bytes);
  const unsigned smem = (unsigned)stages * stage_bytes;
  const void* kern = batched_kernel(warps);
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return cuda_error(e, "shared-memory limit of the batched kernel");
  const int grid =
      (int)std::min<unsigned long long>((unsigned long long)batched_grid(smem, warps), tickets);
  void* args[] = {(void*)&d_desc, (void*)&count, (void*)&one_v, (void*)&tickets,
                  (void*)&d_ticket, (void*)&stage_bytes, (void*)&stages};
  e = cudaLaunchKernel(kern, dim3(grid), dim3(batched_block(warps)), args, smem, stream);
  if (e != cudaSuccess) return cuda_error(e, "batched kernel launch");
  note_launch();
  return BREV_OK;
}

// Enqueue the ticket reset, the persistent kernel and the per-array
// fallbacks on `stream` (which may be capturing).
static brev_status enqueue_batch(const BatchPlanData& p, const BatchDesc* d_desc,
                                 unsigned long long* d_ticket, cudaStream_t stream) {
  if (!p.desc.empty()) {
    cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_error(e, "ticket reset");
    brev_status s = launch_batched_kernel(d_desc, (int)p.desc.size(), p.tickets, d_ticket,
                                          p.stage_bytes, p.stages, p.warps, stream);
    if (s != BREV_OK) return s;
  }
  for (const BatchItem& it : p.fallback) {
    brev_status s = launch_single(it.ptr, it.ptr, it.k, it.E, stream);
    if (s != BREV_OK) return s;
  }
  return BREV_OK;
}

void preload_batched() {
  cudaFuncAttributes fa;
  for (int cw : {4, 8})
    if (cudaFuncGetAttributes(&fa, batched_kernel(cw)) != cudaSuccess) cudaGetLastError();
}

brev_status batched_launch(const BatchItem* items, int count, cudaStream_t stream) {
  return batched_launch_forced(items, count, BatchForce{}, stream);
}

brev_status batched_launch_forced(const BatchItem* items, int count, const BatchForce& f,
                                  cudaStream_t stream) {
  BatchPlanData p;
  brev_status s = build_batch(items, count, &p, f);
  if (s != BREV_OK) return s;
  if (p.desc.empty()) return enqueue_batch(p, nullptr, nullptr, stream);
  // stream-ordered workspace: descriptors + ticket counter
  const size_t desc_bytes = p.desc.size() * sizeof(BatchDesc);
  void* ws = nullptr;
  cudaError_t e = ws_alloc(&ws, desc_bytes + 64, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "batched workspace of %zu bytes: %s", desc_bytes + 64,
                     cudaGetErrorString(e));
  }
  // pageable source: staged before the call returns
  e = cudaMemcpyAsync(ws, p.desc.data(), desc_bytes, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) {
    ws_free(ws, stream);
    return cuda_error(e, "descriptor upload");
  }
  auto* d_ticket = reinterpret_cast<unsigned long long*>((char*)ws + ((desc_bytes + 15) / 16) * 16);
  s = enqueue_batch(p, (const BatchDesc*)ws, d_ticket, stream);
  ws_free(ws, stream);
  return s;
}

// ---------------------------------------- single arrays on the pipeline --
// In-place bit reversal of one array as a one-descriptor launch of the
// batched kernel (descriptor passed by value): the tuner's "TMA pipeline"
// candidate (launch order 2) beside the LSU tile kernels.
bool pipeline_shape_ok(int k, int E, int b) { return b > 0 && batched_b_valid(k, E, b); }

int pipeline_shapes(int E, int* out) {
  int n = 0;
  for (int b = 1; b <= 6; ++b)
    if ((E == 4 || E == 8 || E == 16) && batched_shape_ok(E, b)) out[n++] = b;
  return n;
}

brev_status bitrev_inplace_pipelined(void* data, int k, int E, int b, cudaStream_t stream) {
  if (!pipeline_shape_ok(k, E, b) || ((uintptr_t)data % 16) != 0)
    return set_error(BREV_ERR_UNSUPPORTED, "TMA pipeline: k=%d E=%d b=%d", k, E, b);
  BatchDesc d{};
  d.ptr = (char*)data;
  d.k = k;
  d.E = E;
  d.b = b;
  d.mode = BATCH_BITREV;
  d.copy = batched_copy_default(E, b);
  const int w = k - 2 * b;
  const unsigned long long units = (unsigned long long)count_lt(w) + count_self(w);
  if (units > 0xFFFFFFFFull) return set_error(BREV_ERR_UNSUPPORTED, "too many tile units");
  d.units = (unsigned)units;
  // about 8 tickets per resident CTA (the tail of the last wave stays short)
  const unsigned stage = stage_unit_bytes(k, E, b);
  const int stages = batched_stages_default(stage, BATCH_WARPS_DEFAULT);
  const unsigned long long ctas =
      (unsigned long long)batched_grid(stages * stage, BATCH_WARPS_DEFAULT);
  const unsigned long long unit_bytes = 2ull * ((unsigned long long)E << (2 * b));
  d.grain = (unsigned)std::min<unsigned long long>(
      std::max<unsigned long long>(1, units / (8 * ctas)),
      std::max<unsigned long long>(1, BATCH_TICKET_BYTES / unit_bytes));
  d.first_ticket = 0;
  const unsigned long long tickets = (units + d.grain - 1) / d.grain;
  void* ws = nullptr;
  cudaError_t e = ws_alloc(&ws, 16, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "pipeline workspace: %s", cudaGetErrorString(e));
  }
  auto* d_ticket = reinterpret_cast<unsigned long long*>(ws);
  e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) {
    ws_free(ws, stream);
    return cuda_error(e, "ticket reset");
  }
  brev_status st =
      launch_batched_kernel(nullptr, 0, tickets, d_ticket, stage, stages, 0, stream, &d);
  ws_free(ws, stream);
  return st;
}

size_t batched_ws_bytes(int count) {
  return ((size_t)(std::max(count, 0) + BATCH_EXTRA_DESC) * sizeof(BatchDesc) + 15) / 16 * 16 +
         64;
}

brev_status batched_launch_into(const BatchItem* items, int count, void* ws, size_t ws_bytes,
                                cudaStream_t stream) {
  BatchPlanData p;
  brev_status s = build_batch(items, count, &p);
  if (s != BREV_OK) return s;
  if (p.desc.empty()) return enqueue_batch(p, nullptr, nullptr, stream);
  const size_t desc_bytes = p.desc.size() * sizeof(BatchDesc);
  if (!ws || ((desc_bytes + 15) / 16) * 16 + 64 > ws_bytes)
    return set_error(BREV_ERR_INVALID_ARG, "batched workspace too small");
  // pageable source: staged before the call returns
  cudaError_t e = cudaMemcpyAsync(ws, p.desc.data(), desc_bytes, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_error(e, "descriptor upload");
  auto* d_ticket = reinterpret_cast<unsigned long long*>((char*)ws + ((desc_bytes + 15) / 16) * 16);
  return enqueue_batch(p, (const BatchDesc*)ws, d_ticket, stream);
}

int transpose_pipelined_b(int E) {
  switch (E) {
    case 16: return 5;
    case 8: return 5;
    case 4: return 6;
  }
  return -1;
}

brev_status transpose_inplace_pipelined(void* data, int a, int E, cudaStream_t stream) {
  const int b = transpose_pipelined_b(E);
  if (b < 0 || a < b || ((uintptr_t)data % 16) != 0)
    return set_error(BREV_ERR_UNSUPPORTED, "pipelined transposition: a=%d E=%d", a, E);
  BatchDesc d{};
  d.ptr = (char*)data;
  d.k = a;
  d.E = E;
  d.b = b;
  d.mode = BATCH_TRANSPOSE;
  d.copy = batched_copy_default(E, b);
  const unsigned long long T = 1ull << (a - b);
  const unsigned long long units = T * (T - 1) / 2 + T;
  if (units > 0xFFFFFFFFull)
    return set_error(BREV_ERR_UNSUPPORTED, "too many tile pairs for one launch");
  d.units = (unsigned)units;
  const unsigned long long unit_bytes = 2ull * ((unsigned long long)E << (2 * b));
  d.grain = (unsigned)std::min<unsigned long long>(
      std::max<unsigned long long>(1, BATCH_TICKET_BYTES / unit_bytes), units);
  d.first_ticket = 0;
  const unsigned long long tickets = (units + d.grain - 1) / d.grain;
  // the descriptor travels by value; only the ticket counter needs
  // stream-ordered device memory (so the call can be captured in a graph)
  void* ws = nullptr;
  cudaError_t e = ws_alloc(&ws, 16, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BREV_ERR_OOM, "transposition workspace: %s", cudaGetErrorString(e));
  }
  auto* d_ticket = reinterpret_cast<unsigned long long*>(ws);
  e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) {
    ws_free(ws, stream);
    return cuda_error(e, "ticket reset");
  }
  brev_status st = launch_batched_kernel(nullptr, 0, tickets, d_ticket,
                                         stage_unit_bytes(2 * b, E, b), 0, 0, stream, &d);
  ws_free(ws, stream);
  return st;
}

// ---------------------------------------------- resident serving, host --
// A request's units are spread over about two tickets per resident CTA (a
// request finishes soonest when all CTAs share it), with tickets of one
// unit at least and of about 256 KiB at most.
bool resident_shape(int k, int E, int ctas, bool backlog, int* b, unsigned* units,
                    unsigned* grain) {
  if (!(E == 4 || E == 8 || E == 16) || k <= 1 || k > BREV_MAX_LOG2N) return false;
  const int bb = batched_b(k, E);
  if (bb < 0) return false;
  unsigned long long n_units, unit_bytes;
  if (bb == 0) {
    n_units = 1;
    unit_bytes = (unsigned long long)E << k;
  } else {
    const int w = k - 2 * bb;
    n_units = (unsigned long long)count_lt(w) + count_self(w);
    unit_bytes = 2ull * ((unsigned long long)E << (2 * bb));
  }
  if (n_units > 0x7FFFFFFFull) return false;
  *b = bb;
  *units = (unsigned)n_units;
  if (backlog) {  // the CTAs have work queued: large tickets, fewer claims per byte
    *grain = (unsigned)std::min<unsigned long long>(
        n_units, std::max<unsigned long long>(1, BREV_SERVE_BACKLOG_TICKET_BYTES / unit_bytes));
    return true;
  }
  const unsigned long long max_grain =
      std::max<unsigned long long>(1, BREV_SERVE_MAX_TICKET_BYTES / unit_bytes);
  *grain = (unsigned)std::min<unsigned long long>(
      std::max<unsigned long long>(
          1, n_units / ((unsigned long long)BREV_SERVE_TICKETS_PER_CTA *
                        (unsigned long long)std::max(ctas, 1))),
      max_grain);
  return true;
}

int resident_backlog_requests() { return BREV_SERVE_BACKLOG_REQUESTS; }

// Stage size that holds any unit the resident kernel may meet (every
// (E, b) the batched path accepts, and whole arrays of up to 32 KiB).
static unsigned serve_stage_bytes() {
  unsigned m = (unsigned)BATCH_WHOLE_MAX_BYTES;
  for (int E : {4, 8, 16})
    for (int b = 1; b <= 6; ++b)
      if (batched_shape_ok(E, b)) m = std::max(m, stage_unit_bytes(2 * b, E, b));
  return m;
}

brev_status resident_alloc(ResidentState* st, unsigned ring, unsigned ticket_table) {
  if (!st || ring == 0 || (ring & (ring - 1)) || ticket_table == 0 ||
      (ticket_table & (ticket_table - 1)))
    return set_error(BREV_ERR_INVALID_ARG, "resident ring / ticket table sizes");
  *st = ResidentState{};
  st->ring = ring;
  st->ticket_table = ticket_table;
  cudaError_t e = cudaHostAlloc((void**)&st->h_ring, ring * sizeof(ServeHostReq),
                                cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&st->h_ctl, 256, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&st->h_done, ring * sizeof(unsigned long long),
                      cudaHostAllocMapped | cudaHostAllocPortable);
  const size_t dbytes = 256 + ring * sizeof(ServeDesc) + ring * sizeof(unsigned) +
                        (size_t)ticket_table * sizeof(int);
  if (e == cudaSuccess) e = cudaMalloc(&st->d_mem, dbytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    resident_free(st);
    return set_error(BREV_ERR_OOM, "resident serving state: %s", cudaGetErrorString(e));
  }
  const unsigned smem = BATCH_STAGES * serve_stage_bytes();
  e = ensure_smem((const void*)k_serve, smem);
  int per_sm = 0;
  if (e != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, SERVE_BLOCK, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  st->ctas = per_sm * current_device_sm_count();
  return BREV_OK;
}

void resident_free(ResidentState* st) {
  if (!st) return;
  if (st->h_ring) cudaFreeHost(st->h_ring);
  if (st->h_ctl) cudaFreeHost(st->h_ctl);
  if (st->h_done) cudaFreeHost(st->h_done);
  if (st->d_mem) cudaFree(st->d_mem);
  *st = ResidentState{};
}

brev_status resident_launch(ResidentState* st, cudaStream_t stream,
                            unsigned long long idle_ns) {
  if (!st || !st->d_mem) return set_error(BREV_ERR_INVALID_ARG, "no resident state");
  memset(st->h_ctl, 0, 256);
  memset(st->h_done, 0, st->ring * sizeof(unsigned long long));
  ServeArgs A{};
  char* dm = (char*)st->d_mem;
  A.ctl = (ServeCtl*)dm;
  A.d_ring = (ServeDesc*)(dm + 256);
  A.d_done = (unsigned*)(dm + 256 + st->ring * sizeof(ServeDesc));
  A.d_treq = (int*)(dm + 256 + st->ring * (sizeof(ServeDesc) + sizeof(unsigned)));
  cudaError_t e = cudaHostGetDevicePointer((void**)&A.h_ring, st->h_ring, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&A.h_ctl, st->h_ctl, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&A.h_done, st->h_done, 0);
  if (e != cudaSuccess) return cuda_error(e, "device view of the serving ring");
  A.ring = st->ring;
  A.ticket_table = st->ticket_table;
  A.stage_bytes = serve_stage_bytes();
  A.idle_ns = idle_ns;
  e = cudaMemsetAsync(A.ctl, 0, sizeof(ServeCtl), stream);
  if (e != cudaSuccess) return cuda_error(e, "serving control reset");
  const unsigned smem = BATCH_STAGES * A.stage_bytes;
  e = ensure_smem((const void*)k_serve, smem);
  if (e != cudaSuccess) return cuda_error(e, "shared-memory limit of the serving kernel");
  void* args[] = {(void*)&A};
  e = cudaLaunchKernel((const void*)k_serve, dim3(std::max(st->ctas, 1)), dim3(SERVE_BLOCK),
                       args, smem, stream);
  if (e != cudaSuccess) return cuda_error(e, "serving kernel launch");
  note_launch();
  return BREV_OK;
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
  BREV_TRACE("brev_plan_create");
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

extern "C" brev_status brev_batched_shape(int log2n, int elem_bytes, int* b) {
  if (!b) return set_error(BREV_ERR_INVALID_ARG, "b is NULL");
  if (log2n < 0 || log2n > BREV_MAX_LOG2N)
    return set_error(BREV_ERR_INVALID_ARG, "log2n=%d", log2n);
  const int v = (elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 16) && log2n > 1
                    ? batched_b(log2n, elem_bytes)
                    : -1;
  if (v < 0)
    return set_error(BREV_ERR_UNSUPPORTED,
                     "log2n=%d elem_bytes=%d runs as a single-array launch in a batch", log2n,
                     elem_bytes);
  *b = v;
  return BREV_OK;
}

extern "C" brev_status brev_wait_timeouts(uint64_t* out) {
  if (!out) return set_error(BREV_ERR_INVALID_ARG, "out is NULL");
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_batched_wait_timeouts, sizeof(v));
  if (e != cudaSuccess) return cuda_error(e, "reading the wait-timeout counter");
  *out = v;
  return BREV_OK;
}

extern "C" brev_status brev_plan_launch(brev_plan* plan, void* stream) {
  BREV_TRACE("brev_plan_launch");
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

// Host-side staging in one fixed static block (guarded by g_noalloc_call_mu
// for the whole call): nothing is allocated on the host either.
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
  BREV_TRACE("brev_permute_batched_noalloc");
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
  unsigned stage_bytes = 0;
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
    d.copy = b == 0 ? BATCH_COPY_BULK : batched_copy(it.k, it.E, b);
    unsigned long long unit_bytes;
    if (b == 0) {
      d.units = 1;
      unit_bytes = (unsigned long long)it.E << it.k;
    } else {
      const int w = it.k - 2 * b;
      d.units = count_lt(w) + count_self(w);
      unit_bytes = 2ull * ((unsigned long long)it.E << (2 * b));
    }
    stage_bytes = std::max(stage_bytes, stage_unit_bytes(it.k, it.E, b));
    const unsigned long long g =
        std::max<unsigned long long>(1, BATCH_TICKET_BYTES / unit_bytes);
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
    s = launch_batched_kernel(d_desc, nd, tickets, d_ticket, stage_bytes, 0, 0, st);
    if (s != BREV_OK) return s;
  }
  for (int i = 0; i < nf; ++i) {
    brev_status s = launch_single(h.fallback[i].ptr, h.fallback[i].ptr, h.fallback[i].k,
                                  h.fallback[i].E, st);
    if (s != BREV_OK) return s;
  }
  return BREV_OK;
}
