// Native serving loop: continuous batching of bit-reversal requests over a
// caller-owned device arena (no counterpart in the paper, which permutes one
// array at a time).
//
// Policy (the same as paper_1708_01873_gb300/serve.py, which is the
// reference tested on the CPU):
//   * requests wait in a FIFO; the head is admitted when a slot is free and
//     the first-fit pool over the arena has room for its 2^k * E bytes (the
//     head waits rather than being overtaken, so large requests cannot starve);
//   * every loop iteration takes all admitted requests (at most max_batch)
//     into ONE launch on an idle stream (round robin over n_streams): a batch
//     of one is a single-array launch, larger ones one persistent batched
//     launch;
//   * a CUDA event per batch marks completion; the request's completion time
//     is read on the device clock (elapsed time from a reference event
//     recorded when the run starts) and its memory and slot are released.
// Latency = when the serving thread sees the request complete - arrival
// time (the device-clock completion time is reported beside it).
//
// Resident mode (cfg.resident): the same admission policy, but no launch
// per request.  One kernel (resident_launch) stays on the GPU for the run;
// each admitted request is written into a ring in page-locked host memory
// and published at once; the kernel writes a completion word per request
// into host memory, and latency = when the serving thread sees that word -
// arrival time.  Besides slots and pool memory, admission needs a free ring
// slot and room in the kernel's ticket window (the ticket table maps
// ticket & (table - 1) to a ring slot, so the tickets between the oldest
// request in flight and the newest must fit in the table).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "brev_internal.h"
#include "brev_trace.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pool {
  // first-fit over [0, capacity): free blocks by offset, coalesced on free
  std::map<uint64_t, uint64_t> free_blocks;
  std::map<uint64_t, uint64_t> used;
  uint64_t capacity = 0, in_use = 0, peak = 0;
  static constexpr uint64_t kAlign = 256;

  explicit Pool(uint64_t cap) : capacity(cap) {
    if (cap) free_blocks[0] = cap;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = (std::max<uint64_t>(bytes, 1) + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= need) {
        const uint64_t o = it->first, len = it->second;
        free_blocks.erase(it);
        if (len > need) free_blocks[o + need] = len - need;
        used[o] = need;
        in_use += need;
        peak = std::max(peak, in_use);
        *off = o;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off) {
    auto u = used.find(off);
    if (u == used.end()) return;
    uint64_t o = off, len = u->second;
    used.erase(u);
    in_use -= len;
    auto next = free_blocks.lower_bound(o);
    if (next != free_blocks.end() && o + len == next->first) {
      len += next->second;
      next = free_blocks.erase(next);
    }
    if (next != free_blocks.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += len;
        return;
      }
    }
    free_blocks[o] = len;
  }
};

struct Req {
  uint64_t id;
  int k, E;
  double arrival;  // seconds since the run started
  uint64_t offset = 0;
  double launch = 0, done = 0;
  double seen = 0;  // completion as seen by the serving thread
  int batch = -1;
  bool admitted = false;
};

constexpr unsigned kResidentRing = 4096;
constexpr unsigned kResidentTickets = 1u << 22;
constexpr unsigned long long kResidentIdleNs = 2000000000ull;
constexpr double kResidentStopIdle = 0.5;  // seconds
constexpr double kLivenessCheck = 0.05;    // seconds without progress before asking the stream

struct Inflight {
  cudaEvent_t ev;
  int stream;
  std::vector<size_t> reqs;
};

uint64_t splitmix64(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& state) {  // (0, 1]
  return ((splitmix64(state) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const double pos = p / 100.0 * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace

struct brev_server {
  brev_server_config cfg;
  char* arena = nullptr;
  uint64_t arena_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<void*> ws;  // per stream: descriptor workspace of its batched launches
  size_t ws_bytes = 0;
  std::vector<cudaEvent_t> spare_events;
  int device = 0;
  brev::ResidentState res;  // resident mode only
};

namespace {

// Statistics and trace of a finished run (both modes).
void finish_stats(const std::vector<Req>& reqs, const std::vector<double>& lat_us,
                  const std::vector<double>& queue_us, uint64_t completed, uint64_t bytes_moved,
                  uint64_t batches, uint64_t launches, uint64_t peak_pool, int max_inflight,
                  double wall, brev_server_request* trace, uint64_t trace_capacity,
                  brev_server_stats* out) {
  out->completed = completed;
  out->batches = batches;
  out->launches = launches;
  // lat_us: completion on the device clock (launches) or as seen (resident)
  std::vector<double> host_us;
  host_us.reserve(reqs.size());
  for (const Req& r : reqs)
    if (r.seen > 0) host_us.push_back((r.seen - r.arrival) * 1e6);
  out->p50_us = percentile(host_us, 50);
  out->p99_us = percentile(host_us, 99);
  out->max_us = host_us.empty() ? 0 : *std::max_element(host_us.begin(), host_us.end());
  double sum = 0;
  for (double v : host_us) sum += v;
  out->mean_us = host_us.empty() ? 0 : sum / (double)host_us.size();
  out->queue_p99_us = percentile(queue_us, 99);
  out->device_p50_us = percentile(lat_us, 50);
  out->device_p99_us = percentile(lat_us, 99);
  out->wall_s = wall;
  out->req_per_s = (double)completed / wall;
  out->gbs = (double)bytes_moved / wall / 1e9;
  out->peak_pool_bytes = peak_pool;
  out->max_inflight = max_inflight;
  out->offered = (uint64_t)reqs.size();
  if (trace) {
    for (uint64_t i = 0; i < reqs.size() && i < trace_capacity; ++i) {
      trace[i].offset = reqs[i].offset;
      trace[i].log2n = reqs[i].k;
      trace[i].elem_bytes = reqs[i].E;
      trace[i].batch = reqs[i].batch;
      trace[i].arrival_us = reqs[i].arrival * 1e6;
      trace[i].launch_us = reqs[i].launch * 1e6;
      trace[i].done_us = reqs[i].done * 1e6;
      trace[i].seen_us = reqs[i].seen * 1e6;
    }
  }
}

// Resident mode: see the comment at the top of the file.
brev_status run_resident(brev_server* srv, std::vector<Req>& reqs, int hold_results,
                         brev_server_request* trace, uint64_t trace_capacity,
                         brev_server_stats* out) {
  using namespace brev;
  ResidentState& R = srv->res;
  Pool pool(srv->arena_bytes);
  struct Live {
    size_t req;
    unsigned long long seq, first_ticket;
  };
  std::deque<size_t> waiting;
  std::vector<Live> live;                      // requests in flight
  std::map<unsigned long long, int> firsts;    // first tickets in flight (count)
  std::vector<double> lat_us, queue_us;
  lat_us.reserve(reqs.size());
  queue_us.reserve(reqs.size());
  uint64_t completed = 0, bytes_moved = 0, publications = 0;
  unsigned long long next_seq = 0, tickets = 0;
  int max_inflight = 0;
  brev_status result = BREV_OK, s = BREV_OK;
  const uint64_t launches0 = brev_launch_count();
  cudaStream_t ks = srv->streams[0];

  // the kernel does not wait on other streams: finish earlier device work
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "device synchronize before serving");
  const Clock::time_point t0 = Clock::now();
  auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  // The kernel runs while there is traffic.  After kResidentStopIdle s with
  // nothing in flight or waiting, the host stops it (so its own 2 s limit
  // only fires if this thread stalls); the next request launches it again,
  // with sequence numbers and tickets counted from 0.
  bool running = false;
  double last_busy = 0, last_progress = 0;
  const double idle_stop =
      srv->cfg.idle_stop_ms > 0 ? srv->cfg.idle_stop_ms * 1e-3 : kResidentStopIdle;
  auto stop_kernel = [&]() -> cudaError_t {
    __atomic_store_n(&R.h_ctl->stop, 1, __ATOMIC_RELEASE);
    running = false;
    return cudaStreamSynchronize(ks);
  };

  size_t next_arrival = 0;
  while (result == BREV_OK && (next_arrival < reqs.size() || !waiting.empty() || !live.empty())) {
    const double now = now_s();
    while (next_arrival < reqs.size() && reqs[next_arrival].arrival <= now)
      waiting.push_back(next_arrival++);
    // completions: the kernel wrote seq + 1 into the slot's done word
    for (size_t i = 0; i < live.size();) {
      const unsigned slot = (unsigned)(live[i].seq & (R.ring - 1));
      if (__atomic_load_n(&R.h_done[slot], __ATOMIC_ACQUIRE) != live[i].seq + 1) {
        ++i;
        continue;
      }
      Req& r = reqs[live[i].req];
      r.done = r.seen = now_s();
      last_progress = r.done;
      lat_us.push_back((r.done - r.arrival) * 1e6);
      queue_us.push_back((r.launch - r.arrival) * 1e6);
      bytes_moved += 2 * ((uint64_t)r.E << r.k);
      ++completed;
      if (!hold_results) pool.release(r.offset);
      auto f = firsts.find(live[i].first_ticket);
      if (--f->second == 0) firsts.erase(f);
      live[i] = live.back();
      live.pop_back();
    }
    if (!live.empty() || !waiting.empty()) last_busy = now;
    if (running && live.empty() && waiting.empty() && now - last_busy > idle_stop) {
      e = stop_kernel();
      if (e != cudaSuccess) {
        result = cuda_error(e, "resident serving kernel");
        break;
      }
    }
    // a kernel that ended with work outstanding gave up on a wait; asked
    // only after kLivenessCheck s without progress, so that a healthy run
    // makes no CUDA call between its launch and its stop (a CUDA call can
    // block for tens of milliseconds when the driver is busy elsewhere)
    if (!live.empty() && now - last_progress > kLivenessCheck &&
        cudaStreamQuery(ks) != cudaErrorNotReady) {
      cudaGetLastError();
      result = set_error(BREV_ERR_CUDA,
                         "the resident serving kernel stopped with %zu requests in flight "
                         "(see brev_wait_timeouts)",
                         live.size());
      break;
    }
    // admission and publication
    bool published = false;
    while (!waiting.empty() && (int)live.size() < srv->cfg.max_slots) {
      Req& r = reqs[waiting.front()];
      int b = 0;
      unsigned units = 0, grain = 1;
      // many requests in flight at once: the server is queueing
      const bool backlog = (int)live.size() >= resident_backlog_requests();
      if (!resident_shape(r.k, r.E, R.ctas, backlog, &b, &units, &grain)) {
        result = set_error(BREV_ERR_UNSUPPORTED, "request k=%d E=%d in resident mode", r.k, r.E);
        break;
      }
      const unsigned long long nt = (units + grain - 1) / grain;
      const unsigned long long oldest_seq = live.empty() ? next_seq : [&] {
        unsigned long long m = next_seq;
        for (const Live& l : live) m = std::min(m, l.seq);
        return m;
      }();
      const unsigned long long oldest_ticket = firsts.empty() ? tickets : firsts.begin()->first;
      if (next_seq - oldest_seq >= R.ring) break;  // ring slot still in use
      if (nt > R.ticket_table) {
        result = set_error(BREV_ERR_UNSUPPORTED, "request k=%d E=%d has more tickets than the "
                           "resident kernel's window", r.k, r.E);
        break;
      }
      if (tickets + nt - oldest_ticket > R.ticket_table) break;  // ticket window full
      uint64_t off = 0;
      if (!pool.alloc((uint64_t)r.E << r.k, &off)) {
        if (hold_results && live.empty())
          result = set_error(BREV_ERR_OOM, "arena too small to hold every result of the stream");
        break;
      }
      if (!running) {  // (re)start: nothing is in flight, count from 0
        next_seq = 0;
        tickets = 0;
        s = resident_launch(&R, ks, kResidentIdleNs);
        if (s != BREV_OK) {
          result = s;
          break;
        }
        running = true;
      }
      r.offset = off;
      r.admitted = true;
      r.launch = now_s();
      r.batch = (int)publications;
      const unsigned slot = (unsigned)(next_seq & (R.ring - 1));
      ServeHostReq& h = R.h_ring[slot];
      h.ptr = srv->arena + off;
      h.units = units;
      h.grain = grain;
      h.k = r.k;
      h.E = r.E;
      h.b = b;
      h.seq = next_seq;
      h.first_ticket = tickets;
      live.push_back(Live{waiting.front(), next_seq, tickets});
      ++firsts[tickets];
      tickets += nt;
      ++next_seq;
      waiting.pop_front();
      published = true;
    }
    if (result != BREV_OK) break;
    if (published) {
      last_progress = now_s();
      __atomic_store_n(&R.h_ctl->requests, next_seq, __ATOMIC_RELEASE);
      ++publications;
      max_inflight = std::max(max_inflight, (int)live.size());
    }
  }
  // end of the run: the kernel drains and exits
  e = running ? stop_kernel() : cudaStreamSynchronize(ks);
  const double wall = now_s();
  if (e != cudaSuccess && result == BREV_OK) result = cuda_error(e, "resident serving kernel");
  if (result != BREV_OK) return result;
  finish_stats(reqs, lat_us, queue_us, completed, bytes_moved, publications,
               brev_launch_count() - launches0, pool.peak, max_inflight, wall, trace,
               trace_capacity, out);
  return BREV_OK;
}

}  // namespace

using namespace brev;

extern "C" {

brev_status brev_server_create(const brev_server_config* cfg, void* arena, uint64_t arena_bytes,
                               brev_server** out) {
  if (!out) return set_error(BREV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->max_slots < 1 || cfg->max_batch < 1 || cfg->n_streams < 1 ||
      cfg->n_streams > 64 || (cfg->resident != 0 && cfg->resident != 1) ||
      (cfg->resident && cfg->max_slots > (int)kResidentRing) || cfg->idle_stop_ms < 0)
    return set_error(BREV_ERR_INVALID_ARG, "bad server configuration");
  if (!arena || arena_bytes == 0 || (uintptr_t)arena % 256)
    return set_error(BREV_ERR_INVALID_ARG, "arena must be a 256-byte aligned device buffer");
  brev_status s = check_device_range(arena, arena_bytes, "arena");
  if (s != BREV_OK) return s;
  brev_server* srv = new (std::nothrow) brev_server();
  if (!srv) return set_error(BREV_ERR_OOM, "server allocation");
  srv->cfg = *cfg;
  srv->arena = (char*)arena;
  cudaGetDevice(&srv->device);
  for (int i = 0; i < cfg->n_streams; ++i) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      brev_server_destroy(srv);
      return cuda_error(e, "server stream");
    }
    srv->streams.push_back(st);
    // the stream's batched launches reuse one descriptor workspace (a batch
    // is launched on a stream only once its previous batch has completed)
    void* w = nullptr;
    srv->ws_bytes = batched_ws_bytes(cfg->max_batch);
    e = cudaMalloc(&w, srv->ws_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      brev_server_destroy(srv);
      return set_error(BREV_ERR_OOM, "server workspace: %s", cudaGetErrorString(e));
    }
    srv->ws.push_back(w);
  }
  if (cfg->resident) {
    s = resident_alloc(&srv->res, kResidentRing, kResidentTickets);
    if (s != BREV_OK) {
      brev_server_destroy(srv);
      return s;
    }
  }
  srv->arena_bytes = arena_bytes;
  *out = srv;
  return BREV_OK;
}

void brev_server_destroy(brev_server* srv) {
  if (!srv) return;
  for (cudaStream_t st : srv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (void* w : srv->ws) cudaFree(w);
  for (cudaEvent_t e : srv->spare_events) cudaEventDestroy(e);
  resident_free(&srv->res);
  delete srv;
}

brev_status brev_server_run_poisson(brev_server* srv, uint64_t seed, double rate_per_s,
                                    double seconds, int k_min, int k_max,
                                    const int* elem_bytes, int n_elem_bytes, int hold_results,
                                    brev_server_request* trace, uint64_t trace_capacity,
                                    brev_server_stats* out) {
  BREV_TRACE("brev_server_run_poisson");
  if (!srv || !out) return set_error(BREV_ERR_INVALID_ARG, "NULL server or stats");
  if (!(rate_per_s > 0) || !(seconds > 0) || k_min < 0 || k_max < k_min ||
      k_max > BREV_MAX_LOG2N || !elem_bytes || n_elem_bytes < 1)
    return set_error(BREV_ERR_INVALID_ARG, "bad load description");
  for (int i = 0; i < n_elem_bytes; ++i) {
    const int E = elem_bytes[i];
    if (!(E == 1 || E == 2 || E == 4 || E == 8 || E == 16))
      return set_error(BREV_ERR_INVALID_ARG, "elem_bytes[%d]=%d", i, E);
    if (((uint64_t)E << k_max) > srv->arena_bytes)
      return set_error(BREV_ERR_INVALID_ARG, "largest request exceeds the arena");
  }
  memset(out, 0, sizeof(*out));

  // the arrival stream: exponential gaps, k and E uniform (seeded)
  std::vector<Req> reqs;
  {
    uint64_t st = seed;
    double t = 0;
    for (uint64_t id = 0;; ++id) {
      t += -std::log(uniform01(st)) / rate_per_s;
      if (t >= seconds) break;
      Req r;
      r.id = id;
      r.k = k_min + (int)(splitmix64(st) % (uint64_t)(k_max - k_min + 1));
      r.E = elem_bytes[splitmix64(st) % (uint64_t)n_elem_bytes];
      r.arrival = t;
      reqs.push_back(r);
    }
  }
  if (srv->cfg.resident) {
    for (int i = 0; i < n_elem_bytes; ++i)
      if (!(elem_bytes[i] == 4 || elem_bytes[i] == 8 || elem_bytes[i] == 16))
        return set_error(BREV_ERR_UNSUPPORTED, "resident mode serves 4-, 8- and 16-byte elements");
    return run_resident(srv, reqs, hold_results, trace, trace_capacity, out);
  }
  Pool pool(srv->arena_bytes);
  std::deque<size_t> waiting, admitted;
  std::vector<Inflight> inflight;
  std::vector<bool> busy(srv->cfg.n_streams, false);
  int next_stream = 0, slots = 0, batches = 0, max_inflight = 0;
  std::vector<double> lat_us, queue_us;
  lat_us.reserve(reqs.size());
  queue_us.reserve(reqs.size());
  uint64_t completed = 0, bytes_moved = 0;
  const uint64_t launches0 = brev_launch_count();
  brev_status result = BREV_OK;

  // load every kernel the stream may launch before the clock starts (the
  // first launch of a kernel would otherwise pay its loading, ~2.5 ms)
  for (int i = 0; i < n_elem_bytes; ++i)
    for (int k = k_min; k <= k_max; ++k) preload_single(k, elem_bytes[i], true);
  preload_batched();
  // the server's streams do not wait on other streams: finish all earlier
  // work on the device (e.g. the client writing the arena) before serving
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "device synchronize before serving");
  cudaEvent_t ref;
  e = cudaEventCreate(&ref);
  if (e != cudaSuccess) return cuda_error(e, "reference event");
  cudaEventRecord(ref, srv->streams[0]);
  cudaEventSynchronize(ref);
  const Clock::time_point t0 = Clock::now();
  auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };

  auto get_event = [&](cudaEvent_t* ev) -> cudaError_t {
    if (!srv->spare_events.empty()) {
      *ev = srv->spare_events.back();
      srv->spare_events.pop_back();
      return cudaSuccess;
    }
    return cudaEventCreate(ev);
  };

  size_t next_arrival = 0;
  while (result == BREV_OK &&
         (next_arrival < reqs.size() || !waiting.empty() || !admitted.empty() ||
          !inflight.empty())) {
    const double now = now_s();
    while (next_arrival < reqs.size() && reqs[next_arrival].arrival <= now)
      waiting.push_back(next_arrival++);
    // completions
    for (size_t i = 0; i < inflight.size();) {
      cudaError_t q = cudaEventQuery(inflight[i].ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q != cudaSuccess) {
        result = cuda_error(q, "batch completion");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, ref, inflight[i].ev);
      const double done = ms * 1e-3;
      const double seen = now_s();
      for (size_t ri : inflight[i].reqs) {
        Req& r = reqs[ri];
        r.done = done;
        r.seen = seen;
        lat_us.push_back((done - r.arrival) * 1e6);
        queue_us.push_back((r.launch - r.arrival) * 1e6);
        bytes_moved += 2 * ((uint64_t)r.E << r.k);
        ++completed;
        if (!hold_results) pool.release(r.offset);
        --slots;
      }
      busy[inflight[i].stream] = false;
      srv->spare_events.push_back(inflight[i].ev);
      inflight[i] = inflight.back();
      inflight.pop_back();
    }
    if (result != BREV_OK) break;
    // admission: FIFO, by slots and pool memory
    while (!waiting.empty() && slots < srv->cfg.max_slots) {
      Req& r = reqs[waiting.front()];
      uint64_t off = 0;
      if (!pool.alloc((uint64_t)r.E << r.k, &off)) {
        if (hold_results && inflight.empty() && admitted.empty()) {
          // held results fill the arena and nothing will free it
          result = set_error(BREV_ERR_OOM,
                             "arena too small to hold every result of the stream");
        }
        break;
      }
      r.offset = off;
      r.admitted = true;
      admitted.push_back(waiting.front());
      waiting.pop_front();
      ++slots;
    }
    if (result != BREV_OK) break;
    // launch: everything admitted, on an idle stream
    if (!admitted.empty()) {
      int s = -1;
      for (int j = 0; j < srv->cfg.n_streams; ++j) {
        const int c = (next_stream + j) % srv->cfg.n_streams;
        if (!busy[c]) {
          s = c;
          break;
        }
      }
      if (s >= 0) {
        next_stream = (s + 1) % srv->cfg.n_streams;
        const size_t nb = std::min<size_t>(admitted.size(), (size_t)srv->cfg.max_batch);
        Inflight f;
        f.stream = s;
        std::vector<BatchItem> items;
        items.reserve(nb);
        const double tl = now_s();
        for (size_t j = 0; j < nb; ++j) {
          Req& r = reqs[admitted.front()];
          admitted.pop_front();
          r.launch = tl;
          r.batch = batches;
          f.reqs.push_back((size_t)(&r - reqs.data()));
          items.push_back(BatchItem{srv->arena + r.offset, r.k, r.E});
        }
        brev_status ls;
        if (nb == 1)
          ls = launch_single(items[0].ptr, items[0].ptr, items[0].k, items[0].E,
                             srv->streams[s]);
        else
          ls = batched_launch_into(items.data(), (int)nb, srv->ws[s], srv->ws_bytes,
                                   srv->streams[s]);
        if (ls != BREV_OK) {
          result = ls;
          break;
        }
        e = get_event(&f.ev);
        if (e == cudaSuccess) e = cudaEventRecord(f.ev, srv->streams[s]);
        if (e != cudaSuccess) {
          result = cuda_error(e, "batch event");
          break;
        }
        busy[s] = true;
        inflight.push_back(std::move(f));
        ++batches;
        max_inflight = std::max(max_inflight, (int)inflight.size());
      }
    }
  }
  for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
  const double wall = now_s();
  cudaEventDestroy(ref);
  for (Inflight& f : inflight) srv->spare_events.push_back(f.ev);
  if (result != BREV_OK) return result;

  finish_stats(reqs, lat_us, queue_us, completed, bytes_moved, (uint64_t)batches,
               brev_launch_count() - launches0, pool.peak, max_inflight, wall, trace,
               trace_capacity, out);
  return BREV_OK;
}

}  // extern "C"
