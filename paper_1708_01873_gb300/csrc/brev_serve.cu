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
// Latency = device completion time - arrival time.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "brev_internal.h"

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
  int batch = -1;
  bool admitted = false;
};

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
  std::vector<cudaEvent_t> spare_events;
  int device = 0;
};

using namespace brev;

extern "C" {

brev_status brev_server_create(const brev_server_config* cfg, void* arena, uint64_t arena_bytes,
                               brev_server** out) {
  if (!out) return set_error(BREV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->max_slots < 1 || cfg->max_batch < 1 || cfg->n_streams < 1 ||
      cfg->n_streams > 64)
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
  for (cudaEvent_t e : srv->spare_events) cudaEventDestroy(e);
  delete srv;
}

brev_status brev_server_run_poisson(brev_server* srv, uint64_t seed, double rate_per_s,
                                    double seconds, int k_min, int k_max,
                                    const int* elem_bytes, int n_elem_bytes, int hold_results,
                                    brev_server_request* trace, uint64_t trace_capacity,
                                    brev_server_stats* out) {
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
      for (size_t ri : inflight[i].reqs) {
        Req& r = reqs[ri];
        r.done = done;
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
          ls = batched_launch(items.data(), (int)nb, srv->streams[s]);
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

  out->completed = completed;
  out->batches = (uint64_t)batches;
  out->launches = brev_launch_count() - launches0;
  out->p50_us = percentile(lat_us, 50);
  out->p99_us = percentile(lat_us, 99);
  out->max_us = lat_us.empty() ? 0 : *std::max_element(lat_us.begin(), lat_us.end());
  double sum = 0;
  for (double v : lat_us) sum += v;
  out->mean_us = lat_us.empty() ? 0 : sum / (double)lat_us.size();
  out->queue_p99_us = percentile(queue_us, 99);
  out->wall_s = wall;
  out->req_per_s = (double)completed / wall;
  out->gbs = (double)bytes_moved / wall / 1e9;
  out->peak_pool_bytes = pool.peak;
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
    }
  }
  return BREV_OK;
}

}  // extern "C"
