"""Continuous-batching serving loop for bit-reversed permutations.

Requests (an array of 2^k elements of E bytes each) arrive over time.  The
server

  * admits a waiting request when a slot is free and the HBM pool can hold
    its buffer (admission by free HBM: the pool's own accounting, not
    cudaMemGetInfo, which is far too slow per request);
  * hands the admitted request's buffer to the client (``on_admit``), which
    writes the input there -- on the device, no PCIe in the loop;
  * every loop iteration gathers all admitted, not yet launched requests into
    ONE in-place batched launch (brev_permute_batched_mixed) on the next of S
    streams, so requests that arrive while others run are admitted and
    launched as slots and memory free up, and their work overlaps on the
    device;
  * detects completion with a CUDA event per batch, stamps each request's
    completion on the device clock, releases its memory and slot, and hands
    the result to ``on_complete`` before the buffer is reused.

Latency = device completion time - arrival time.  The GPU side is behind a
small backend interface so the admission / slot / ordering logic runs
against a fake backend on the CPU in tests.
"""
from __future__ import annotations

import bisect
import heapq
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


# ----------------------------------------------------------------- pool --
class PoolAllocator:
    """First-fit allocator over one preallocated arena of ``capacity`` bytes,
    ``align``-byte aligned blocks, free neighbours coalesced."""

    def __init__(self, capacity: int, align: int = 256):
        self.capacity = int(capacity)
        self.align = int(align)
        self._free_off = [0]            # sorted offsets of free blocks
        self._free_len = {0: self.capacity}
        self._used = {}                  # offset -> length
        self.used_bytes = 0
        self.peak_bytes = 0

    def _round(self, n: int) -> int:
        return (int(n) + self.align - 1) // self.align * self.align

    def alloc(self, nbytes: int) -> Optional[int]:
        need = self._round(max(1, nbytes))
        for i, off in enumerate(self._free_off):
            ln = self._free_len[off]
            if ln >= need:
                del self._free_len[off]
                self._free_off.pop(i)
                if ln > need:
                    rest = off + need
                    self._free_len[rest] = ln - need
                    bisect.insort(self._free_off, rest)
                self._used[off] = need
                self.used_bytes += need
                self.peak_bytes = max(self.peak_bytes, self.used_bytes)
                return off
        return None

    def free(self, off: int) -> None:
        ln = self._used.pop(off)
        self.used_bytes -= ln
        i = bisect.bisect_left(self._free_off, off)
        # merge with the following block
        if i < len(self._free_off) and off + ln == self._free_off[i]:
            nxt = self._free_off.pop(i)
            ln += self._free_len.pop(nxt)
        # merge with the preceding block
        if i > 0:
            prv = self._free_off[i - 1]
            if prv + self._free_len[prv] == off:
                self._free_len[prv] += ln
                return
        self._free_off.insert(i, off)
        self._free_len[off] = ln

    @property
    def free_bytes(self) -> int:
        return self.capacity - self.used_bytes

    def largest_free(self) -> int:
        return max(self._free_len.values(), default=0)


# -------------------------------------------------------------- requests --
@dataclass
class Request:
    rid: int
    k: int
    E: int
    arrival: float                  # seconds, server clock
    state: str = "new"              # queued admitted running done cancelled
    offset: int = -1
    t_admit: float = 0.0
    t_launch: float = 0.0
    t_done: float = 0.0             # device completion, server clock
    batch: int = -1

    @property
    def nbytes(self) -> int:
        return self.E << self.k


@dataclass
class Stats:
    completed: int = 0
    cancelled: int = 0
    batches: int = 0
    launched_requests: int = 0
    bytes_moved: int = 0            # 2 n E summed over completed requests
    latencies_us: list = field(default_factory=list)
    queue_us: list = field(default_factory=list)
    peak_pool_bytes: int = 0
    max_inflight_batches: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        lat = np.array(self.latencies_us) if self.latencies_us else np.zeros(1)
        q = np.array(self.queue_us) if self.queue_us else np.zeros(1)
        return {
            "completed": self.completed, "cancelled": self.cancelled,
            "batches": self.batches,
            "mean_batch": round(self.launched_requests / max(1, self.batches), 2),
            "p50_us": round(float(np.percentile(lat, 50)), 1),
            "p99_us": round(float(np.percentile(lat, 99)), 1),
            "max_us": round(float(lat.max()), 1),
            "queue_p99_us": round(float(np.percentile(q, 99)), 1),
            "req_per_s": round(self.completed / max(self.wall_s, 1e-9), 1),
            "gbs": round(self.bytes_moved / max(self.wall_s, 1e-9) / 1e9, 1),
            "peak_pool_bytes": self.peak_pool_bytes,
            "max_inflight_batches": self.max_inflight_batches,
            "wall_s": round(self.wall_s, 3),
        }


# ---------------------------------------------------------------- server --
class Server:
    """Continuous batching over ``backend`` (see GpuBackend for the
    interface).  Single host thread; call ``step()`` in a loop or ``run()``."""

    def __init__(self, backend, pool_bytes: int, max_slots: int = 64,
                 max_batch: int = 256, n_streams: int = 4,
                 on_admit: Optional[Callable] = None,
                 on_complete: Optional[Callable] = None,
                 clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.pool = PoolAllocator(pool_bytes)
        self.max_slots = max_slots
        self.max_batch = max_batch
        self.n_streams = n_streams
        self.on_admit = on_admit
        self.on_complete = on_complete
        self.clock = clock
        self.waiting: list[Request] = []     # FIFO of queued requests
        self.admitted: list[Request] = []    # admitted, not launched
        self.inflight = []                    # (handle, stream, [requests])
        self.busy_streams: set[int] = set()
        self.next_stream = 0
        self.slots_used = 0
        self.stats = Stats()
        self._by_id = {}

    # -- client side --
    def submit(self, req: Request) -> None:
        if req.nbytes > self.pool.capacity:
            raise ValueError(f"request {req.rid} ({req.nbytes} B) exceeds the pool")
        req.state = "queued"
        self.waiting.append(req)
        self._by_id[req.rid] = req

    def cancel(self, rid: int) -> bool:
        """Cancel a request that has not been launched; returns whether it
        was cancelled (launched requests run to completion)."""
        r = self._by_id.get(rid)
        if r is None or r.state not in ("queued", "admitted"):
            return False
        if r.state == "queued":
            self.waiting.remove(r)
        else:
            self.admitted.remove(r)
            self.pool.free(r.offset)
            self.slots_used -= 1
        r.state = "cancelled"
        self.stats.cancelled += 1
        return True

    # -- loop --
    def _poll(self) -> None:
        keep = []
        for handle, s, reqs in self.inflight:
            if self.backend.done(handle):
                t = self.backend.completion_time(handle)
                for r in reqs:
                    r.t_done = t
                    r.state = "done"
                    if self.on_complete:
                        self.on_complete(r, self.backend)
                    self.pool.free(r.offset)
                    self.slots_used -= 1
                    self.stats.completed += 1
                    self.stats.bytes_moved += 2 * r.nbytes
                    self.stats.latencies_us.append((t - r.arrival) * 1e6)
                    self.stats.queue_us.append((r.t_launch - r.arrival) * 1e6)
                self.busy_streams.discard(s)
                self.backend.release(handle)
            else:
                keep.append((handle, s, reqs))
        self.inflight = keep

    def _admit(self, now: float) -> None:
        # FIFO admission: the head waits for memory rather than being
        # overtaken, so large requests cannot starve
        while self.waiting and self.slots_used < self.max_slots:
            r = self.waiting[0]
            off = self.pool.alloc(r.nbytes)
            if off is None:
                break
            self.waiting.pop(0)
            r.offset = off
            r.state = "admitted"
            r.t_admit = now
            self.slots_used += 1
            if self.on_admit:
                self.on_admit(r, self.backend)
            self.admitted.append(r)
        self.stats.peak_pool_bytes = max(self.stats.peak_pool_bytes, self.pool.used_bytes)

    def _launch(self, now: float) -> None:
        if not self.admitted:
            return
        free = [s for s in range(self.n_streams) if s not in self.busy_streams]
        if not free:
            return
        # round robin over idle streams
        s = min(free, key=lambda x: (x - self.next_stream) % self.n_streams)
        self.next_stream = (s + 1) % self.n_streams
        batch, self.admitted = self.admitted[:self.max_batch], self.admitted[self.max_batch:]
        for r in batch:
            r.state = "running"
            r.t_launch = now
            r.batch = self.stats.batches
        handle = self.backend.launch(batch, s)
        self.inflight.append((handle, s, batch))
        self.busy_streams.add(s)
        self.stats.batches += 1
        self.stats.launched_requests += len(batch)
        self.stats.max_inflight_batches = max(self.stats.max_inflight_batches,
                                              len(self.inflight))

    def step(self) -> None:
        now = self.clock()
        self._poll()
        self._admit(now)
        self._launch(now)

    def idle(self) -> bool:
        return not (self.waiting or self.admitted or self.inflight)

    def run(self, arrivals: list[Request], until_drained: bool = True) -> Stats:
        """Replay ``arrivals`` (sorted by .arrival, seconds from start) in
        real time, then drain."""
        t0 = self.clock()
        self.backend.start(t0)
        i = 0
        n = len(arrivals)
        while i < n or (until_drained and not self.idle()):
            now = self.clock() - t0
            while i < n and arrivals[i].arrival <= now:
                r = arrivals[i]
                r.arrival += t0
                self.submit(r)
                i += 1
            self.step()
        self.backend.sync()
        self.stats.wall_s = self.clock() - t0
        return self.stats


def poisson_requests(seed: int, rate_per_s: float, duration_s: float,
                     k_range=(10, 24), elem_sizes=(4, 8, 16)) -> list[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate), k uniform in
    k_range (inclusive), E uniform over elem_sizes."""
    rng = np.random.default_rng(seed)
    t, out, rid = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        E = int(rng.choice(elem_sizes))
        out.append(Request(rid, k, E, t))
        rid += 1
    return out


# ----------------------------------------------------------- GPU backend --
class GpuBackend:
    """Device side of the server: one HBM arena (the pool's memory), S CUDA
    streams, one batched library launch per server launch, and a CUDA event
    per batch for completion.  Completion times are read on the device
    clock (elapsed time from a reference event) and mapped to the server
    clock."""

    DTYPES = None

    def __init__(self, pool_bytes: int, n_streams: int = 4, device: int = 0,
                 fill_seed: Optional[int] = 1):
        import torch
        from . import brev
        self.torch = torch
        self.brev = brev
        self.L = brev.lib()
        self.device = torch.device("cuda", device)
        self.arena = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        if fill_seed is not None:
            from . import inputs
            inputs.fill_torch(self.arena, fill_seed, "u8", chunk=1 << 28)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self._events = []
        self.ref = None
        self.t_ref = 0.0
        self.launches = 0

    def view(self, req: Request):
        import torch
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.float32, 8: torch.complex64,
              16: torch.complex128}[req.E]
        return self.arena[req.offset:req.offset + req.nbytes].view(dt)

    def start(self, t0: float) -> None:
        torch = self.torch
        torch.cuda.synchronize(self.device)
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref.record(self.streams[0])
        self.ref.synchronize()
        self.t_ref = time.perf_counter()

    def launch(self, reqs: list, s: int):
        import ctypes
        n = len(reqs)
        base = self.arena.data_ptr()
        st = self.streams[s]
        if n == 1:
            # a batch of one: the single-array launch (no batch workspace)
            r = reqs[0]
            p = base + r.offset
            rc = self.L.brev_permute_to(p, p, r.k, r.E, st.cuda_stream)
        else:
            ptrs = (ctypes.c_void_p * n)(*[base + r.offset for r in reqs])
            ks = (ctypes.c_int * n)(*[r.k for r in reqs])
            es = (ctypes.c_int * n)(*[r.E for r in reqs])
            rc = self.L.brev_permute_batched_mixed(ptrs, ks, es, n, st.cuda_stream)
        if rc != 0:
            raise RuntimeError(self.brev.brev_last_error())
        ev = self._events.pop() if self._events else self.torch.cuda.Event(enable_timing=True)
        ev.record(st)
        self.launches += 1
        return ev

    def done(self, handle) -> bool:
        return handle.query()

    def completion_time(self, handle) -> float:
        # completion as the serving thread sees it (the clock its arrivals
        # use), as the native loop reports; the device-clock time of the
        # event would be read against a reference event that completed a
        # few microseconds before t_ref, and so run late by that gap
        return time.perf_counter()

    def release(self, handle) -> None:
        self._events.append(handle)

    def sync(self) -> None:
        self.torch.cuda.synchronize(self.device)


def serve_poisson(seconds: float = 10.0, rate: float = 20000.0, seed: int = 5,
                  pool_bytes: int = 16 << 30, max_slots: int = 256, max_batch: int = 256,
                  n_streams: int = 4, k_range=(10, 24), elem_sizes=(4, 8, 16),
                  device: int = 0) -> dict:
    """The serving workload: Poisson arrivals at ``rate`` req/s for
    ``seconds``, k uniform in k_range, E uniform over elem_sizes."""
    backend = GpuBackend(pool_bytes, n_streams, device)
    srv = Server(backend, pool_bytes, max_slots=max_slots, max_batch=max_batch,
                 n_streams=n_streams)
    # warm-up: one short burst compiles nothing but settles the pools
    warm = poisson_requests(seed + 1000, rate, 0.05, k_range, elem_sizes)
    Server(backend, pool_bytes, max_slots, max_batch, n_streams).run(warm)
    arrivals = poisson_requests(seed, rate, seconds, k_range, elem_sizes)
    c0 = backend.L.brev_launch_count()
    stats = srv.run(arrivals)
    out = stats.summary()
    out.update({"offered_req_per_s": rate, "seconds": seconds, "streams": n_streams,
                "max_slots": max_slots, "pool_bytes": pool_bytes,
                "offered_gbs": round(sum(2 * r.nbytes for r in arrivals) / seconds / 1e9, 1),
                "gpu_launches": int(backend.L.brev_launch_count() - c0)})
    return out
