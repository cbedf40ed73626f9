"""Serving loop host logic on the CPU: pool accounting, admission by free
HBM and slots, FIFO order, batching limits, stream limits, cancellation.
A fake backend stands in for the GPU (completion after a few polls)."""
import random

import numpy as np
import pytest

from paper_1708_01873_gb300.serve import PoolAllocator, Request, Server, poisson_requests


def test_pool_alloc_free_coalesce():
    p = PoolAllocator(4096, align=256)
    a = p.alloc(100)
    b = p.alloc(256)
    c = p.alloc(1000)
    assert (a, b, c) == (0, 256, 512)
    assert p.used_bytes == 256 + 256 + 1024
    assert p.alloc(4096) is None
    p.free(b)
    assert p.alloc(200) == 256          # first fit reuses the hole
    p.free(a)
    p.free(256)
    p.free(c)
    assert p.used_bytes == 0 and p.largest_free() == 4096  # fully coalesced
    assert p.alloc(4096) == 0


def test_pool_random_against_model():
    rng = random.Random(1)
    cap = 1 << 20
    p = PoolAllocator(cap, align=64)
    live = {}
    for _ in range(5000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            p.free(off)
            del live[off]
        else:
            n = rng.randrange(1, 40000)
            off = p.alloc(n)
            if off is None:
                # refused only if no free block can hold it
                assert p.largest_free() < (n + 63) // 64 * 64
                continue
            assert off % 64 == 0 and off + n <= cap
            for o, m in live.items():   # no overlap with live blocks
                assert off + n <= o or o + m <= off
            live[off] = n
        assert p.used_bytes == sum((m + 63) // 64 * 64 for m in live.values())


class FakeBackend:
    """Completes each batch after `latency` polls; records launches."""

    def __init__(self, latency=3):
        self.latency = latency
        self.launched = []
        self.t = 0.0

    def start(self, t0):
        pass

    def launch(self, reqs, s):
        h = {"left": self.latency, "reqs": list(reqs), "stream": s}
        self.launched.append(h)
        return h

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def completion_time(self, h):
        return self.t

    def release(self, h):
        pass

    def sync(self):
        pass


def make_server(pool=1 << 20, slots=8, batch=4, streams=2, latency=3):
    be = FakeBackend(latency)
    clock = {"t": 0.0}

    def tick():
        clock["t"] += 1e-6
        be.t = clock["t"]
        return clock["t"]

    srv = Server(be, pool, max_slots=slots, max_batch=batch, n_streams=streams, clock=tick)
    return srv, be


def test_admission_respects_memory_and_slots_and_fifo():
    srv, be = make_server(pool=64 << 10, slots=3, batch=8, streams=2, latency=4)
    reqs = [Request(i, k, 4, 0.0) for i, k in enumerate([12, 13, 12, 10, 13, 11, 12, 10])]
    for r in reqs:
        srv.submit(r)
    order = []
    for _ in range(500):
        srv.step()
        assert srv.pool.used_bytes <= srv.pool.capacity
        assert srv.slots_used <= 3
        assert len(srv.inflight) <= 2
        for r in reqs:
            if r.state in ("admitted", "running", "done") and r.rid not in order:
                order.append(r.rid)
        if srv.idle():
            break
    assert srv.idle()
    assert order == sorted(order)                      # admitted in arrival order
    assert all(r.state == "done" for r in reqs)
    assert srv.stats.completed == len(reqs)
    for h in be.launched:
        assert len(h["reqs"]) <= 8


def test_head_of_line_waits_for_memory():
    # a big request at the head blocks smaller ones behind it (no starvation)
    srv, be = make_server(pool=1 << 16, slots=8, batch=8, streams=1, latency=2)
    small = Request(0, 13, 4, 0.0)    # 32 KiB
    big = Request(1, 14, 4, 0.0)      # 64 KiB: needs the whole pool
    tail = Request(2, 10, 4, 0.0)
    for r in (small, big, tail):
        srv.submit(r)
    srv.step()
    assert small.state == "running" and big.state == "queued" and tail.state == "queued"
    while big.state == "queued":
        srv.step()
    assert small.state == "done"
    assert tail.state in ("queued", "admitted")
    while not srv.idle():
        srv.step()
    assert tail.t_launch >= big.t_launch


def test_batch_and_stream_limits():
    srv, be = make_server(pool=1 << 24, slots=100, batch=5, streams=3, latency=6)
    for i in range(40):
        srv.submit(Request(i, 10, 8, 0.0))
    peak = 0
    while not srv.idle():
        srv.step()
        peak = max(peak, len(srv.inflight))
        assert len({s for _, s, _ in srv.inflight}) == len(srv.inflight)  # one batch per stream
    assert peak == 3
    assert max(len(h["reqs"]) for h in be.launched) == 5
    assert srv.stats.completed == 40


def test_cancellation():
    srv, be = make_server(pool=1 << 14, slots=2, batch=1, streams=1, latency=5)
    reqs = [Request(i, 11, 4, 0.0) for i in range(5)]   # 8 KiB each, 2 fit
    for r in reqs:
        srv.submit(r)
    srv.step()   # r0 launched, r1 admitted (slot 2)
    assert reqs[0].state == "running" and reqs[1].state == "admitted"
    assert not srv.cancel(0)              # running: cannot cancel
    assert srv.cancel(1)                  # admitted: memory and slot returned
    assert srv.cancel(4)                  # queued
    assert srv.pool.used_bytes == 8 << 10 and srv.slots_used == 1
    while not srv.idle():
        srv.step()
    assert [r.state for r in reqs] == ["done", "cancelled", "done", "done", "cancelled"]
    assert srv.stats.cancelled == 2 and srv.stats.completed == 3


def test_poisson_generator():
    reqs = poisson_requests(5, 20000.0, 1.0)
    assert 19000 < len(reqs) < 21000
    gaps = np.diff([r.arrival for r in reqs])
    assert abs(gaps.mean() - 50e-6) < 3e-6
    ks = np.array([r.k for r in reqs])
    assert ks.min() == 10 and ks.max() == 24
    assert set(r.E for r in reqs) == {4, 8, 16}
    # seeded
    assert [r.k for r in poisson_requests(5, 20000.0, 0.01)] == \
        [r.k for r in reqs[: len(poisson_requests(5, 20000.0, 0.01))]]


def test_request_larger_than_pool_rejected():
    srv, _ = make_server(pool=1 << 12)
    with pytest.raises(ValueError):
        srv.submit(Request(0, 12, 4, 0.0))
