"""Serving loop on the GPU: every request's result is the same served in the
mix (continuous batching, several streams, memory reused) as permuted alone,
and equals the CPU oracle."""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, assert_bytes_equal, device_array, host_array, to_bytes
from paper_1708_01873_gb300 import inputs
from paper_1708_01873_gb300.serve import GpuBackend, Server, poisson_requests

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_and_oracle(brev_lib, oracle_lib, cuda_device):
    pool = 64 << 20   # small pool: admission has to wait for memory
    backend = GpuBackend(pool, n_streams=3, fill_seed=None)
    results = {}

    def on_admit(r, be):
        # the client writes request r's input into its admitted buffer
        v = be.arena[r.offset:r.offset + r.nbytes]
        inputs.fill_torch(v, 70000 + r.rid, KIND[r.E])
        torch.cuda.current_stream().synchronize()

    def on_complete(r, be):
        results[r.rid] = be.arena[r.offset:r.offset + r.nbytes].cpu().numpy().copy()

    srv = Server(backend, pool, max_slots=24, max_batch=16, n_streams=3,
                 on_admit=on_admit, on_complete=on_complete)
    reqs = poisson_requests(21, 4000.0, 0.25, k_range=(4, 20), elem_sizes=(4, 8, 16))
    n = len(reqs)
    stats = srv.run(reqs)
    assert stats.completed == n and len(results) == n
    assert stats.batches < n            # requests really were batched
    assert stats.max_inflight_batches >= 1
    assert stats.peak_pool_bytes <= pool
    for r in reqs:
        src = torch.empty(r.nbytes, dtype=torch.uint8, device="cuda")
        inputs.fill_torch(src, 70000 + r.rid, KIND[r.E])
        alone = torch.empty_like(src)
        brev_lib.brev_permute_to(alone.view(DTYPE[r.E]), src.view(DTYPE[r.E]))
        assert_bytes_equal(results[r.rid], alone.cpu().numpy(), r.E,
                           f"request {r.rid} k={r.k} E={r.E}: mix vs alone")
        if r.k <= 14:
            h = inputs.array_np(70000 + r.rid, 1 << r.k, KIND[r.E])
            assert_bytes_equal(results[r.rid], oracle_lib.brev_oop(h, r.k, r.E), r.E,
                               f"request {r.rid}: vs oracle")
    lat = np.array(stats.latencies_us)
    assert (lat > 0).all()


def test_serving_workload_runs(brev_lib, cuda_device):
    from paper_1708_01873_gb300.serve import serve_poisson
    out = serve_poisson(seconds=0.5, rate=20000.0, pool_bytes=4 << 30)
    assert out["completed"] > 5000
    assert out["p99_us"] >= out["p50_us"] > 0
    assert out["gpu_launches"] >= out["batches"]


def test_native_server_results_equal_alone(brev_lib, oracle_lib, cuda_device):
    """The native loop serves a Poisson stream in the mix (continuous
    batching over 2 streams); with results held, every request's region of
    the arena must equal the single-array permutation of that region's
    initial bytes (and the oracle for the small ones).  Arrivals 10 us apart
    on average outpace a launch per request, so batches form (at a few
    thousand requests per second every request is served alone)."""
    arena = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    inputs.fill_torch(arena, 99, "u8", chunk=1 << 26)
    initial = arena.clone()
    torch.cuda.synchronize()
    stats, trace = brev_lib.brev_server_run_poisson(
        arena, seed=7, rate_per_s=100000.0, seconds=0.015, k_range=(4, 17),
        elem_sizes=(4, 8, 16), max_slots=32, max_batch=12, n_streams=2,
        hold_results=True, trace=True)
    torch.cuda.synchronize()
    assert stats["completed"] == stats["offered"] == len(trace) > 1000
    assert stats["batches"] < stats["completed"]   # requests were batched
    spans = sorted((r["offset"], r["offset"] + (r["elem_bytes"] << r["log2n"])) for r in trace)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))  # disjoint buffers
    for i, r in enumerate(trace):
        E, k, off = r["elem_bytes"], r["log2n"], r["offset"]
        nb = E << k
        src = initial[off:off + nb].view(DTYPE[E])
        alone = torch.empty_like(src)
        brev_lib.brev_permute_to(alone, src)
        got = arena[off:off + nb].cpu().numpy()
        assert_bytes_equal(got, alone.view(torch.uint8).cpu().numpy(), E,
                           f"request {i} k={k} E={E}: mix vs alone")
        if k <= 11:
            exp = oracle_lib.brev_oop(initial[off:off + nb].cpu().numpy(), k, E)
            assert_bytes_equal(got, exp, E, f"request {i}: vs oracle")
        # arrival and launch on the host clock, done on the device clock
        assert r["arrival_us"] <= r["launch_us"] <= r["done_us"] + 20.0


def test_native_server_production_mode(brev_lib, cuda_device):
    arena = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    stats, _ = brev_lib.brev_server_run_poisson(arena, seed=5, rate_per_s=20000.0, seconds=0.5)
    assert stats["completed"] == stats["offered"] > 8000
    assert 0 < stats["p50_us"] <= stats["p99_us"] <= stats["max_us"]
    assert stats["peak_pool_bytes"] <= arena.numel()
    with pytest.raises(brev_lib.BrevError):   # hold mode that cannot fit: refused, no hang
        brev_lib.brev_server_run_poisson(arena[: 64 << 20], seed=1, rate_per_s=20000.0,
                                         seconds=0.2, k_range=(20, 22), hold_results=True)


def _check_held_results(brev_lib, oracle_lib, arena, initial, trace, k_oracle=11):
    for i, r in enumerate(trace):
        E, k, off = r["elem_bytes"], r["log2n"], r["offset"]
        nb = E << k
        src = initial[off:off + nb].view(DTYPE[E])
        alone = torch.empty_like(src)
        brev_lib.brev_permute_to(alone, src)
        got = arena[off:off + nb].cpu().numpy()
        assert_bytes_equal(got, alone.view(torch.uint8).cpu().numpy(), E,
                           f"request {i} k={k} E={E}: mix vs alone")
        if k <= k_oracle:
            exp = oracle_lib.brev_oop(initial[off:off + nb].cpu().numpy(), k, E)
            assert_bytes_equal(got, exp, E, f"request {i}: vs oracle")
        assert r["arrival_us"] <= r["launch_us"] <= r["done_us"]


def test_resident_server_results_equal_alone(brev_lib, oracle_lib, cuda_device):
    """Resident mode: one kernel fed through host memory serves a Poisson
    stream (requests overlapping on the device); with results held, every
    request's region equals the single-array permutation of its initial
    bytes, and the oracle for the small ones."""
    t0 = brev_lib.brev_wait_timeouts()
    arena = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    inputs.fill_torch(arena, 98, "u8", chunk=1 << 26)
    initial = arena.clone()
    torch.cuda.synchronize()
    stats, trace = brev_lib.brev_server_run_poisson(
        arena, seed=9, rate_per_s=100000.0, seconds=0.015, k_range=(2, 17),
        elem_sizes=(4, 8, 16), max_slots=32, hold_results=True, trace=True, resident=True)
    torch.cuda.synchronize()
    assert stats["completed"] == stats["offered"] == len(trace) > 1000
    assert stats["launches"] == 1 and stats["max_inflight"] > 1   # overlapping requests
    spans = sorted((r["offset"], r["offset"] + (r["elem_bytes"] << r["log2n"])) for r in trace)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    _check_held_results(brev_lib, oracle_lib, arena, initial, trace)
    assert brev_lib.brev_wait_timeouts() == t0


def test_resident_server_backlog_results_equal_alone(brev_lib, cuda_device):
    """Resident mode above the device's bandwidth (about 8 TB/s offered in
    requests of 2 to 64 MiB): the backlog reaches 16 requests in flight, so
    requests are admitted with the large backlog tickets.  Every request's
    region equals the single-array permutation of its initial bytes
    (compared on the device)."""
    t0 = brev_lib.brev_wait_timeouts()
    arena = torch.empty(16 << 30, dtype=torch.uint8, device="cuda")
    inputs.fill_torch(arena, 97, "u8", chunk=1 << 28)
    initial = arena.clone()
    torch.cuda.synchronize()
    stats, trace = brev_lib.brev_server_run_poisson(
        arena, seed=13, rate_per_s=300000.0, seconds=0.0015, k_range=(19, 22),
        elem_sizes=(4, 8, 16), max_slots=64, hold_results=True, trace=True, resident=True)
    torch.cuda.synchronize()
    assert stats["completed"] == stats["offered"] == len(trace) > 250
    assert stats["max_inflight"] >= 16   # the backlog tickets were in use
    for i, r in enumerate(trace):
        E, k, off = r["elem_bytes"], r["log2n"], r["offset"]
        nb = E << k
        alone = torch.empty(nb, dtype=torch.uint8, device="cuda")
        brev_lib.brev_permute_to(alone.view(DTYPE[E]), initial[off:off + nb].view(DTYPE[E]))
        assert torch.equal(arena[off:off + nb], alone), f"request {i} k={k} E={E}"
    assert brev_lib.brev_wait_timeouts() == t0
    del arena, initial
    torch.cuda.empty_cache()


def test_resident_server_restarts_after_idle(brev_lib, oracle_lib, cuda_device):
    """Arrivals further apart than the idle limit: the host stops the kernel
    between them and launches it again; every result is still right."""
    t0 = brev_lib.brev_wait_timeouts()
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    inputs.fill_torch(arena, 97, "u8", chunk=1 << 26)
    initial = arena.clone()
    torch.cuda.synchronize()
    stats, trace = brev_lib.brev_server_run_poisson(
        arena, seed=3, rate_per_s=3.0, seconds=2.0, k_range=(8, 16), elem_sizes=(8, 16),
        max_slots=8, hold_results=True, trace=True, resident=True)
    torch.cuda.synchronize()
    assert stats["completed"] == stats["offered"] >= 2
    assert stats["launches"] >= 2   # stopped while idle and launched again
    _check_held_results(brev_lib, oracle_lib, arena, initial, trace)
    assert brev_lib.brev_wait_timeouts() == t0


def test_resident_server_production_rate(brev_lib, cuda_device):
    t0 = brev_lib.brev_wait_timeouts()
    arena = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    stats, _ = brev_lib.brev_server_run_poisson(arena, seed=5, rate_per_s=20000.0, seconds=0.5,
                                                resident=True)
    assert stats["completed"] == stats["offered"] > 8000
    assert 0 < stats["p50_us"] <= stats["p99_us"] <= stats["max_us"]
    assert stats["device_p50_us"] == stats["p50_us"]
    assert stats["launches"] == 1
    assert brev_lib.brev_wait_timeouts() == t0
    with pytest.raises(brev_lib.BrevError):   # held results that cannot fit: refused, no hang
        brev_lib.brev_server_run_poisson(arena[: 64 << 20], seed=1, rate_per_s=20000.0,
                                         seconds=0.2, k_range=(20, 22), hold_results=True,
                                         resident=True)
    x = torch.empty(1 << 20, dtype=torch.complex64, device="cuda")   # the device still works
    brev_lib.brev_permute(x, in_place=True)
    torch.cuda.synchronize()
    with pytest.raises(brev_lib.BrevError):   # more slots than the request ring
        brev_lib.brev_server_run_poisson(arena[: 64 << 20], seed=1, rate_per_s=1000.0,
                                         seconds=0.01, max_slots=5000, resident=True)
    with pytest.raises(brev_lib.BrevError):   # 1- and 2-byte elements: launches only
        brev_lib.brev_server_run_poisson(arena[: 64 << 20], seed=1, rate_per_s=1000.0,
                                         seconds=0.01, elem_sizes=(2, 4), resident=True)


def _arrivals(seed, rate, seconds):
    """The server's seeded arrival times (SplitMix64, exponential gaps), as
    brev_server_run_poisson draws them."""
    import math
    M = (1 << 64) - 1
    state = [seed & M]

    def sm64():
        state[0] = (state[0] + 0x9E3779B97F4A7C15) & M
        z = state[0]
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    t, out = 0.0, []
    while True:
        t += -math.log(((sm64() >> 11) + 1) * (1.0 / 9007199254740992.0)) / rate
        if t >= seconds:
            return out
        out.append(t)
        sm64()
        sm64()   # k and E draws


def test_resident_kernel_idle_limit_is_reported(brev_lib, oracle_lib, cuda_device):
    """Failure detection without a fault: with the host's idle stop disabled
    (20 s) and a 3 s gap between two requests, the kernel's own 2 s idle
    limit ends it; the next request finds no kernel, the run returns
    BREV_ERR_CUDA, the wait timeout is counted, and the device keeps
    working."""
    seed = next(s for s in range(200)
                if len(a := _arrivals(s, 0.5, 6.0)) >= 2 and a[0] < 1.5 and a[1] - a[0] > 3.0)
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    before = brev_lib.brev_wait_timeouts()
    with pytest.raises(brev_lib.BrevError) as err:
        brev_lib.brev_server_run_poisson(arena, seed=seed, rate_per_s=0.5, seconds=6.0,
                                         k_range=(10, 12), elem_sizes=(8,), resident=True,
                                         idle_stop_ms=20000)
    assert err.value.status == 5   # BREV_ERR_CUDA
    assert brev_lib.brev_wait_timeouts() > before
    x = device_array(77, 14, 16)
    y = torch.empty_like(x)
    brev_lib.brev_permute_to(y, x)
    assert_bytes_equal(to_bytes(y), oracle_lib.brev_oop(host_array(77, 14, 16), 14, 16), 16,
                       "after the timeout")
