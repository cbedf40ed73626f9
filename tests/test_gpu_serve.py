"""Serving loop on the GPU: every request's result is the same served in the
mix (continuous batching, several streams, memory reused) as permuted alone,
and equals the CPU oracle."""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, assert_bytes_equal
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
