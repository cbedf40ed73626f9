"""Multi-rank host logic on the CPU (gloo, world sizes 2 and 4).

The sweep runs as replicas (each rank permutes its own arrays, no data-path
collective; the timing is reduced with a max over ranks and the bytes
summed).  A batch shards by array (brev_shard_batch).  One array spread over
G ranks takes one all-to-all between two local passes (brev_dist_*).  These
tests run the reduction, the barrier, the reference arm's launch under
torchrun, the batch sharding and the distributed single-array steps, with
gloo on 127.0.0.1 and the local passes on the CPU."""
import ctypes
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        m = bench.max_over_ranks(local_ms, world)
        dist.barrier()
        v = bench.whole_job_gbs(1e9, world, m * 1e-3)
        # replicas: each rank's batch is its own; nothing is exchanged
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, m, v in res:
        assert m == 15.0                                  # slowest rank
        assert abs(v - 2 * 1e9 / 15e-3 / 1e9) < 1e-9      # both ranks' bytes / max time


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_gbs(2e9, 1, 1.0) == 2.0


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1",
           "--ref-seconds", "3"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the same config object as the GPU arm's line (its sample is in cpu_baseline)
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.sweep_config(28, "u32,f32,c64,c128", 2, None)
    assert "bounded sample" in d["cpu_baseline"]["sample"]


def test_sweep_config_counts():
    """The sweep's reported size against a closed form: every k = 10..28 of
    4 + 4 + 8 + 16 bytes per element, read and written, out of place and in
    place -- 2 * 2 * (2^29 - 2^10) * 32 bytes in 152 points."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.sweep_config(28, "u32,f32,c64,c128", 1, 129)
    assert c["points_per_step"] == 152
    assert c["bytes_per_step"] == 2 * 2 * ((1 << 29) - (1 << 10)) * 32 == 68719345664
    assert "64 GiB moved per step" in c["l2"] and "L2 = 129 MiB" in c["l2"]
    assert c["parallelism"] == "1 GPU"
    small = bench.sweep_config(14, "c128", 4, 129)
    assert small["points_per_step"] == 2 * 5
    assert small["bytes_per_step"] == 2 * 2 * ((1 << 15) - (1 << 10)) * 16
    assert "can stay in L2" in small["l2"] and small["parallelism"] == "replicas x4"


# ------------------------------------------------------------------------
# One array over G ranks (brev_dist_*): the exchange plan and the three
# steps, with the local passes restated on the CPU and the exchange run as a
# gloo all-to-all between real processes.

def _finish_cpu(block, recv, k, g, E):
    """Step 3 restated: block[r 2^g + rev_g(p)] = recv[p R + r]."""
    import numpy as np
    G, R = 1 << g, 1 << (k - 2 * g)
    rv = recv.view(torch.uint8).numpy().reshape(G, R, E)
    out = block.view(torch.uint8).numpy().reshape(R, G, E)
    for p in range(G):
        out[:, int(format(p, f"0{g}b")[::-1], 2) if g else 0, :] = rv[p]


def _dist_worker(rank, world, port, k, E, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_1708_01873_gb300 import brev, inputs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        g = world.bit_length() - 1
        n_loc = 1 << (k - g)
        full = inputs.array_np(77, 1 << k, {4: "f32", 8: "c64", 16: "c128", 1: "u8"}[E])
        block = torch.from_numpy(full.reshape(-1, E)[rank * n_loc:(rank + 1) * n_loc]
                                 .reshape(-1).copy())
        recv = torch.zeros_like(block)

        def pack(b):
            a = b.numpy()
            oracle.brev_inplace(a, k - g, E)

        def exchange(r, s, seg):
            assert seg == 1 << (k - 2 * g)
            dist.all_to_all_single(r, s)

        brev.dist_steps(block, recv, k, g, rank, pack, exchange,
                        lambda b, r: _finish_cpu(b, r, k, g, E))
        exp = oracle.brev_oop(full, k, E).reshape(-1, E)[rank * n_loc:(rank + 1) * n_loc]
        q.put((rank, bool(np.array_equal(block.numpy().reshape(-1, E), exp))))
    finally:
        dist.destroy_process_group()


def _spawn(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=target, args=(r, world, port, *args, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return sorted(q.get(timeout=30) for _ in range(world))


@pytest.mark.parametrize("world,k,E", [(2, 12, 16), (4, 13, 8), (4, 8, 4), (2, 2, 1)])
def test_distributed_single_array_over_gloo_ranks(world, k, E):
    """Every rank's block equals its part of the oracle's permutation of the
    whole array, after pack -> all-to-all -> finish across real processes."""
    res = _spawn(_dist_worker, world, k, E)
    assert [ok for _, ok in res] == [True] * world


def test_distributed_plan_and_index_identity():
    """The plan's equal segments, and the index map behind the three steps
    (concatenation identity: element (p, m, l) lands on rank rev(l) at
    offset rev(m) 2^g + rev(p)) checked element by element."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1708_01873_gb300 import brev
    oracle.build()
    for k, g in ((6, 3), (9, 2), (4, 1), (2, 1), (10, 0)):
        G = 1 << g
        for rank in range(G):
            so, ro, seg = brev.brev_dist_plan(k, g, 16, rank)
            assert seg == 1 << (k - 2 * g) and so == ro == [q * seg for q in range(G)]
        for i in range(1 << k):
            p, j = i >> (k - g), i & ((1 << (k - g)) - 1)
            l, m = j & (G - 1), j >> g
            q_, off = oracle.rev_bits(l, g), (oracle.rev_bits(m, k - 2 * g) << g) | oracle.rev_bits(p, g)
            assert (q_ << (k - g)) | off == oracle.rev_bits(i, k)
    L = brev.lib()
    so, ro, seg = (ctypes.c_uint64 * 4)(), (ctypes.c_uint64 * 4)(), ctypes.c_uint64()
    assert L.brev_dist_plan(3, 2, 16, 0, so, ro, ctypes.byref(seg)) == 1  # 2g > k
    assert L.brev_dist_plan(8, 2, 16, 4, so, ro, ctypes.byref(seg)) == 1  # rank out of range


def _shard_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_1708_01873_gb300 import brev, inputs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        rng = np.random.default_rng(4)
        ks = [int(x) for x in rng.integers(2, 13, size=300)]
        es = [int(x) for x in rng.choice([8, 16], size=300)]
        owner = brev.brev_shard_batch(ks, es, world)
        mine = {}
        for i, (k, E) in enumerate(zip(ks, es)):
            if owner[i] == rank:
                x = inputs.array_np(40000 + i, 1 << k, "c64" if E == 8 else "c128")
                oracle.brev_inplace(x, k, E)  # stands in for this rank's batched launch
                mine[i] = x.tobytes()
        got = [None] * world
        dist.all_gather_object(got, mine)
        union = {}
        for part in got:
            for i, v in part.items():
                assert i not in union  # every array on exactly one rank
                union[i] = v
        ok = sorted(union) == list(range(len(ks)))
        for i, (k, E) in enumerate(zip(ks, es)):
            x = inputs.array_np(40000 + i, 1 << k, "c64" if E == 8 else "c128")
            ok = ok and union[i] == oracle.brev_oop(x, k, E).tobytes()
        q.put((rank, ok, owner))
    finally:
        dist.destroy_process_group()


def test_batch_sharded_by_array_over_gloo_ranks():
    """A batch split by array: every array is permuted on exactly one rank,
    all ranks agree on the owners, and the union equals the oracle."""
    res = _spawn(_shard_worker, 2)
    assert all(ok for _, ok, _ in res)
    assert res[0][2] == res[1][2]


def test_shard_batch_balance():
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1708_01873_gb300 import brev
    rng = np.random.default_rng(9)
    for world in (1, 2, 3, 8):
        ks = [int(x) for x in rng.integers(8, 21, size=4096)]
        es = [int(x) for x in rng.choice([8, 16], size=4096)]
        own = brev.brev_shard_batch(ks, es, world)
        assert sorted(set(own)) == list(range(world))
        load = [0] * world
        for k, E, o in zip(ks, es, own):
            load[o] += E << k
        biggest = max(E << k for k, E in zip(ks, es))
        assert max(load) - min(load) <= biggest  # within one array of each other


def test_latency_by_size_classes():
    """The bench's per-size-class latency summary on a synthetic trace: the
    slowest 1 % all in the large class, classes counted and split right,
    requests never seen by the serving thread left out."""
    sys.path.insert(0, ROOT)
    import bench
    trace = []
    for i in range(1000):
        k = 10 + (i % 15)                      # k 10..24
        lat = 100.0 if k >= 23 and i % 7 == 0 else 10.0
        trace.append({"log2n": k, "arrival_us": float(i), "seen_us": float(i) + lat})
    trace.append({"log2n": 12, "arrival_us": 5.0, "seen_us": 0.0})  # never seen
    out = bench.latency_by_size(trace)
    assert sum(v["count"] for v in out.values()) == 1000
    assert out["k23-24"]["share_of_slowest_1pct"] == 1.0
    assert out["k10-16"]["p50_us"] == 10.0 and out["k23-24"]["p99_us"] == 100.0
    assert bench.latency_by_size([]) is None
