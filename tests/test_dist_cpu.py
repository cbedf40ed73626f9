"""Multi-rank host logic on the CPU (gloo, world size 2).

The GPU path runs as replicas: each rank permutes its own arrays with no
data-path collective; only the timing is reduced (max over ranks) and the
bytes summed.  These tests run that reduction, the barrier, and the
reference arm's launch under torchrun, with gloo on 127.0.0.1."""
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
