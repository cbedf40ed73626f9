"""Batched persistent launch and captured plans vs the CPU oracle."""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, assert_bytes_equal, device_array, host_array, to_bytes
from paper_1708_01873_gb300 import inputs

pytestmark = pytest.mark.gpu


def _make_batch(rng, count, ks, Es, seed0):
    arrays, hosts = [], []
    for i in range(count):
        k = int(rng.choice(ks))
        E = int(rng.choice(Es))
        arrays.append(device_array(seed0 + i, k, E))
        hosts.append((k, E, host_array(seed0 + i, k, E)))
    return arrays, hosts


def _expect(oracle_lib, hosts):
    return [oracle_lib.brev_oop(h, k, E) for k, E, h in hosts]


def test_batched_mixed_vs_oracle(brev_lib, oracle_lib, cuda_device):
    rng = np.random.default_rng(11)
    arrays, hosts = _make_batch(rng, 300, list(range(0, 19)), [4, 8, 16], 100)
    t0 = brev_lib.brev_wait_timeouts()
    c0 = brev_lib.brev_launch_count()
    brev_lib.brev_permute_batched(arrays)
    torch.cuda.synchronize()
    assert brev_lib.brev_launch_count() - c0 == 1  # one persistent launch
    for a, e, (k, E, _) in zip(arrays, _expect(oracle_lib, hosts), hosts):
        assert_bytes_equal(to_bytes(a), e, E, f"batched k={k} E={E}")
    assert brev_lib.brev_wait_timeouts() == t0  # no CTA gave up on its copies


def test_batched_single_elem_size_api(brev_lib, oracle_lib, cuda_device):
    rng = np.random.default_rng(12)
    arrays, hosts = _make_batch(rng, 64, list(range(6, 17)), [16], 700)
    L = brev_lib.lib()
    import ctypes
    ptrs = (ctypes.c_void_p * len(arrays))(*[a.data_ptr() for a in arrays])
    ks = (ctypes.c_int * len(arrays))(*[k for k, _, _ in hosts])
    rc = L.brev_permute_batched(ptrs, ks, len(arrays), 16,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 0, brev_lib.brev_last_error()
    torch.cuda.synchronize()
    for a, e, (k, E, _) in zip(arrays, _expect(oracle_lib, hosts), hosts):
        assert_bytes_equal(to_bytes(a), e, E, f"batched k={k}")


def test_batched_fallback_arrays(brev_lib, oracle_lib, cuda_device):
    """1- and 2-byte elements and arrays not 16-byte aligned are permuted by
    single-array launches inside the same call."""
    rng = np.random.default_rng(13)
    arrays, hosts = _make_batch(rng, 40, list(range(0, 16)), [1, 2, 4, 8, 16], 900)
    # unaligned views
    for i, (k, E) in enumerate(((12, 8), (15, 4), (9, 8))):
        n = 1 << k
        big = device_array(1200 + i, k, E, extra_elems=1)
        v = big[1:1 + n]
        arrays.append(v)
        hosts.append((k, E, to_bytes(v)))
    brev_lib.brev_permute_batched(arrays)
    torch.cuda.synchronize()
    for a, e, (k, E, _) in zip(arrays, _expect(oracle_lib, hosts), hosts):
        assert_bytes_equal(to_bytes(a), e, E, f"fallback k={k} E={E}")


def test_batched_edge_cases(brev_lib, cuda_device):
    brev_lib.brev_permute_batched([])  # count 0: no-op
    L = brev_lib.lib()
    t = device_array(1, 12, 8)
    import ctypes
    # overlapping arrays are refused
    ptrs = (ctypes.c_void_p * 2)(t.data_ptr(), t.data_ptr() + 8 * 16)
    ks = (ctypes.c_int * 2)(10, 10)
    c0 = brev_lib.brev_launch_count()
    assert L.brev_permute_batched(ptrs, ks, 2, 8, None) == 3
    ks_bad = (ctypes.c_int * 2)(10, 99)
    ptrs2 = (ctypes.c_void_p * 2)(t.data_ptr(), t.data_ptr() + 8 * 2048)
    assert L.brev_permute_batched(ptrs2, ks_bad, 2, 8, None) == 1
    assert L.brev_permute_batched(ptrs2, ks, -1, 8, None) == 1
    assert brev_lib.brev_launch_count() == c0
    # identity-size arrays (k <= 1) launch nothing
    tiny = [device_array(5, 0, 16), device_array(6, 1, 8)]
    ref = [to_bytes(x) for x in tiny]
    brev_lib.brev_permute_batched(tiny)
    torch.cuda.synchronize()
    assert brev_lib.brev_launch_count() == c0
    for x, r in zip(tiny, ref):
        assert np.array_equal(to_bytes(x), r)


def test_plan_replay(brev_lib, oracle_lib, cuda_device):
    rng = np.random.default_rng(14)
    arrays, hosts = _make_batch(rng, 200, list(range(2, 19)), [8, 16], 3000)
    plan = brev_lib.BrevPlan(arrays)
    s = torch.cuda.Stream()
    c0 = brev_lib.brev_launch_count()
    plan.launch(s)
    s.synchronize()
    assert brev_lib.brev_launch_count() - c0 == 1
    exp = _expect(oracle_lib, hosts)
    for a, e, (k, E, _) in zip(arrays, exp, hosts):
        assert_bytes_equal(to_bytes(a), e, E, f"plan k={k} E={E}")
    # second replay restores the inputs; the third permutes again
    plan.launch(s)
    s.synchronize()
    for a, (k, E, h) in zip(arrays, hosts):
        assert_bytes_equal(to_bytes(a), h, E, f"plan twice k={k} E={E}")
    # contents may change between launches
    for i, a in enumerate(arrays):
        a.view(torch.uint8).zero_()
        a.view(torch.uint8)[0] = i % 251
    plan.launch(s)
    s.synchronize()
    for i, a in enumerate(arrays):
        b = to_bytes(a)
        assert b[0] == i % 251 and b[1:].sum() == 0  # element 0 is a fixed point
    plan.close()


def test_batched_config4_full_size(brev_lib, oracle_lib, cuda_device):
    """4096 arrays, k uniform in [8, 20], E uniform in {8, 16}: one captured
    persistent launch; arrays up to 2^14 compared in full, larger ones at
    sampled outputs; a second replay restores every array."""
    rng = np.random.default_rng(4)
    count = 4096
    ks = rng.integers(8, 21, size=count)
    Es = rng.choice([8, 16], size=count)
    arrays = []
    for i in range(count):
        E, k = int(Es[i]), int(ks[i])
        a = torch.empty((1 << k) * E, dtype=torch.uint8, device="cuda")
        inputs.fill_torch(a, 40000 + i, KIND[E], chunk=1 << 26)
        arrays.append(a.view(DTYPE[E]))
    t0 = brev_lib.brev_wait_timeouts()
    plan = brev_lib.BrevPlan(arrays)
    plan.launch()
    torch.cuda.synchronize()
    srng = np.random.default_rng(5)
    for i in range(count):
        E, k = int(Es[i]), int(ks[i])
        if k <= 14:
            h = inputs.array_np(40000 + i, 1 << k, KIND[E])
            assert_bytes_equal(to_bytes(arrays[i]), oracle_lib.brev_oop(h, k, E), E,
                               f"array {i} k={k} E={E}")
        elif i % 8 == 0:
            j = srng.integers(0, 1 << k, size=512, dtype=np.uint64)
            src_idx = np.array([oracle_lib.rev_bits(int(v), k) for v in j], dtype=np.uint64)
            exp = inputs.elements_np(40000 + i, src_idx, KIND[E]).reshape(-1)
            jt = torch.from_numpy(j.astype(np.int64)).cuda()
            got = arrays[i].view(torch.uint8).view(-1, E).index_select(0, jt).cpu().numpy()
            assert_bytes_equal(got.reshape(-1), exp, E, f"array {i} sampled")
    plan.launch()
    torch.cuda.synchronize()
    for i in range(0, count, 16):
        E, k = int(Es[i]), int(ks[i])
        ref = torch.empty((1 << k) * E, dtype=torch.uint8, device="cuda")
        inputs.fill_torch(ref, 40000 + i, KIND[E], chunk=1 << 26)
        assert torch.equal(arrays[i].view(torch.uint8), ref), f"array {i} after two replays"
    plan.close()
    assert brev_lib.brev_wait_timeouts() == t0


def test_batched_with_a_16gib_array(brev_lib, cuda_device):
    """A batch holding one 2^32-element float32 array (16 GiB, indices past
    2^32) and small ones: each array equals its single-array permutation, and
    a second launch restores the inputs."""
    t0 = brev_lib.brev_wait_timeouts()
    big = device_array(4321, 32, 4)
    small = [device_array(4400 + i, k, E) for i, (k, E) in enumerate(((9, 8), (14, 16), (20, 4)))]
    arrays = [big] + small
    refs = []
    for a in arrays:
        r = a.clone()
        brev_lib.brev_permute(r, in_place=True)
        refs.append(r)
    torch.cuda.synchronize()
    brev_lib.brev_permute_batched(arrays)
    torch.cuda.synchronize()
    for a, r in zip(arrays, refs):
        assert torch.equal(a.view(torch.uint8), r.view(torch.uint8))
    del refs
    brev_lib.brev_permute_batched(arrays)
    torch.cuda.synchronize()
    assert torch.equal(big.view(torch.uint8), device_array(4321, 32, 4).view(torch.uint8))
    assert brev_lib.brev_wait_timeouts() == t0


def test_host_path(brev_lib, oracle_lib, cuda_device):
    for k, E in ((0, 16), (7, 4), (20, 16), (23, 8)):
        hb = host_array(70 + k, k, E)
        h = torch.from_numpy(hb.copy()).view(DTYPE[E]).pin_memory()
        out = torch.empty_like(h).pin_memory()
        brev_lib.brev_permute_host(out, h)
        assert_bytes_equal(out.view(torch.uint8).numpy(), oracle_lib.brev_oop(hb, k, E), E,
                           f"host path k={k} E={E}")
        # in place on the host buffer, pageable memory
        pb = host_array(80 + k, k, E)
        p = torch.from_numpy(pb.copy()).view(DTYPE[E])
        brev_lib.brev_permute_host(p, p)
        assert_bytes_equal(p.view(torch.uint8).numpy(), oracle_lib.brev_oop(pb, k, E), E,
                           f"host path in place k={k} E={E}")
        # in place on a page-locked buffer: the tile kernel reads and writes it directly
        qb = host_array(90 + k, k, E)
        q = torch.from_numpy(qb.copy()).view(DTYPE[E]).pin_memory()
        brev_lib.brev_permute_host(q, q)
        assert_bytes_equal(q.view(torch.uint8).numpy(), oracle_lib.brev_oop(qb, k, E), E,
                           f"host path in place, page-locked, k={k} E={E}")
    L = brev_lib.lib()
    d = device_array(1, 10, 8)
    assert L.brev_permute_host(d.data_ptr(), d.data_ptr(), 10, 8, None) == 1  # device ptr


def test_autotune_and_cache(brev_lib, oracle_lib, cuda_device, tmp_path):
    path = str(tmp_path / "tune.json")
    brev_lib.brev_reset_tuning()  # only what this call tunes ends up in the file
    brev_lib.brev_autotune(12, 16, 8, path)
    import json
    d = json.load(open(path))
    assert d["sm_count"] > 0 and d["entries"]
    single = [e for e in d["entries"] if "batched_b" not in e]
    batched = [e for e in d["entries"] if "batched_b" in e]
    assert single and batched
    for e in single:
        assert (e["bx"], e["bz"], e["order"]) in \
            brev_lib.brev_shapes(e["elem_bytes"], e["in_place"])
    # one batched entry per k with a choice (k = 12..16, E = 8)
    assert sorted(e["log2n"] for e in batched) == list(range(12, 17))
    brev_lib.brev_reset_tuning()
    brev_lib.brev_load_tune_cache(path)
    for e in single:
        if e["elem_bytes"] == 8 and 12 <= e["log2n"] <= 16:
            assert brev_lib.brev_tile_shape(e["log2n"], 8, bool(e["in_place"])) == \
                (e["bx"], e["bz"], e["order"])
    for e in batched:
        assert brev_lib.brev_batched_shape(e["log2n"], 8) == e["batched_b"]
    # a batch under the tuned exponents gives the oracle's result
    rng = np.random.default_rng(17)
    arrays, hosts = _make_batch(rng, 40, list(range(12, 17)), [8], 1700)
    brev_lib.brev_permute_batched(arrays)
    torch.cuda.synchronize()
    for a, ex, (k, E, _) in zip(arrays, _expect(oracle_lib, hosts), hosts):
        assert_bytes_equal(to_bytes(a), ex, E, f"tuned batched k={k}")
    # tuned shapes give the same result
    for k in (12, 16):
        src = device_array(90 + k, k, 8)
        out = torch.empty_like(src)
        brev_lib.brev_permute_to(out, src)
        assert_bytes_equal(to_bytes(out), oracle_lib.brev_oop(host_array(90 + k, k, 8), k, 8),
                           8, f"tuned k={k}")
    brev_lib.brev_reset_tuning()
    brev_lib.brev_load_tune_cache(brev_lib.DEFAULT_TUNE_CACHE)  # the state later tests expect


def _cache_for(brev_lib, entries):
    """A tuning cache for the current device holding only `entries`."""
    import json
    info = brev_lib.brev_get_device_info()
    return json.dumps({"format": "brev-tune-1", "device": info["name"],
                       "sm_count": info["sm_count"], "entries": entries})


@pytest.mark.parametrize("E,b", [(4, 5), (4, 6), (8, 4), (8, 5), (16, 3), (16, 4), (16, 5)])
def test_batched_every_stage_count_and_staging(brev_lib, oracle_lib, cuda_device, tmp_path, E, b):
    """Every (tile exponent, CTA shape, stage count, row staging) the tuner
    may pick,
    imposed through a tuning cache on arrays of k = 2b + 3 (several tile
    pairs and self tiles each), batched with smaller arrays of the same
    element size whose stages are smaller, so that the launch takes the
    imposed stage count -- all bit-exact against the oracle, with no wait
    given up.  (Guided ticket splits need batches of hundreds of MB; the
    4096-array test covers them.)"""
    import ctypes
    k = 2 * b + 3
    L = brev_lib.lib()
    # stage counts that fit one CTA for this array's stage (2 .. 6)
    path = str(tmp_path / "t.json")
    tried = 0
    for warps, stages, copy in [(w, s_, c) for w in (4, 8) for s_ in range(2, 7) for c in (0, 1)]:
        with open(path, "w") as f:
            f.write(_cache_for(brev_lib, [{"elem_bytes": E, "log2n": k, "batched_b": b,
                                           "batched_stages": stages, "batched_copy": copy,
                                           "batched_warps": warps, "gbs": 1.0}]))
        brev_lib.brev_reset_tuning()
        brev_lib.brev_load_tune_cache(path)
        if brev_lib.brev_batched_shape(k, E) != b:
            continue  # not a candidate for this (k, E)
        rng = np.random.default_rng(1000 * E + 100 * warps + 10 * stages + copy)
        arrays, hosts = _make_batch(rng, 96, [k], [E], 5000 + 100 * stages + copy + warps)
        # smaller arrays ride along under the same stage count (their stages are
        # smaller: a smaller tile, or the whole array staged)
        more, more_h = _make_batch(rng, 40, list(range(2, 2 * b)), [E], 7000 + stages)
        t0 = brev_lib.brev_wait_timeouts()
        brev_lib.brev_permute_batched(arrays + more)
        torch.cuda.synchronize()
        assert brev_lib.brev_wait_timeouts() == t0
        for a, ex, (kk, EE, _) in zip(arrays + more, _expect(oracle_lib, hosts + more_h),
                                      hosts + more_h):
            assert_bytes_equal(to_bytes(a), ex, EE,
                               f"E={E} b={b} warps={warps} stages={stages} copy={copy} "
                               f"k={kk} E'={EE}")
        tried += 1
    assert tried >= 4
    brev_lib.brev_reset_tuning()
    brev_lib.brev_load_tune_cache(brev_lib.DEFAULT_TUNE_CACHE)  # the state later tests expect
