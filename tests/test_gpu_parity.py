"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bit-exact comparison (elements are moved, never computed).  Sizes span
several tiles with ragged middles (odd k - 2b), every compiled tile shape,
the element-wide path for pointers that are not 16-byte aligned, the
degenerate sizes k = 0 and 1, and the full-size workloads (4 GiB arrays)
checked at sampled outputs the oracle computes one by one.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, assert_bytes_equal, device_array, host_array, to_bytes
from paper_1708_01873_gb300 import inputs

pytestmark = pytest.mark.gpu

ES = (16, 8, 4, 2, 1)


@pytest.mark.parametrize("E", ES)
def test_out_of_place_all_k(brev_lib, oracle_lib, cuda_device, E):
    for k in range(0, 23):
        seed = 1000 + 31 * k + E
        src = device_array(seed, k, E)
        dst = torch.empty_like(src)
        brev_lib.brev_permute_to(dst, src)
        exp = oracle_lib.brev_oop(host_array(seed, k, E), k, E)
        assert_bytes_equal(to_bytes(dst), exp, E, f"oop k={k} E={E}")
        assert_bytes_equal(to_bytes(src), host_array(seed, k, E), E, "source untouched")


@pytest.mark.parametrize("E", ES)
def test_in_place_all_k(brev_lib, oracle_lib, cuda_device, E):
    for k in range(0, 23):
        seed = 2000 + 31 * k + E
        buf = device_array(seed, k, E)
        brev_lib.brev_permute(buf, in_place=True)
        exp = host_array(seed, k, E).copy()
        oracle_lib.brev_inplace(exp, k, E)
        assert_bytes_equal(to_bytes(buf), exp, E, f"in-place k={k} E={E}")


@pytest.mark.parametrize("E", ES)
def test_single_pointer_out_of_place(brev_lib, oracle_lib, cuda_device, E):
    for k in (0, 1, 5, 13, 18):
        seed = 3000 + k + E
        n = 1 << k
        buf = torch.empty(2 * n * E, dtype=torch.uint8, device="cuda")
        inputs.fill_torch(buf[: n * E], seed, KIND[E])
        t = buf.view(DTYPE[E])
        brev_lib.brev_permute(t, in_place=False)
        exp = oracle_lib.brev_oop(host_array(seed, k, E), k, E)
        assert_bytes_equal(to_bytes(buf[n * E:]), exp, E, f"[src|dst] k={k} E={E}")


@pytest.mark.parametrize("E", ES)
def test_every_compiled_shape(brev_lib, oracle_lib, cuda_device, E):
    for inplace in (False, True):
        for bx, bz, order in brev_lib.brev_shapes(E, inplace):
            # both launch orders; the blocked one needs >= 6 middle bits,
            # and odd middle widths exercise its palindromic blocks
            for k in sorted({bx + bz, bx + bz + 1, bx + bz + 2, bx + bz + 5, bx + bz + 6,
                             bx + bz + 7, 19}):
                seed = 4000 + 97 * bx + 13 * bz + k
                src = device_array(seed, k, E)
                h = host_array(seed, k, E)
                if inplace:
                    brev_lib.brev_permute_shape(src, src, bx, bz, order)
                    got = src
                else:
                    got = torch.empty_like(src)
                    brev_lib.brev_permute_shape(got, src, bx, bz, order)
                exp = oracle_lib.brev_oop(h, k, E)
                assert_bytes_equal(to_bytes(got), exp, E,
                                   f"shape {bx}x{bz} order {order} k={k} E={E} "
                                   f"inplace={inplace}")


@pytest.mark.parametrize("E", (8, 4, 2, 1))
def test_element_wide_path_unaligned(brev_lib, oracle_lib, cuda_device, E):
    """Pointers aligned to E but not to 16 bytes take the element-wide path."""
    for k in (3, 2 * ({8: 4, 4: 5, 2: 6, 1: 7}[E]), 15, 20):
        seed = 5000 + k + E
        n = 1 << k
        big = device_array(seed, k, E, extra_elems=2)
        src = big[1:1 + n]
        assert src.data_ptr() % 16 != 0
        host = to_bytes(src)
        out_big = torch.zeros_like(big)
        dst = out_big[1:1 + n]
        brev_lib.brev_permute_to(dst, src)
        assert_bytes_equal(to_bytes(dst), oracle_lib.brev_oop(host, k, E), E,
                           f"unaligned oop k={k} E={E}")
        brev_lib.brev_permute(src, in_place=True)
        exp = host.copy()
        oracle_lib.brev_inplace(exp, k, E)
        assert_bytes_equal(to_bytes(src), exp, E, f"unaligned in-place k={k} E={E}")
        # neighbours untouched
        assert to_bytes(out_big[:1]).sum() == 0 and to_bytes(out_big[-1:]).sum() == 0


def test_special_bit_patterns_preserved(brev_lib, oracle_lib, cuda_device):
    """NaNs with payloads, -0.0 and denormals move as bytes."""
    k = 12
    vals = np.array([np.nan, -0.0, 5e-324, np.inf, -np.inf, 1.0], dtype=np.float64)
    h = np.resize(vals, 1 << k).view(np.uint64).copy()
    h[::7] = 0x7FF8DEADBEEF0001  # NaN with a payload
    t = torch.from_numpy(h.view(np.float64).copy()).cuda()
    out = torch.empty_like(t)
    brev_lib.brev_permute_to(out, t)
    exp = oracle_lib.brev_oop(h.view(np.uint8), k, 8)
    assert_bytes_equal(to_bytes(out), exp, 8, "special values")


def test_in_place_twice_is_identity(brev_lib, cuda_device):
    for k, E in ((24, 16), (25, 8), (23, 4), (21, 1)):
        buf = device_array(77 + k, k, E)
        ref = buf.clone()
        brev_lib.brev_permute(buf, in_place=True)
        assert not torch.equal(buf.view(torch.uint8), ref.view(torch.uint8))
        brev_lib.brev_permute(buf, in_place=True)
        assert torch.equal(buf.view(torch.uint8), ref.view(torch.uint8))


def _sample_positions(rng, k, count=4096, runs=4, run_len=2048):
    n = 1 << k
    idx = [rng.integers(0, n, size=count, dtype=np.uint64)]
    for _ in range(runs):
        s = int(rng.integers(0, n - run_len))
        idx.append(np.arange(s, s + run_len, dtype=np.uint64))
    idx.append(np.array([0, 1, n - 2, n - 1], dtype=np.uint64))
    return np.concatenate(idx)


def _check_sampled(oracle_lib, out: torch.Tensor, seed: int, k: int, E: int, kind: str,
                   rng, what: str):
    """out[j] must equal input element rev_k(j): the oracle reverses each
    sampled j and the seeded generator regenerates that input element."""
    j = _sample_positions(rng, k)
    src_idx = np.array([oracle_lib.rev_bits(int(v), k) for v in j], dtype=np.uint64)
    exp = inputs.elements_np(seed, src_idx, kind).reshape(-1)
    jt = torch.from_numpy(j.astype(np.int64)).to(out.device)
    got = out.view(torch.uint8).view(-1, E).index_select(0, jt).cpu().numpy().reshape(-1)
    assert_bytes_equal(got, exp, E, what)


@pytest.mark.parametrize("k,E,kind,inplace", [
    (28, 16, "c128", True),    # 4 GiB complex<double>, in place
    (30, 4, "f32", True),      # 4 GiB float32, in place
    (29, 8, "c64", False),     # 4 GiB complex<float>, odd k, out of place
    (26, 16, "c128", False),
    (27, 4, "u32", False),
    # beyond 2^32 elements / bytes: 64-bit index arithmetic (16 GiB arrays)
    (32, 4, "u32", True),
    (33, 2, "u16", True),
    (34, 1, "u8", False),      # the largest log2n the API accepts
])
def test_full_size_sampled(brev_lib, oracle_lib, cuda_device, k, E, kind, inplace):
    rng = np.random.default_rng(k * 100 + E)
    seed = 9000 + k
    src = device_array(seed, k, E, kind=kind)
    if inplace:
        brev_lib.brev_permute(src, in_place=True)
        out = src
    else:
        out = torch.empty_like(src)
        brev_lib.brev_permute_to(out, src)
    torch.cuda.synchronize()
    _check_sampled(oracle_lib, out, seed, k, E, kind, rng, f"k={k} E={E} inplace={inplace}")
    # applying it again restores the input everywhere
    again = out if inplace else torch.empty_like(out)
    if inplace:
        brev_lib.brev_permute(again, in_place=True)
    else:
        brev_lib.brev_permute_to(again, out)
        del src
    ref = device_array(seed, k, E, kind=kind)
    assert torch.equal(again.view(torch.uint8), ref.view(torch.uint8))


def test_launch_count_increments(brev_lib, cuda_device):
    t = device_array(1, 16, 8)
    c0 = brev_lib.brev_launch_count()
    brev_lib.brev_permute(t, in_place=True)
    brev_lib.brev_permute(t, in_place=True)
    assert brev_lib.brev_launch_count() - c0 == 2


def test_error_statuses_launch_nothing(brev_lib, cuda_device):
    L = brev_lib.lib()
    t = device_array(3, 10, 8)
    p = t.data_ptr()
    c0 = brev_lib.brev_launch_count()
    assert L.brev_permute_to(p, p, 10, 3, None) == 1           # bad elem_bytes
    assert L.brev_permute_to(p, p, -1, 8, None) == 1           # bad k
    assert L.brev_permute_to(p, p, 35, 8, None) == 1           # k too large
    assert L.brev_permute_to(None, p, 10, 8, None) == 1        # NULL
    assert L.brev_permute_to(p + 4, p + 4, 9, 8, None) == 2    # misaligned
    assert L.brev_permute_to(p + 8, p, 9, 8, None) == 3        # partial overlap
    cpu = torch.zeros(1 << 10, dtype=torch.int64)
    assert L.brev_permute_to(cpu.data_ptr(), cpu.data_ptr(), 10, 8, None) == 1  # host ptr
    assert L.brev_permute_shape(p, p, 10, 8, 4, 5, 0, None) == 1  # in-place needs square
    assert L.brev_permute_shape(p, p, 10, 8, 9, 9, 0, None) == 1  # tile larger than array
    assert L.brev_permute_shape(p, p, 10, 8, 5, 5, 3, None) == 1  # no such order
    q = device_array(4, 10, 8)
    assert L.brev_permute_shape(q.data_ptr(), p, 10, 8, 5, 5, 2, None) == 6  # pipeline: in place only
    assert L.brev_permute_shape(p, p, 10, 8, 3, 3, 2, None) == 6  # b the pipeline does not stage
    assert brev_lib.brev_launch_count() == c0
    with pytest.raises(brev_lib.BrevError) as ei:
        brev_lib.brev_permute_shape(t, t, 3, 3)                # 64 B rows: not compiled
    assert ei.value.status_name == "BREV_ERR_UNSUPPORTED"
    with pytest.raises(ValueError):
        brev_lib.brev_permute_to(t, torch.empty(3, dtype=t.dtype, device="cuda"))


def test_past_allocation_end_rejected(brev_lib, cuda_device):
    """A request that runs past the end of its allocation is refused before
    any launch (the allocation comes straight from the driver, so its size is
    exact)."""
    L = brev_lib.lib()
    torch.cuda.synchronize()
    cu = ctypes.CDLL("libcuda.so.1")
    ptr = ctypes.c_uint64()
    assert cu.cuMemAlloc_v2(ctypes.byref(ptr), ctypes.c_size_t(1 << 20)) == 0
    try:
        c0 = brev_lib.brev_launch_count()
        assert L.brev_permute_to(ptr.value, ptr.value, 17, 16, None) == 1  # 2 MiB > 1 MiB
        assert "past the end" in brev_lib.brev_last_error()
        assert brev_lib.brev_launch_count() == c0
        assert L.brev_permute_to(ptr.value, ptr.value, 16, 16, None) == 0  # exactly fits
        torch.cuda.synchronize()
    finally:
        cu.cuMemFree_v2(ptr)
