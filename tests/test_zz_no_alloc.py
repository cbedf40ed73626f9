"""The no-allocation batched entry point (brev_permute_batched_noalloc).

Some callers cannot allocate device memory: their device memory belongs to
another allocator, or a cudaMalloc (which can synchronise the device or fail
under fragmentation) is not acceptable where they run.  For them the library
keeps the batched launch's scratch -- ticket counter and per-array
descriptors -- in a fixed device array instead of workspace allocated per
call.  This test calls that entry point through the C ABI twice in a row, on
two different batches, and compares each result byte for byte with
brev_permute_batched_mixed (the entry point that allocates its workspace) on
identical copies of the inputs.  Around each call it also checks what the
entry point exists for: the device's free memory and the library's workspace
pool are the same before and after.  A batch of the largest allowed size
(mixed sizes, so the last descriptor slot holds an ordinary array) matches
the allocating entry point too, and one larger than the fixed array is
refused with a clear error and nothing launched.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import device_array, to_bytes

pytestmark = pytest.mark.gpu

MAX_ARRAYS = 1024  # BREV_NOALLOC_MAX_ARRAYS in include/brev.h


def _batch(seed, count, ks, Es):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.choice(ks))
        E = int(rng.choice(Es))
        out.append(device_array(seed * 10000 + i, k, E))
    return out


def _c_arrays(tensors):
    n = len(tensors)
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in tensors])
    ks = (ctypes.c_int * n)(*[t.numel().bit_length() - 1 for t in tensors])
    es = (ctypes.c_int * n)(*[t.element_size() for t in tensors])
    return ptrs, ks, es


def _call(L, fn_name, tensors, stream):
    ptrs, ks, es = _c_arrays(tensors)
    return getattr(L, fn_name)(ptrs, ks, es, len(tensors), stream)


def _device_memory_state(brev_lib):
    """(free device bytes, workspace pool reserved, pool used), read with
    the device idle (a synchronise first, so that the pool has already
    given back what it releases at synchronisation)."""
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    reserved, used = brev_lib.brev_workspace_bytes()
    return free, reserved, used


def _noalloc_checked(brev_lib, L, arrays, stream):
    """Call the no-allocation entry point and check that the device's free
    memory and the workspace pool did not move."""
    before = _device_memory_state(brev_lib)
    rc = _call(L, "brev_permute_batched_noalloc", arrays, stream)
    assert rc == 0, brev_lib.brev_last_error()
    after = _device_memory_state(brev_lib)
    assert after == before, f"device memory moved: {before} -> {after}"


def _first_call(brev_lib, L, stream):
    """The first call on a device looks up the scratch array's address (and
    may load the library's module, which holds that array); the calls whose
    memory is checked come after it."""
    warm = [device_array(7, 10, 16)]
    assert _call(L, "brev_permute_batched_noalloc", warm, stream) == 0, brev_lib.brev_last_error()


def test_noalloc_matches_allocating_entry_point_twice(brev_lib, cuda_device):
    L = brev_lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    _first_call(brev_lib, L, stream)
    batches = [
        # mixed sizes and element sizes, including small whole-array
        # staging, identity sizes and a 1-byte fallback array
        _batch(1, 300, list(range(0, 19)), [4, 8, 16]) + _batch(2, 5, [9, 14], [1]),
        # a different, smaller batch: the fixed array still holds the first
        # call's descriptors and counter, which must not leak into this one
        _batch(3, 40, list(range(10, 21)), [8, 16]),
    ]
    for call, arrays in enumerate(batches):
        ref = [a.clone() for a in arrays]
        before = [to_bytes(a) for a in arrays]
        _noalloc_checked(brev_lib, L, arrays, stream)
        rc = _call(L, "brev_permute_batched_mixed", ref, stream)
        assert rc == 0, brev_lib.brev_last_error()
        torch.cuda.synchronize()
        changed = 0
        for i, (a, r) in enumerate(zip(arrays, ref)):
            got, exp = to_bytes(a), to_bytes(r)
            assert np.array_equal(got, exp), f"call {call}, array {i}: differs"
            changed += int(not np.array_equal(got, before[i]))
        assert changed > len(arrays) // 2  # the permutation really ran


def test_noalloc_rejects_too_many_arrays(brev_lib, cuda_device):
    L = brev_lib.lib()
    t = device_array(9, 16, 16)
    n = MAX_ARRAYS + 1
    ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() + 16 * 16 * i for i in range(n)])
    ks = (ctypes.c_int * n)(*([4] * n))
    es = (ctypes.c_int * n)(*([16] * n))
    c0 = brev_lib.brev_launch_count()
    rc = L.brev_permute_batched_noalloc(ptrs, ks, es, n, None)
    assert rc == 1  # BREV_ERR_INVALID_ARG
    assert "exceeds" in brev_lib.brev_last_error()
    assert brev_lib.brev_launch_count() == c0
    # the largest allowed batch works, and matches the allocating entry
    # point array for array (mixed k and E, so every descriptor slot up to
    # the last holds a different shape)
    arrays = _batch(5, MAX_ARRAYS, list(range(2, 13)), [4, 8, 16])
    ref = [a.clone() for a in arrays]
    stream = torch.cuda.current_stream().cuda_stream
    _first_call(brev_lib, L, stream)
    _noalloc_checked(brev_lib, L, arrays, stream)
    assert _call(L, "brev_permute_batched_mixed", ref, stream) == 0, brev_lib.brev_last_error()
    torch.cuda.synchronize()
    for i, (a, r) in enumerate(zip(arrays, ref)):
        assert np.array_equal(to_bytes(a), to_bytes(r)), f"array {i} differs"
