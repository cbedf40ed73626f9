"""Transpositions, even-odd step, perfect shuffle, segmented and recursive
bit reversal on the GPU vs the CPU oracle (bit-exact)."""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, assert_bytes_equal, device_array, host_array, to_bytes

pytestmark = pytest.mark.gpu

ES = (16, 8, 4, 2, 1)
SHAPES = [(0, 0), (0, 6), (6, 0), (1, 1), (1, 12), (12, 1), (2, 10), (10, 2), (5, 5),
          (7, 9), (9, 7), (11, 11), (3, 16), (16, 3), (13, 8)]


@pytest.mark.parametrize("E", ES)
def test_transpose_out_of_place(brev_lib, oracle_lib, cuda_device, E):
    for a, c in SHAPES:
        k = a + c
        seed = 100 * a + c + E
        src = device_array(seed, k, E)
        dst = torch.empty_like(src)
        brev_lib.brev_transpose(dst, src, a, c)
        exp = oracle_lib.transpose(host_array(seed, k, E), a, c, E)
        assert_bytes_equal(to_bytes(dst), exp, E, f"transpose {a}x{c} E={E}")


@pytest.mark.parametrize("E", ES)
def test_transpose_in_place_square(brev_lib, oracle_lib, cuda_device, E):
    for a in (0, 1, 2, 4, 5, 6, 7, 8, 9, 11):
        seed = 300 + a + E
        buf = device_array(seed, 2 * a, E)
        brev_lib.brev_transpose(buf, buf, a, a)
        exp = oracle_lib.transpose(host_array(seed, 2 * a, E), a, a, E)
        assert_bytes_equal(to_bytes(buf), exp, E, f"in-place transpose {a} E={E}")


@pytest.mark.parametrize("E", (8, 4, 2))
def test_transpose_unaligned(brev_lib, oracle_lib, cuda_device, E):
    for a, c in ((4, 7), (9, 3), (6, 6)):
        n = 1 << (a + c)
        big = device_array(500 + a + c, a + c, E, extra_elems=1)
        src = big[1:1 + n]
        host = to_bytes(src)
        out_big = torch.zeros_like(big)
        dst = out_big[1:1 + n]
        brev_lib.brev_transpose(dst, src, a, c)
        assert_bytes_equal(to_bytes(dst), oracle_lib.transpose(host, a, c, E), E,
                           f"unaligned transpose {a}x{c}")


@pytest.mark.parametrize("E", ES)
def test_even_odd_and_shuffle(brev_lib, oracle_lib, cuda_device, E):
    for k in list(range(0, 16)) + [20, 22]:
        seed = 600 + k + E
        src = device_array(seed, k, E)
        h = host_array(seed, k, E)
        eo = torch.empty_like(src)
        brev_lib.brev_even_odd(eo, src)
        assert_bytes_equal(to_bytes(eo), oracle_lib.even_odd(h, k, E), E, f"even-odd k={k}")
        sh = torch.empty_like(src)
        brev_lib.brev_perfect_shuffle(sh, src)
        assert_bytes_equal(to_bytes(sh), oracle_lib.perfect_shuffle(h, k, E), E,
                           f"shuffle k={k}")
        back = torch.empty_like(src)
        brev_lib.brev_perfect_shuffle(back, eo)
        assert torch.equal(back.view(torch.uint8), src.view(torch.uint8))


@pytest.mark.parametrize("E", ES)
def test_segments(brev_lib, oracle_lib, cuda_device, E):
    for s_log, m in ((0, 9), (3, 5), (4, 12), (6, 14), (2, 18), (10, 8), (5, 1), (7, 0)):
        seed = 700 + s_log * 31 + m + E
        k = s_log + m
        buf = device_array(seed, k, E)
        h = host_array(seed, k, E)
        brev_lib.brev_permute_segments(buf, s_log)
        seg = (1 << m) * E
        exp = np.concatenate([oracle_lib.brev_oop(h[i * seg:(i + 1) * seg], m, E)
                              for i in range(1 << s_log)])
        assert_bytes_equal(to_bytes(buf), exp, E, f"segments 2^{s_log} x 2^{m} E={E}")


@pytest.mark.parametrize("E", ES)
def test_recursive_method(brev_lib, oracle_lib, cuda_device, E):
    for k in list(range(0, 15)) + [17, 20, 21]:
        seed = 800 + k + E
        buf = device_array(seed, k, E)
        brev_lib.brev_permute_recursive(buf)
        exp = oracle_lib.brev_oop(host_array(seed, k, E), k, E)
        assert_bytes_equal(to_bytes(buf), exp, E, f"recursive k={k} E={E}")


def test_recursive_full_size_equals_one_pass(brev_lib, cuda_device):
    for k, E in ((26, 16), (27, 8), (28, 4)):
        a = device_array(900 + k, k, E)
        b = a.clone()
        brev_lib.brev_permute_recursive(a)
        brev_lib.brev_permute(b, in_place=True)
        assert torch.equal(a.view(torch.uint8), b.view(torch.uint8))


def test_transpose_full_size_twice_identity(brev_lib, cuda_device):
    for a, c, E in ((14, 14, 16), (20, 8, 8), (27, 1, 4), (1, 27, 16)):
        src = device_array(950 + a, a + c, E)
        t = torch.empty_like(src)
        brev_lib.brev_transpose(t, src, a, c)
        back = torch.empty_like(src)
        brev_lib.brev_transpose(back, t, c, a)
        assert torch.equal(back.view(torch.uint8), src.view(torch.uint8))


def test_transpose_in_place_full_size_equals_out_of_place(brev_lib, cuda_device):
    """16384 x 16384 complex<double> (4 GiB) and 8192 x 8192 float32 in
    place (the pipelined tile-pair kernel) against the out-of-place
    transposition, then in place again back to the input."""
    t0 = brev_lib.brev_wait_timeouts()
    for a, E in ((14, 16), (13, 4)):
        src = device_array(970 + a, 2 * a, E)
        ref = torch.empty_like(src)
        brev_lib.brev_transpose(ref, src, a, a)
        buf = src.clone()
        brev_lib.brev_transpose(buf, buf, a, a)
        assert torch.equal(buf.view(torch.uint8), ref.view(torch.uint8)), (a, E)
        brev_lib.brev_transpose(buf, buf, a, a)
        assert torch.equal(buf.view(torch.uint8), src.view(torch.uint8)), (a, E)
        del src, ref, buf
    assert brev_lib.brev_wait_timeouts() == t0


def test_transpose_past_2_to_32_elements(brev_lib, cuda_device):
    """65536 x 65536 uint32 (16 GiB, indices past 2^32): in place equals
    out of place, and transposing back restores the input."""
    t0 = brev_lib.brev_wait_timeouts()
    a, E = 16, 4
    src = device_array(991, 2 * a, E)
    ref = torch.empty_like(src)
    brev_lib.brev_transpose(ref, src, a, a)
    buf = src.clone()
    brev_lib.brev_transpose(buf, buf, a, a)
    assert torch.equal(buf.view(torch.uint8), ref.view(torch.uint8))
    del ref
    brev_lib.brev_transpose(buf, buf, a, a)
    assert torch.equal(buf.view(torch.uint8), src.view(torch.uint8))
    assert brev_lib.brev_wait_timeouts() == t0


def test_transpose_in_place_captured_in_graph(brev_lib, oracle_lib, cuda_device):
    """The in-place transposition enqueues only capturable work (a
    stream-ordered allocation, a memset and the kernel): capture it once,
    replay twice (the second replay restores the input)."""
    a, E = 9, 8
    buf = device_array(990, 2 * a, E)
    h = host_array(990, 2 * a, E)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        brev_lib.brev_transpose(buf, buf, a, a, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert_bytes_equal(to_bytes(buf), oracle_lib.transpose(h, a, a, E), E, "replay 1")
    g.replay()
    torch.cuda.synchronize()
    assert_bytes_equal(to_bytes(buf), h, E, "replay 2")


def test_calls_after_a_synchronise_do_not_remap_workspace(brev_lib, oracle_lib, cuda_device):
    """The in-place transposition takes a 16-byte stream-ordered ticket
    counter per call.  Its workspace comes from the library's own pool,
    which keeps memory reserved across synchronisations, so a call made
    right after a synchronise costs the host a few microseconds, not the
    ~0.1 ms of mapping memory again that the device's default pool (release
    threshold 0) charged.  Median of 11 synchronised calls, generous bound;
    the results stay exact (an even number of transpositions restores the
    input)."""
    import time
    a, E = 10, 16
    buf = device_array(991, 2 * a, E)
    h = host_array(991, 2 * a, E)
    L = brev_lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    p = buf.data_ptr()
    host_us = []
    for _ in range(12):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert L.brev_transpose(p, p, a, a, E, stream) == 0
        host_us.append((time.perf_counter() - t0) * 1e6)
    torch.cuda.synchronize()
    assert_bytes_equal(to_bytes(buf), h, E, "12 in-place transpositions")
    med = sorted(host_us[1:])[len(host_us[1:]) // 2]
    assert med < 50.0, f"median host time per synchronised call {med:.1f} us: {host_us}"


def test_transpose_errors(brev_lib, cuda_device):
    L = brev_lib.lib()
    t = device_array(1, 12, 8)
    p = t.data_ptr()
    c0 = brev_lib.brev_launch_count()
    assert L.brev_transpose(p, p, 5, 7, 8, None) == 6      # non-square in place
    assert L.brev_transpose(p, p, -1, 3, 8, None) == 1
    assert L.brev_transpose(p + 8, p, 5, 6, 8, None) == 3   # partial overlap
    assert L.brev_even_odd(p, p, 12, 8, None) == 6
    assert brev_lib.brev_launch_count() == c0
