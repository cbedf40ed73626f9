"""Bit reversal fused with the first radix-2 DIT FFT stages, GPU vs the CPU
oracle (double precision).

Tolerance (derived from the arithmetic): inputs lie in [-1, 1) per
component.  After s stages every value is a sum of 2^s inputs times unit
twiddles, so |value| <= 2^s * sqrt(2).  Each stage rounds a complex product
(about 3 ulp) and a sum (1 ulp) -- or, in the double-precision multiply-add
form, two multiply-adds and 2a - a' (under 2 ulp) -- so the error grows by at
most 4 eps * 2^s * sqrt(2) per stage, and after S stages the absolute error
per component is below (S + 1) * 8 * eps * 2^S, with eps = 2^-24 for
complex<float> (float arithmetic; the oracle is exact to 2^-53 by
comparison) and 2^-53 for complex<double>.  Zero stages are the plain
permutation and must match bit for bit.

The constant butterflies (twiddles 1, -i and the eighth turns (+-1 - i)/sqrt 2,
used in the first pass and in the second pass's groups j = 0 and j = 4) stay
inside the same per-stage allowance: an eighth-turn product is one rounded
sum of the two components (|sum| <= 2^s), scaled by sqrt(1/2) inside a
multiply-add that adds a (one rounding, |a'| <= 2^s sqrt 2), then
b' = 2a - a' (one more), i.e. under (0.36 + 0.71 + 0.71) eps 2^s per
component against the 4 eps 2^s sqrt 2 = 5.66 eps 2^s allowed per stage;
the rounding of sqrt(1/2) itself adds 2^-54 relative (complex<double>) or
2^-25 (complex<float>), far inside the rest.  1 and -i are exact.
"""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, device_array, host_array, to_bytes
from paper_1708_01873_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = {8: 2.0 ** -24, 16: 2.0 ** -53}


def tol(E, S):
    return (S + 1) * 8 * EPS[E] * 2.0 ** S


def as_complex(b: np.ndarray, E: int) -> np.ndarray:
    return b.view(np.complex64 if E == 8 else np.complex128).astype(np.complex128)


def check(got_bytes, x, k, E, S, inverse, what):
    exp = __import__("oracle").fft_dit_stages(x, k, S, inverse)
    got = as_complex(got_bytes, E)
    if S == 0:
        assert np.array_equal(got, exp), what
        return
    err = np.max(np.abs(got - exp)) if got.size else 0.0
    assert err <= tol(E, S), f"{what}: max error {err:.3e} > {tol(E, S):.3e}"


@pytest.mark.parametrize("E", (8, 16))
def test_fused_stages_vs_oracle(brev_lib, oracle_lib, cuda_device, E):
    for k in list(range(0, 15)) + [17, 20]:
        for S in sorted({0, 1, 2, 3, 4, min(k, 5), min(k, 6)}):  # every pass split
            if S > k:
                continue
            for inplace in (False, True):
                for inverse in (False, True):
                    seed = 1000 * k + 10 * S + E + 2 * inverse + inplace
                    src = device_array(seed, k, E)
                    x = as_complex(host_array(seed, k, E), E)
                    if inplace:
                        brev_lib.brev_fft_stages(src, src, S, inverse)
                        out = src
                    else:
                        out = torch.empty_like(src)
                        brev_lib.brev_fft_stages(out, src, S, inverse)
                    check(to_bytes(out), x, k, E, S, inverse,
                          f"k={k} S={S} E={E} inplace={inplace} inverse={inverse}")


@pytest.mark.parametrize("E,S", [(8, 6), (16, 5)])
def test_eighth_turn_groups_both_directions(brev_lib, oracle_lib, cuda_device, E, S):
    """The largest stage count of each element size (6 for complex<float>,
    5 for complex<double>) runs the second pass's j = 0 and j = 4 groups on
    the compile-time butterflies; the inverse conjugates around them.  Both
    directions, in and out of place, several sizes, against the oracle
    within the derived tolerance."""
    for k in (S, 10, 13, 16, 19, 22):
        for inplace in (False, True):
            for inverse in (True, False):
                seed = 9000 + 10 * k + E + 2 * inverse + inplace
                src = device_array(seed, k, E)
                x = as_complex(host_array(seed, k, E), E)
                if inplace:
                    brev_lib.brev_fft_stages(src, src, S, inverse)
                    out = src
                else:
                    out = torch.empty_like(src)
                    brev_lib.brev_fft_stages(out, src, S, inverse)
                check(to_bytes(out), x, k, E, S, inverse,
                      f"k={k} S={S} E={E} inplace={inplace} inverse={inverse}")


def test_streaming_out_of_place_equals_in_place(brev_lib, oracle_lib, cuda_device):
    """complex<double> with 2^5 x 2^5 tiles and more units than resident
    slots runs the streaming kernels: one CTA per slot, units claimed from a
    counter.  Out of place (k >= 20 on GB300) the unit is a tile and the next
    one is loaded while the current one is computed; in place (k >= 21) the
    unit is a tile pair, one buffer per CTA.  Both run the same butterflies
    as the one-unit-per-CTA kernels, so out of place and in place must agree
    byte for byte at every size: one unit per CTA in both modes (k <= 19),
    streaming out of place only (k = 20), a few claims per CTA in both
    (k = 21) and many (k = 23), for every pass split.  Up to k = 21 the
    results are also checked against the oracle."""
    for k in (6, 10, 16, 20, 21, 23):
        for S in (0, 1, 3, 4, 5):
            if S > k:
                continue
            for inverse in (False, True):
                seed = 11000 + 10 * k + S + inverse
                src = device_array(seed, k, 16)
                out = torch.empty_like(src)
                brev_lib.brev_fft_stages(out, src, S, inverse)
                brev_lib.brev_fft_stages(src, src, S, inverse)
                torch.cuda.synchronize()
                assert torch.equal(out.view(torch.uint8), src.view(torch.uint8)), \
                    f"k={k} S={S} inverse={inverse}: out of place differs from in place"
                if k <= 21:
                    x = as_complex(host_array(seed, k, 16), 16)
                    check(to_bytes(out), x, k, 16, S, inverse,
                          f"k={k} S={S} inverse={inverse}")


def test_streaming_fft_captured_in_graph(brev_lib, cuda_device):
    """The streaming complex<double> kernels enqueue a stream-ordered
    allocation of their 16-byte unit counter, its memset, the kernel and the
    counter's release: all capturable.  Capture each mode once (k = 21, where
    both modes stream) and replay it twice; every replay equals the eager
    call byte for byte (in place, the input is restored between replays)."""
    k, S = 21, 5
    src = device_array(12000, k, 16)
    ref = torch.empty_like(src)
    brev_lib.brev_fft_stages(ref, src, S, False)  # eager: also sets the kernels' smem limits
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    out = torch.empty_like(src)
    work = src.clone()
    for inplace in (False, True):
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            if inplace:
                brev_lib.brev_fft_stages(work, work, S, False, stream=s)
            else:
                brev_lib.brev_fft_stages(out, src, S, False, stream=s)
        for replay in range(2):
            if inplace:
                work.copy_(src)
            else:
                out.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            got = work if inplace else out
            assert torch.equal(got.view(torch.uint8), ref.view(torch.uint8)), \
                f"inplace={inplace} replay {replay}"
        del g


@pytest.mark.parametrize("E", (8, 16))
def test_full_fft_small_arrays(brev_lib, oracle_lib, cuda_device, E):
    """All stages in one CTA for arrays that fit: the whole FFT."""
    for k in range(1, 12):
        seed = 5000 + k + E
        src = device_array(seed, k, E)
        x = as_complex(host_array(seed, k, E), E)
        out = torch.empty_like(src)
        brev_lib.brev_fft_stages(out, src, k)
        check(to_bytes(out), x, k, E, k, False, f"full FFT k={k}")
        assert np.allclose(as_complex(to_bytes(out), E), np.fft.fft(x),
                           atol=tol(E, k) * 4)


@pytest.mark.parametrize("k,E,S,inverse,inplace", [
    (26, 8, 6, False, False), (26, 16, 5, False, False), (27, 8, 5, False, False),
    (26, 16, 5, True, False), (25, 8, 6, True, False), (26, 16, 5, False, True),
    # the bench's complex<double> workload (4 GiB), both streaming kernels
    (28, 16, 5, False, False), (28, 16, 5, True, True),
    # the largest array the call accepts (k = 31, 32 GiB), in place
    (31, 16, 5, False, True)])
def test_fused_full_size_sampled_blocks(brev_lib, oracle_lib, cuda_device, k, E, S, inverse,
                                        inplace):
    """After S stages, output block b (2^S elements) is the S-stage result of
    the inputs spaced n / 2^S apart starting at rev_{k-S}(b) (pinned on the
    oracle); sampled blocks are checked against the oracle on those inputs,
    regenerated from the seed.  In place the result overwrites the input."""
    seed = 7000 + k
    src = device_array(seed, k, E)
    if inplace:
        out = src
    else:
        out = torch.empty_like(src)
    brev_lib.brev_fft_stages(out, src, S, inverse)
    torch.cuda.synchronize()
    n, m = 1 << k, 1 << S
    rng = np.random.default_rng(k)
    blocks = np.concatenate([rng.integers(0, n // m, size=64), [0, n // m - 1]])
    got = out.view(torch.uint8).view(-1, m * E)
    for b in blocks.tolist():
        r = oracle_lib.rev_bits(b, k - S)
        idx = np.arange(r, n, n // m, dtype=np.uint64)
        sub = as_complex(inputs.elements_np(seed, idx, KIND[E]).reshape(-1), E)
        exp = oracle_lib.fft_dit_stages(sub, S, S, inverse)
        g = as_complex(got[b].cpu().numpy(), E)
        err = np.max(np.abs(g - exp))
        assert err <= tol(E, S), f"block {b}: {err:.3e}"


def test_fused_errors(brev_lib, cuda_device):
    L = brev_lib.lib()
    t = device_array(1, 20, 16)
    p = t.data_ptr()
    c0 = brev_lib.brev_launch_count()
    assert L.brev_fft_stages(p, p, 20, 4, 3, 0, None) == 1      # not a complex size
    assert L.brev_fft_stages(p, p, 20, 16, 21, 0, None) == 1    # more stages than bits
    assert L.brev_fft_stages(p, p, 20, 16, 9, 0, None) == 6     # too many for a tile row
    assert L.brev_fft_stages(p + 8, p + 8, 10, 16, 2, 0, None) == 2
    assert brev_lib.brev_launch_count() == c0
