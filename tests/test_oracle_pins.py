"""The CPU oracle pinned to the paper (runs without a GPU).

Every check in ``pins.py`` runs against the oracle.  The mutation tests then
plant typical mistakes in Python copies of the oracle (a dropped bit, a
rotation for a reversal, a partly copied element, a missing comparison in
the swap loop, an off-by-one shift) and require that some check fails for
each, which shows the pins are strong enough to catch them.
"""
import numpy as np
import pytest

import pins


class OracleImpl:
    def __init__(self, oracle):
        self.o = oracle

    def rev(self, i, k):
        return self.o.rev_bits(i, k)

    def oop(self, src, k, E):
        return self.o.brev_oop(src, k, E)

    def inplace(self, buf, k, E):
        return self.o.brev_inplace(buf, k, E)


@pytest.fixture(scope="module")
def impl(oracle_lib):
    return OracleImpl(oracle_lib)


def test_p1_worked_example(impl):
    pins.check_worked_example(impl)


def test_p2_even_odd_golden():
    pins.check_even_odd_golden()


def test_p3_brute_force(impl):
    pins.check_brute_force(impl, kmax=12)


def test_p4_involution(impl):
    pins.check_involution(impl, ks=range(0, 19))


def test_p4_involution_large(impl, oracle_lib):
    # k = 22, 16-byte elements (64 MiB), out-of-place twice and in-place twice
    k, E = 22, 16
    x = pins.fingerprint_elems(1 << k, E, salt=22)
    y = oracle_lib.brev_oop(x, k, E)
    assert not np.array_equal(x, y)
    assert np.array_equal(oracle_lib.brev_oop(y, k, E), x)
    b = x.copy()
    oracle_lib.brev_inplace(b, k, E)
    assert np.array_equal(b, y)


def test_p5_stockham(impl):
    pins.check_stockham(impl, kmax=13)


def test_p6_xor_induction(impl):
    pins.check_xor_induction(impl, kmax=16)


def test_p7_counts(impl):
    pins.check_counts(impl, kmax=20)


def test_p8_branch_and_bound_classes(impl):
    pins.check_classes(impl, kmax=12)


def test_p9_concatenation(impl):
    pins.check_concatenation(impl)


def test_p10_odd_k(impl):
    pins.check_odd_k(impl)


def test_p11_cobra_schedule(impl):
    pins.check_cobra_schedule(impl, kmax=11)


def test_p12_recursive_square(impl):
    pins.check_recursive_square(impl)


def test_multithreaded_oracle_matches(oracle_lib):
    for k, E in ((0, 4), (5, 8), (17, 16), (20, 4)):
        x = pins.fingerprint_elems(1 << k, E, salt=k)
        for t in (1, 3, 8):
            got, used = oracle_lib.brev_oop_mt(x, k, E, t)
            assert used >= 1
            assert np.array_equal(got, oracle_lib.brev_oop(x, k, E))


def test_gather_matches(oracle_lib):
    k, E = 15, 8
    x = pins.fingerprint_elems(1 << k, E, salt=1)
    full = oracle_lib.brev_oop(x, k, E).reshape(-1, E)
    idx = np.array([0, 1, 7, 1000, (1 << k) - 1, 12345], dtype=np.uint64)
    got = oracle_lib.brev_gather(x, idx, k, E).reshape(-1, E)
    assert np.array_equal(got, full[idx.astype(np.int64)])


def test_oracle_rejects_bad_args(oracle_lib):
    L = oracle_lib.lib()
    assert L.oracle_brev_oop(None, None, 3, 4) == -1
    buf = np.zeros(64, dtype=np.uint8)
    assert L.oracle_brev_inplace(buf.ctypes.data, -1, 4) == -1
    assert L.oracle_brev_inplace(buf.ctypes.data, 3, 0) == -1


# ------------------------------------------------------------ mutants --
def _rev_vec(idx, k):
    r = np.zeros_like(idx)
    x = idx.copy()
    for _ in range(k):
        r = (r << np.uint64(1)) | (x & np.uint64(1))
        x = x >> np.uint64(1)
    return r


class _Mutant:
    """Python copy of the oracle with one planted mistake."""

    def rev_vec(self, idx, k):
        return _rev_vec(idx, k)

    def rev(self, i, k):
        return int(self.rev_vec(np.array([i], dtype=np.uint64), k)[0])

    def copy_elem(self, dst, di, src, si, E):
        dst[di] = src[si]

    def oop(self, src, k, E):
        n = 1 << k
        s = np.ascontiguousarray(src).view(np.uint8).reshape(n, E)
        d = np.zeros_like(s)
        r = self.rev_vec(np.arange(n, dtype=np.uint64), k).astype(np.int64)
        self.copy_elem(d, r, s, np.arange(n), E)
        return d.reshape(-1)

    def inplace(self, buf, k, E):
        buf[:] = self.oop(buf, k, E)
        return buf


class RotateNotReverse(_Mutant):
    def rev_vec(self, idx, k):
        if k == 0:
            return np.zeros_like(idx)
        return (idx >> np.uint64(1)) | ((idx & np.uint64(1)) << np.uint64(k - 1))


class DroppedLowBit(_Mutant):
    def rev_vec(self, idx, k):
        return _rev_vec(idx & ~np.uint64(1), k) | (idx & np.uint64(1) if k else 0)


class OffByOneWidth(_Mutant):
    def rev_vec(self, idx, k):
        return _rev_vec(idx, k + 1) & np.uint64((1 << k) - 1)


class PartialElementCopy(_Mutant):
    def copy_elem(self, dst, di, src, si, E):
        dst[di, : max(E - 1, 0)] = src[si, : max(E - 1, 0)]


class SwapWithoutComparison(_Mutant):
    def inplace(self, buf, k, E):
        n = 1 << k
        a = buf.reshape(n, E)
        for i in range(n):
            r = self.rev(i, k)
            t = a[i].copy()
            a[i] = a[r]
            a[r] = t
        return buf


class InPlaceWithoutCopy(_Mutant):
    """The in-place definition applied to the buffer itself, without a copy
    of the input: later reads see elements already overwritten."""

    def inplace(self, buf, k, E):
        n = 1 << k
        a = buf.reshape(n, E)
        r = self.rev_vec(np.arange(n, dtype=np.uint64), k).astype(np.int64)
        for i in range(n):
            a[r[i]] = a[i]
        return buf


class HalvesSwapped(_Mutant):
    """rev(x y) computed as rev(x) rev(y) (operands of the concatenation
    transposed)."""

    def rev_vec(self, idx, k):
        h = k // 2
        lo = idx & np.uint64((1 << h) - 1)
        hi = idx >> np.uint64(h)
        return (_rev_vec(hi, k - h) << np.uint64(h)) | _rev_vec(lo, h)


@pytest.mark.parametrize("mutant", [RotateNotReverse, DroppedLowBit, OffByOneWidth,
                                    PartialElementCopy, SwapWithoutComparison,
                                    InPlaceWithoutCopy, HalvesSwapped])
def test_pins_catch_planted_mistake(mutant):
    m = mutant()
    fast = [
        lambda: pins.check_worked_example(m),
        lambda: pins.check_brute_force(m, kmax=6),
        lambda: pins.check_involution(m, ks=range(0, 9), Es=(4, 16)),
        lambda: pins.check_stockham(m, kmax=6),
        lambda: pins.check_xor_induction(m, kmax=8),
        lambda: pins.check_counts(m, kmax=8),
        lambda: pins.check_classes(m, kmax=6),
        lambda: pins.check_concatenation(m, trials=300),
    ]
    caught = 0
    for chk in fast:
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught {mutant.__name__}"


# ------------------------------------------------ transposition oracles --
def test_even_odd_golden_on_c_oracle(oracle_lib):
    """P2 on the C oracle: [0..7] -> [0,2,4,6,1,3,5,7] (Introduction)."""
    g = pins.read_golden("even_odd_k3.txt")
    exp = [int(x) for x in g["output"]]
    for E in (1, 4, 16):
        got = pins.decode_index(oracle_lib.even_odd(pins.index_elems(8, E), 3, E), E).tolist()
        assert got == exp


def test_transpose_matches_numpy(oracle_lib):
    """A library routine as the pin: numpy's transpose of the matrix view."""
    for a, c in ((0, 0), (0, 3), (3, 0), (1, 5), (5, 1), (4, 4), (6, 3), (2, 9)):
        for E in (1, 4, 16):
            x = pins.fingerprint_elems(1 << (a + c), E, salt=a * 10 + c)
            exp = x.reshape(1 << a, 1 << c, E).transpose(1, 0, 2).reshape(-1)
            assert np.array_equal(oracle_lib.transpose(x, a, c, E), exp), (a, c, E)


def test_even_odd_is_half_by_two_transpose_and_shuffle_inverts(oracle_lib):
    for k in range(1, 14):
        for E in (4, 8):
            x = pins.fingerprint_elems(1 << k, E, salt=k)
            eo = oracle_lib.even_odd(x, k, E)
            assert np.array_equal(eo, oracle_lib.transpose(x, k - 1, 1, E))
            assert np.array_equal(oracle_lib.perfect_shuffle(eo, k, E), x)
            assert np.array_equal(oracle_lib.perfect_shuffle(x, k, E),
                                  oracle_lib.transpose(x, 1, k - 1, E))


def test_stockham_recursion_with_c_even_odd(oracle_lib):
    """P5 with the C even-odd step: even-odd, then each half recursively,
    equals the bit-reversed permutation."""
    def rec(x, k, E):
        if k == 0:
            return x.copy()
        eo = oracle_lib.even_odd(x, k, E)
        h = (1 << (k - 1)) * E
        return np.concatenate([rec(eo[:h], k - 1, E), rec(eo[h:], k - 1, E)])
    for k in range(0, 13):
        x = pins.fingerprint_elems(1 << k, 8, salt=k)
        assert np.array_equal(rec(x, k, 8), oracle_lib.brev_oop(x, k, 8))


def test_recursive_method_with_c_transpose(oracle_lib):
    """Methods, cache-oblivious recursive method: reverse every block, square
    transpose, reverse every block again (even k), with the C transpose."""
    for k in (2, 4, 6, 8, 10, 12):
        h = k // 2
        for E in (4, 16):
            x = pins.fingerprint_elems(1 << k, E, salt=k)
            s = 1 << h
            blocks = [oracle_lib.brev_oop(x[r * s * E:(r + 1) * s * E], h, E) for r in range(s)]
            t = oracle_lib.transpose(np.concatenate(blocks), h, h, E)
            blocks = [oracle_lib.brev_oop(t[r * s * E:(r + 1) * s * E], h, E) for r in range(s)]
            assert np.array_equal(np.concatenate(blocks), oracle_lib.brev_oop(x, k, E))


# ------------------------------------------- bit reversal + FFT stages --
def test_fft_stages_full_equals_numpy_dft(oracle_lib):
    """stages = k is the whole FFT: numpy's FFT (a library routine) and, for
    small n, the DFT sum written out."""
    rng = np.random.default_rng(1)
    for k in range(0, 13):
        x = rng.uniform(-1, 1, 1 << k) + 1j * rng.uniform(-1, 1, 1 << k)
        got = oracle_lib.fft_dit_stages(x, k, k)
        exp = np.fft.fft(x)
        assert np.max(np.abs(got - exp)) <= 1e-12 * max(1, np.max(np.abs(exp))) * (k + 1)
        inv = oracle_lib.fft_dit_stages(x, k, k, inverse=True)
        assert np.max(np.abs(inv - np.fft.ifft(x) * (1 << k))) <= 1e-12 * (1 << k) * (k + 1)
    for k in (2, 3, 5):
        n = 1 << k
        x = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
        dft = np.array([sum(x[t] * np.exp(-2j * np.pi * f * t / n) for t in range(n))
                        for f in range(n)])
        assert np.allclose(oracle_lib.fft_dit_stages(x, k, k), dft, atol=1e-12)


def test_fft_stages_partial_structure(oracle_lib):
    """stages = 0 is the permutation; after s stages every block of 2^s
    consecutive outputs is the 2^s-point DFT of its (bit-reversed) inputs,
    i.e. the DFT of the inputs spaced n / 2^s apart."""
    rng = np.random.default_rng(2)
    for k in (4, 7, 10):
        n = 1 << k
        x = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
        perm = oracle_lib.brev_oop(x.astype(np.complex128), k, 16).view(np.complex128)
        assert np.array_equal(oracle_lib.fft_dit_stages(x, k, 0), perm)
        for s in range(1, k + 1):
            got = oracle_lib.fft_dit_stages(x, k, s)
            m = 1 << s
            for blk in range(0, n // m, max(1, (n // m) // 4)):
                # block `blk` holds inputs with index = rev_{k-s}(blk) + t * (n / m)
                r = oracle_lib.rev_bits(blk, k - s)
                sub = x[r::n // m]
                assert np.allclose(got[blk * m:(blk + 1) * m], np.fft.fft(sub), atol=1e-11)


def test_fft_stages_impulse_and_linearity(oracle_lib):
    k = 9
    n = 1 << k
    d = np.zeros(n, dtype=np.complex128)
    d[0] = 1
    assert np.allclose(oracle_lib.fft_dit_stages(d, k, k), np.ones(n))
    rng = np.random.default_rng(3)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    for s in (1, 4, k):
        lhs = oracle_lib.fft_dit_stages(2 * a - 3j * b, k, s)
        rhs = 2 * oracle_lib.fft_dit_stages(a, k, s) - 3j * oracle_lib.fft_dit_stages(b, k, s)
        assert np.allclose(lhs, rhs, atol=1e-10)
