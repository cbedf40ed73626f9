"""Independent pins for the CPU oracle (no GPU).

Each ``check_*`` function takes an implementation object exposing

    rev(i, k)              -> int      reverse the low k bits of i
    oop(src_u8, k, E)      -> u8 array the out-of-place permutation
    inplace(buf_u8, k, E)  -> buf      the in-place permutation

and raises AssertionError when the implementation disagrees with something
the paper or plain mathematics fixes.  ``tests/test_oracle_pins.py`` runs
every check against the oracle, and also against deliberately broken copies
of it, to show that each plausible mistake is caught by at least one check.

Paper passages are cited by section and paragraph title.
"""
from __future__ import annotations

import math
import os
import random

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def fingerprint_elems(n: int, E: int, salt: int = 0) -> np.ndarray:
    """n elements of E bytes in which every byte depends on the element's
    index and its byte position, so any misplaced or partly copied element
    is visible."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(E, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        v = (i * np.uint64(0x9E3779B1) + j * np.uint64(0x85EBCA77)
             + np.uint64(salt)) ^ (i >> np.uint64(8 * (E % 4)))
        v = v ^ (v >> np.uint64(13)) ^ (i >> np.uint64(5))
    b = (v & np.uint64(0xFF)).astype(np.uint8)
    # byte 0 carries the low bits of the index itself
    b[:, 0] = (np.arange(n) & 0xFF).astype(np.uint8)
    return b.reshape(-1)


def index_elems(n: int, E: int) -> np.ndarray:
    """Elements holding their own index as a little-endian integer in the
    first min(E, 8) bytes (rest zero)."""
    a = np.zeros((n, E), dtype=np.uint8)
    idx = np.arange(n, dtype=np.uint64)
    for b in range(min(E, 8)):
        a[:, b] = ((idx >> np.uint64(8 * b)) & np.uint64(0xFF)).astype(np.uint8)
    return a.reshape(-1)


def decode_index(buf: np.ndarray, E: int) -> np.ndarray:
    a = buf.reshape(-1, E)
    out = np.zeros(a.shape[0], dtype=np.uint64)
    for b in range(min(E, 8)):
        out |= a[:, b].astype(np.uint64) << np.uint64(8 * b)
    return out


def brute_rev(i: int, k: int) -> int:
    """Reverse the k-character binary string of i (the worked example
    writes indices as fixed-width bit strings)."""
    if k == 0:
        return 0
    return int(format(i, f"0{k}b")[::-1], 2)


# ------------------------------------------------------------------ P1 --
def check_worked_example(impl) -> None:
    """P1 -- Introduction, worked example: n = 8, [0..7] -> [0,4,2,6,1,5,3,7]."""
    g = read_golden("worked_example_k3.txt")
    k = int(g["k"][0])
    inp = [int(x) for x in g["input"]]
    exp = [int(x) for x in g["output"]]
    for E in (1, 4, 8, 16):
        src = index_elems(len(inp), E)
        got = decode_index(impl.oop(src, k, E), E).tolist()
        assert got == exp, (E, got, exp)
        buf = src.copy()
        got = decode_index(impl.inplace(buf, k, E), E).tolist()
        assert got == exp, ("inplace", E, got, exp)
    # the binary rendering: output position j holds the index whose 3-bit
    # string is the reverse of j's
    for a, b in zip(g["input_bin"], g["output_bin"]):
        assert impl.rev(int(a, 2), k) == int(b, 2), (a, b)


# ------------------------------------------------------------------ P3 --
def check_brute_force(impl, kmax: int = 12) -> None:
    """P3 -- rev_k(i) equals the reversed k-character binary string of i for
    every i < 2^k, k <= kmax; and the permutation of an index array puts
    at position j the index brute_rev(j)."""
    for k in range(0, kmax + 1):
        n = 1 << k
        for i in range(n):
            assert impl.rev(i, k) == brute_rev(i, k), (i, k)
        for E in (4, 16):
            got = decode_index(impl.oop(index_elems(n, E), k, E), E)
            exp = np.array([brute_rev(j, k) for j in range(n)], dtype=np.uint64)
            assert np.array_equal(got, exp), (k, E)


# ------------------------------------------------------------------ P4 --
def check_involution(impl, ks=range(0, 17), Es=(1, 2, 4, 8, 16)) -> None:
    """P4 -- Introduction: rev(rev(i)) = i, so the permutation applied twice
    is the identity; the in-place (pair swap) form equals the out-of-place
    form."""
    for k in ks:
        for E in Es:
            n = 1 << k
            x = fingerprint_elems(n, E, salt=k * 31 + E)
            y = impl.oop(x, k, E)
            assert np.array_equal(impl.oop(y, k, E), x), ("oop twice", k, E)
            b = x.copy()
            impl.inplace(b, k, E)
            assert np.array_equal(b, y), ("inplace != oop", k, E)
            impl.inplace(b, k, E)
            assert np.array_equal(b, x), ("inplace twice", k, E)
    for k in (0, 3, 9, 14):
        n = 1 << k
        for i in range(0, n, max(1, n // 512)):
            assert impl.rev(impl.rev(i, k), k) == i


# ------------------------------------------------------------------ P2 / P5 --
def even_odd(v: list) -> list:
    """One Stockham auto-sort step: even positions first, then odd ones
    (Introduction: the n/2 x 2 transposition)."""
    return v[0::2] + v[1::2]


def stockham_bitrev(v: list) -> list:
    """Recursive definition (Introduction): performing the even-odd step at
    every level of the recursion equals the bit-reversed permutation."""
    if len(v) <= 1:
        return list(v)
    e = even_odd(v)
    h = len(v) // 2
    return stockham_bitrev(e[:h]) + stockham_bitrev(e[h:])


def check_even_odd_golden() -> None:
    """P2 -- Introduction: the 4 x 2 transposition of [0..7]."""
    g = read_golden("even_odd_k3.txt")
    inp = [int(x) for x in g["input"]]
    exp = [int(x) for x in g["output"]]
    assert even_odd(inp) == exp
    r, c = int(g["matrix_rows"][0]), int(g["matrix_cols"][0])
    assert np.array(inp).reshape(r, c).T.reshape(-1).tolist() == exp


def check_stockham(impl, kmax: int = 14) -> None:
    """P5 -- the oracle equals the recursive even-odd definition."""
    rng = random.Random(5)
    for k in range(0, kmax + 1):
        n = 1 << k
        for E in (4, 8):
            x = fingerprint_elems(n, E, salt=rng.randrange(1 << 30))
            elems = [x[i * E:(i + 1) * E].tobytes() for i in range(n)]
            exp = b"".join(stockham_bitrev(elems))
            got = impl.oop(x, k, E).tobytes()
            assert got == exp, (k, E)


# ------------------------------------------------------------------ P6 --
def clz_k(d: int, k: int) -> int:
    """Leading zeros of d in a k-bit word, by scanning from the top."""
    z = 0
    for b in range(k - 1, -1, -1):
        if (d >> b) & 1:
            break
        z += 1
    return z


def xor_induction_sequence(k: int) -> list:
    """Methods, inductive XOR method: start from rev(0) = 0; for each step
    d = i XOR (i+1) has the form 0..01..1, rev(d) is d shifted left by its
    leading-zero count, and rev(i+1) = rev(i) XOR rev(d)."""
    n = 1 << k
    mask = n - 1
    out = [0] * n
    r = 0
    for i in range(n - 1):
        d = i ^ (i + 1)
        rd = (d << clz_k(d, k)) & mask
        r ^= rd
        out[i + 1] = r
    return out


def check_xor_induction(impl, kmax: int = 16) -> None:
    """P6 -- the XOR-generated sequence equals rev_k(i) for every i."""
    for k in range(1, kmax + 1):
        seq = xor_induction_sequence(k)
        n = 1 << k
        if k <= 12:
            assert seq == [impl.rev(i, k) for i in range(n)], k
        else:
            step = 7
            for i in range(0, n, step):
                assert seq[i] == impl.rev(i, k), (k, i)
            # the permutation of an index array agrees with it everywhere:
            # the element arriving at position seq[i] is i
            dst = decode_index(impl.oop(index_elems(n, 4), k, 4), 4)
            assert np.array_equal(dst[np.array(seq, dtype=np.int64)],
                                  np.arange(n, dtype=np.uint64)), k


# ------------------------------------------------------------------ P7 --
def swap_count_recurrence(b: int) -> int:
    """Methods, unrolled closed form: r(b) = 2^(b-2) + 2 r(b-2) with
    r(1) = 0 and r(2) = 1 (green + yellow + red terms)."""
    if b <= 0:
        return 0
    if b == 1:
        return 0
    if b == 2:
        return 1
    return 2 ** (b - 2) + 2 * swap_count_recurrence(b - 2)


def swap_count_closed_form(b: int) -> float:
    """The closed form printed beside the recurrence:
    r(b) = 2^(b/2) ((-1)^b (sqrt2 - 1)/4 - (1 + sqrt2)/4) + 2^(b-1)."""
    s2 = math.sqrt(2.0)
    return 2.0 ** (b / 2) * ((-1) ** b * (s2 - 1) / 4 - (1 + s2) / 4) + 2.0 ** (b - 1)


def swap_count_c_form(b: int) -> float:
    """The same as r(b) = 2^(b-1) - c 2^(b/2); read with c = +1/2 (b even)
    and c = +1/sqrt2 (b odd), the signs that agree with the closed form
    above and with r(2) = 1, r(3) = 2."""
    c = 0.5 if b % 2 == 0 else 1.0 / math.sqrt(2.0)
    return 2.0 ** (b - 1) - c * 2.0 ** (b / 2)


def check_counts(impl, kmax: int = 20) -> None:
    """P7 -- #{i : i < rev(i)} (the swaps Listing 1 performs) and the
    fixed points #{i : i = rev(i)} against the recurrence, the closed
    forms and 2^ceil(k/2)."""
    for b in range(1, 41):
        r = swap_count_recurrence(b)
        assert abs(swap_count_closed_form(b) - r) < 1e-6 * max(1, r), b
        assert abs(swap_count_c_form(b) - r) < 1e-6 * max(1, r), b
        assert 2 * r + 2 ** ((b + 1) // 2) == 2 ** b, b
    for k in range(1, kmax + 1):
        n = 1 << k
        if k <= 12:
            revs = np.array([impl.rev(i, k) for i in range(n)], dtype=np.int64)
        else:
            # rev table through the permutation of an index array
            # (dst[rev(i)] = i), valid since the involution is pinned
            revs = decode_index(impl.oop(index_elems(n, 8), k, 8), 8).astype(np.int64)
        i = np.arange(n, dtype=np.int64)
        assert int((i < revs).sum()) == swap_count_recurrence(k), k
        assert int((i == revs).sum()) == 2 ** ((k + 1) // 2), k


# ------------------------------------------------------------------ P8 --
def check_classes(impl, kmax: int = 12) -> None:
    """P8 -- Methods, unrolled branch and bound: for index = a x c with
    single outer bits a, c: 1x0 is never below its reverse, 0x1 always is,
    and 0x0 / 1x1 are below their reverse exactly when x < rev(x)."""
    for k in range(2, kmax + 1):
        for i in range(1 << k):
            a = i >> (k - 1)
            c = i & 1
            x = (i >> 1) & ((1 << (k - 2)) - 1)
            lt = i < impl.rev(i, k)
            if (a, c) == (1, 0):
                assert not lt, (k, i)
            elif (a, c) == (0, 1):
                assert lt, (k, i)
            else:
                assert lt == (x < impl.rev(x, k - 2)), (k, i)


# ------------------------------------------------------------------ P9 --
def check_concatenation(impl, trials: int = 4000) -> None:
    """P9 -- Introduction (matrix buffer method) and Methods (recursive):
    rev(x y z) = rev(z) rev(y) rev(x) for any split of the bit string."""
    rng = random.Random(9)
    for _ in range(trials):
        k = rng.randrange(0, 41)
        bx = rng.randrange(0, k + 1)
        bz = rng.randrange(0, k - bx + 1)
        by = k - bx - bz
        x = rng.randrange(1 << bx) if bx else 0
        y = rng.randrange(1 << by) if by else 0
        z = rng.randrange(1 << bz) if bz else 0
        i = (x << (by + bz)) | (y << bz) | z
        exp = ((impl.rev(z, bz) << (by + bx)) | (impl.rev(y, by) << bx)
               | impl.rev(x, bx))
        assert impl.rev(i, k) == exp, (k, bx, by, bz, x, y, z)


# ------------------------------------------------------------------ P10 --
def check_odd_k(impl, ks=(1, 3, 5, 7, 9, 11, 13)) -> None:
    """P10 -- Methods, odd number of bits: index = x y z with z one bit; the
    even-odd step gives z x y, then a (k-1)-bit reversal of each half gives
    z rev(y) rev(x) = rev(index)."""
    for k in ks:
        n = 1 << k
        for E in (4, 16):
            x = fingerprint_elems(n, E, salt=k)
            a = x.reshape(n, E)
            eo = np.concatenate([a[0::2], a[1::2]]).reshape(-1)
            h = n // 2 * E
            got = np.concatenate([impl.oop(eo[:h], k - 1, E),
                                  impl.oop(eo[h:], k - 1, E)])
            assert np.array_equal(got, impl.oop(x, k, E)), (k, E)


# ------------------------------------------------------------------ P12 --
def check_recursive_square(impl, ks=(2, 4, 6, 8, 10, 12, 14)) -> None:
    """P12 -- Methods, cache-oblivious recursive method (even k): with
    index = x y (k/2 bits each), reversing every contiguous block of y,
    transposing the square matrix, and reversing every block again gives
    the full permutation."""
    for k in ks:
        n = 1 << k
        h = k // 2
        s = 1 << h
        for E in (4, 8):
            x = fingerprint_elems(n, E, salt=3 * k)
            m = x.reshape(s, s, E)
            m = np.stack([impl.oop(m[r].reshape(-1), h, E).reshape(s, E)
                          for r in range(s)])
            m = np.ascontiguousarray(m.transpose(1, 0, 2))
            m = np.stack([impl.oop(m[r].reshape(-1), h, E).reshape(s, E)
                          for r in range(s)])
            assert np.array_equal(m.reshape(-1), impl.oop(x, k, E)), (k, E)


# ------------------------------------------------------------------ P11 --
def cobra_emulate(src: np.ndarray, k: int, E: int, bh: int, bl: int) -> np.ndarray:
    """Matrix-buffer (COBRA) schedule of the Introduction with a
    2^bh x 2^bl buffer, written out with numpy: index = x y z with
    |x| = bh, |z| = bl; for each y the buffer receives the block
    source[x y z] with rows stored at rev(x), and then output row rev(z)
    receives buffer column z, i.e. dest[rev(z) rev(y) rev(x)]."""
    by = k - bh - bl
    assert by >= 0
    a = src.reshape(1 << bh, 1 << by, 1 << bl, E)
    out = np.empty_like(a).reshape(1 << bl, 1 << by, 1 << bh, E)
    rx = np.array([brute_rev(v, bh) for v in range(1 << bh)], dtype=np.int64)
    rz = np.array([brute_rev(v, bl) for v in range(1 << bl)], dtype=np.int64)
    for y in range(1 << by):
        buff = np.empty((1 << bh, 1 << bl, E), dtype=src.dtype)
        buff[rx] = a[:, y]               # buff[rev(x)][z] <- source[x y z]
        ry = brute_rev(y, by)
        out[rz, ry] = buff.transpose(1, 0, 2)   # dest[rev(z) rev(y) .] <- buff[. z]
    return out.reshape(-1)


def check_cobra_schedule(impl, kmax: int = 12) -> None:
    """P11 -- the tile schedule (any bh + bl <= k) reproduces the oracle.
    This pins the tiling arithmetic used by the GPU kernels (on the CPU),
    not the oracle."""
    for k in range(0, kmax + 1):
        for bh in range(0, k + 1):
            for bl in range(0, k - bh + 1):
                if (bh + bl) > 8:
                    continue
                E = (1, 4, 8, 16)[(k + bh + bl) % 4]
                x = fingerprint_elems(1 << k, E, salt=k + 7 * bh + 13 * bl)
                got = cobra_emulate(x, k, E, bh, bl)
                assert np.array_equal(got, impl.oop(x, k, E)), (k, bh, bl, E)


ALL_IMPL_CHECKS = [
    check_worked_example,
    check_brute_force,
    check_involution,
    check_stockham,
    check_xor_induction,
    check_counts,
    check_classes,
    check_concatenation,
    check_odd_k,
    check_recursive_square,
]
