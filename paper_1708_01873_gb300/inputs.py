"""Seeded synthetic inputs for the bit-reversed permutation.

This module holds no part of the permutation itself: it only draws the array
contents that both the GPU library's tests/bench and the CPU oracle consume.
It imports neither the oracle nor the CUDA library.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter mode.  Draw number c of the
stream seeded with ``seed`` is

    z = seed + (c + 1) * 0x9E3779B97F4A7C15            (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9           (mod 2^64)
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB           (mod 2^64)
    draw = z ^ (z >> 31)

i.e. exactly the c-th output of a sequential SplitMix64 seeded with
``seed``.  Because every element depends only on (seed, its index), any
element can be regenerated on its own, which the full-size tests use to
check sampled outputs without holding the whole input on the host.

Element kinds (the dtypes of the paper's benchmarks and their siblings):

====== ===== =====================================================
kind   bytes value of element i
====== ===== =====================================================
u32    4     low 32 bits of draw(i)                 (U[0, 2^32))
f32    4     (draw(i) >> 40) * 2^-23 - 1            (U[-1, 1), exact)
f64    8     (draw(i) >> 11) * 2^-52 - 1            (U[-1, 1), exact)
c64    8     (f32 of draw(2i), f32 of draw(2i+1))   complex<float>
c128   16    (f64 of draw(2i), f64 of draw(2i+1))   complex<double>
u8     1     low 8 bits of draw(i)
u16    2     low 16 bits of draw(i)
====== ===== =====================================================

The float conversions are exact in both numpy and torch (a 24- or 53-bit
integer scaled by a power of two, minus one), so the host and device
generators give identical bytes.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

KIND_BYTES = {"u8": 1, "u16": 2, "u32": 4, "f32": 4, "f64": 8, "c64": 8,
              "c128": 16}
# default kind for an element size (the dtypes the paper and its
# configurations use: uint32/float32, complex<float>, complex<double>)
DEFAULT_KIND = {1: "u8", 2: "u16", 4: "f32", 8: "c64", 16: "c128"}


def draw_scalar(seed: int, c: int) -> int:
    """Pure-Python SplitMix64 draw (reference for the vectorised versions)."""
    z = (seed + (c + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MUL2) & MASK64
    return z ^ (z >> 31)


def _draws_np(seed: int, counters: np.ndarray) -> np.ndarray:
    c = counters.astype(np.uint64, copy=False)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (c + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MUL2)
    return z ^ (z >> np.uint64(31))


def _f32_of(d: np.ndarray) -> np.ndarray:
    u = (d >> np.uint64(40)).astype(np.float32)
    return u * np.float32(2.0 ** -23) - np.float32(1.0)


def _f64_of(d: np.ndarray) -> np.ndarray:
    u = (d >> np.uint64(11)).astype(np.float64)
    return u * np.float64(2.0 ** -52) - np.float64(1.0)


def elements_np(seed: int, index: np.ndarray, kind: str) -> np.ndarray:
    """Bytes of the elements at positions ``index`` (any int array), shape
    (len(index), elem_bytes), dtype uint8."""
    idx = np.asarray(index, dtype=np.uint64).reshape(-1)
    E = KIND_BYTES[kind]
    if kind in ("u8", "u16", "u32"):
        d = _draws_np(seed, idx)
        t = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32}[kind]
        v = (d & np.uint64((1 << (8 * E)) - 1)).astype(t)
    elif kind == "f32":
        v = _f32_of(_draws_np(seed, idx))
    elif kind == "f64":
        v = _f64_of(_draws_np(seed, idx))
    elif kind == "c64":
        v = np.empty((idx.size, 2), dtype=np.float32)
        v[:, 0] = _f32_of(_draws_np(seed, 2 * idx))
        v[:, 1] = _f32_of(_draws_np(seed, 2 * idx + np.uint64(1)))
    elif kind == "c128":
        v = np.empty((idx.size, 2), dtype=np.float64)
        v[:, 0] = _f64_of(_draws_np(seed, 2 * idx))
        v[:, 1] = _f64_of(_draws_np(seed, 2 * idx + np.uint64(1)))
    else:
        raise ValueError(f"unknown kind {kind!r}")
    return np.ascontiguousarray(v).view(np.uint8).reshape(idx.size, E)


def array_np(seed: int, n: int, kind: str) -> np.ndarray:
    """The whole n-element array as a flat uint8 buffer of n*E bytes."""
    E = KIND_BYTES[kind]
    out = np.empty(n * E, dtype=np.uint8)
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        out[s * E:e * E] = elements_np(seed, np.arange(s, e, dtype=np.uint64),
                                       kind).reshape(-1)
    return out


# ---------------------------------------------------------------- torch --
# The same generator in torch int64 arithmetic, for filling large device
# buffers without a host round trip.  int64 multiplication wraps modulo 2^64
# exactly like uint64, and logical right shifts are formed as arithmetic
# shifts followed by a mask.

def _s64(x: int) -> int:
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _draws_torch(seed: int, c):
    import torch
    z = (c + 1) * _s64(GAMMA) + _s64(seed)
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * _s64(MUL1)
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * _s64(MUL2)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def fill_torch(buf, seed: int, kind: str, first_index: int = 0,
               chunk: int = 1 << 24) -> None:
    """Fill the contiguous tensor ``buf`` (any dtype; its bytes are
    overwritten) with elements ``first_index ..`` of the seeded array."""
    import torch
    E = KIND_BYTES[kind]
    raw = buf.reshape(-1).view(torch.uint8)
    assert raw.numel() % E == 0
    n = raw.numel() // E
    dev = raw.device
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        c = torch.arange(first_index + s, first_index + e, dtype=torch.int64,
                         device=dev)
        dst = raw[s * E:e * E]
        if kind in ("u8", "u16", "u32"):
            d = _draws_torch(seed, c)
            bits = 8 * E
            low = d & ((1 << bits) - 1)
            half = 1 << (bits - 1)
            signed = (low ^ half) - half
            t = {"u8": torch.int8, "u16": torch.int16, "u32": torch.int32}[kind]
            dst.copy_(signed.to(t).view(torch.uint8))
        elif kind == "f32":
            d = _draws_torch(seed, c)
            v = ((d >> 40) & 0xFFFFFF).to(torch.float32) * (2.0 ** -23) - 1.0
            dst.copy_(v.view(torch.uint8))
        elif kind == "f64":
            d = _draws_torch(seed, c)
            v = ((d >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -52) - 1.0
            dst.copy_(v.view(torch.uint8))
        elif kind in ("c64", "c128"):
            ft = torch.float32 if kind == "c64" else torch.float64
            v = torch.empty((e - s, 2), dtype=ft, device=dev)
            for part in (0, 1):
                d = _draws_torch(seed, 2 * c + part)
                if kind == "c64":
                    v[:, part] = ((d >> 40) & 0xFFFFFF).to(ft) * (2.0 ** -23) - 1.0
                else:
                    v[:, part] = (((d >> 11) & ((1 << 53) - 1)).to(ft)
                                  * (2.0 ** -52) - 1.0)
            dst.copy_(v.reshape(-1).view(torch.uint8))
        else:
            raise ValueError(f"unknown kind {kind!r}")
