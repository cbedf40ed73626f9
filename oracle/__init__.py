"""CPU oracle for the bit-reversed permutation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The GPU library and its Python
binding never import it; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C): the definition of the
permutation from the paper's Introduction (element i moves to rev_k(i); the
n = 8 worked example), in place applied to a copy of the input.  This module
only compiles that file with gcc and marshals numpy buffers into it.

Pins that tie the oracle to the paper (worked example, brute force, the
involution, the recursive even-odd definition, the XOR induction, the swap
counts, ...) live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no -march flags so the
    same command works on x86-64 and aarch64 hosts)."""
    stale = (not os.path.exists(LIB_PATH)) or any(
        os.path.getmtime(p) > os.path.getmtime(LIB_PATH) for p in (_SRC, _HDR))
    if force or stale:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-fPIC",
               "-shared", "-pthread", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            u64, i32, i64, vp = (ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                 ctypes.c_void_p)
            L.oracle_rev_bits.argtypes = [u64, i32]
            L.oracle_rev_bits.restype = u64
            L.oracle_brev_oop.argtypes = [vp, vp, i32, i32]
            L.oracle_brev_oop.restype = i32
            L.oracle_brev_inplace.argtypes = [vp, i32, i32]
            L.oracle_brev_inplace.restype = i32
            L.oracle_brev_oop_mt.argtypes = [vp, vp, i32, i32, i32]
            L.oracle_brev_oop_mt.restype = i32
            L.oracle_brev_gather.argtypes = [vp, vp, vp, i64, i32, i32]
            L.oracle_brev_gather.restype = i32
            L.oracle_transpose.argtypes = [vp, vp, i32, i32, i32]
            L.oracle_transpose.restype = i32
            L.oracle_even_odd.argtypes = [vp, vp, i32, i32]
            L.oracle_even_odd.restype = i32
            L.oracle_perfect_shuffle.argtypes = [vp, vp, i32, i32]
            L.oracle_perfect_shuffle.restype = i32
            L.oracle_fft_dit_stages.argtypes = [vp, vp, i32, i32, i32]
            L.oracle_fft_dit_stages.restype = i32
            _lib = L
    return _lib


def _as_bytes(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a.view(np.uint8).reshape(-1)


def rev_bits(i: int, k: int) -> int:
    return int(lib().oracle_rev_bits(int(i), int(k)))


def brev_oop(src: np.ndarray, k: int, elem_bytes: int) -> np.ndarray:
    """Return a new uint8 array: the permutation of ``src`` (2^k elements of
    ``elem_bytes`` bytes each, given as any contiguous array)."""
    s = _as_bytes(src)
    assert s.size == (1 << k) * elem_bytes, (s.size, k, elem_bytes)
    d = np.empty_like(s)
    rc = lib().oracle_brev_oop(d.ctypes.data, s.ctypes.data, k, elem_bytes)
    if rc != 0:
        raise ValueError("oracle_brev_oop rejected its arguments")
    return d


def brev_inplace(v: np.ndarray, k: int, elem_bytes: int) -> np.ndarray:
    """Permute ``v`` in place (it must be a writable contiguous array) and
    return it."""
    assert v.flags["C_CONTIGUOUS"] and v.flags["WRITEABLE"]
    assert v.nbytes == (1 << k) * elem_bytes, (v.nbytes, k, elem_bytes)
    rc = lib().oracle_brev_inplace(v.ctypes.data, k, elem_bytes)
    if rc != 0:
        raise ValueError("oracle_brev_inplace rejected its arguments")
    return v


def brev_oop_mt(src: np.ndarray, k: int, elem_bytes: int, threads: int,
                out: np.ndarray | None = None) -> tuple[np.ndarray, int]:
    s = _as_bytes(src)
    assert s.size == (1 << k) * elem_bytes
    d = np.empty_like(s) if out is None else _as_bytes(out)
    used = lib().oracle_brev_oop_mt(d.ctypes.data, s.ctypes.data, k, elem_bytes,
                                    int(threads))
    if used < 1:
        raise ValueError("oracle_brev_oop_mt rejected its arguments")
    return d, int(used)


def brev_gather(src: np.ndarray, idx: np.ndarray, k: int,
                elem_bytes: int) -> np.ndarray:
    """Expected output bytes at output positions ``idx`` (uint64)."""
    s = _as_bytes(src)
    ix = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(ix.size * elem_bytes, dtype=np.uint8)
    rc = lib().oracle_brev_gather(out.ctypes.data, s.ctypes.data, ix.ctypes.data,
                                  ix.size, k, elem_bytes)
    if rc != 0:
        raise ValueError("oracle_brev_gather rejected its arguments")
    return out


def transpose(src: np.ndarray, log2_rows: int, log2_cols: int, elem_bytes: int) -> np.ndarray:
    """dst[j * 2^a + i] = src[i * 2^c + j] for a 2^a x 2^c matrix."""
    s = _as_bytes(src)
    assert s.size == (1 << (log2_rows + log2_cols)) * elem_bytes
    d = np.empty_like(s)
    if lib().oracle_transpose(d.ctypes.data, s.ctypes.data, log2_rows, log2_cols,
                              elem_bytes) != 0:
        raise ValueError("oracle_transpose rejected its arguments")
    return d


def even_odd(src: np.ndarray, k: int, elem_bytes: int) -> np.ndarray:
    s = _as_bytes(src)
    assert s.size == (1 << k) * elem_bytes
    d = np.empty_like(s)
    if lib().oracle_even_odd(d.ctypes.data, s.ctypes.data, k, elem_bytes) != 0:
        raise ValueError("oracle_even_odd rejected its arguments")
    return d


def perfect_shuffle(src: np.ndarray, k: int, elem_bytes: int) -> np.ndarray:
    s = _as_bytes(src)
    assert s.size == (1 << k) * elem_bytes
    d = np.empty_like(s)
    if lib().oracle_perfect_shuffle(d.ctypes.data, s.ctypes.data, k, elem_bytes) != 0:
        raise ValueError("oracle_perfect_shuffle rejected its arguments")
    return d


def fft_dit_stages(x: np.ndarray, k: int, stages: int, inverse: bool = False) -> np.ndarray:
    """First `stages` radix-2 DIT stages of the bit-reversed ``x`` (complex,
    2^k values); computed in double, returned as complex128."""
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(-1))
    assert z.size == 1 << k
    out = np.empty_like(z)
    if lib().oracle_fft_dit_stages(out.ctypes.data, z.ctypes.data, k, stages,
                                   int(bool(inverse))) != 0:
        raise ValueError("oracle_fft_dit_stages rejected its arguments")
    return out
