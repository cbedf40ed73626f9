"""Python binding of the C ABI in ``include/brev.h`` (ctypes).

Argument marshalling only: every permutation runs in the CUDA kernels of
``libbrev.so``.  Functions carry the C names; they take torch tensors (any
dtype -- the element size is ``tensor.element_size()``; elements are moved
as opaque bytes), infer log2n from the element count, pass the current
torch CUDA stream unless one is given, and raise :class:`BrevError` when the
library returns a non-OK status.  There is no CPU fallback: if the library
is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbrev.so")

BREV_OK = 0
STATUS_NAMES = {0: "BREV_OK", 1: "BREV_ERR_INVALID_ARG", 2: "BREV_ERR_ALIGNMENT",
                3: "BREV_ERR_OVERLAP", 4: "BREV_ERR_OOM", 5: "BREV_ERR_CUDA",
                6: "BREV_ERR_UNSUPPORTED"}

# symbol name -> (restype, argtypes)
_vp, _i, _u64, _cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_char_p
_ip = ctypes.POINTER(ctypes.c_int)
_vpp = ctypes.POINTER(ctypes.c_void_p)


class DeviceInfo(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("l2_bytes", ctypes.c_int),
                ("mem_clock_khz", ctypes.c_int), ("mem_bus_bits", ctypes.c_int),
                ("nominal_gbs", ctypes.c_double), ("max_smem_per_block", ctypes.c_int),
                ("name", ctypes.c_char * 96)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("n_streams", ctypes.c_int), ("resident", ctypes.c_int),
                ("idle_stop_ms", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("offered", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("queue_p99_us", ctypes.c_double), ("req_per_s", ctypes.c_double),
                ("gbs", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("peak_pool_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int),
                ("device_p50_us", ctypes.c_double), ("device_p99_us", ctypes.c_double)]


class ServerRequest(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_uint64), ("log2n", ctypes.c_int),
                ("elem_bytes", ctypes.c_int), ("batch", ctypes.c_int),
                ("arrival_us", ctypes.c_double), ("launch_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("seen_us", ctypes.c_double)]


SIGNATURES = {
    "brev_permute_to": (_i, [_vp, _vp, _i, _i, _vp]),
    "brev_permute": (_i, [_vp, _i, _i, _i, _vp]),
    "brev_permute_batched": (_i, [_vpp, _ip, _i, _i, _vp]),
    "brev_permute_batched_mixed": (_i, [_vpp, _ip, _ip, _i, _vp]),
    "brev_permute_batched_noalloc": (_i, [_vpp, _ip, _ip, _i, _vp]),
    "brev_plan_create": (_i, [_vpp, _ip, _ip, _i, _i, ctypes.POINTER(_vp)]),
    "brev_plan_launch": (_i, [_vp, _vp]),
    "brev_plan_destroy": (None, [_vp]),
    "brev_permute_host": (_i, [_vp, _vp, _i, _i, _vp]),
    "brev_transpose": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "brev_dist_plan": (_i, [_i, _i, _i, _i, ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                            ctypes.POINTER(_u64)]),
    "brev_dist_pack": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "brev_dist_finish": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "brev_shard_batch": (_i, [_ip, _ip, _i, _i, _ip]),
    "brev_even_odd": (_i, [_vp, _vp, _i, _i, _vp]),
    "brev_perfect_shuffle": (_i, [_vp, _vp, _i, _i, _vp]),
    "brev_permute_segments": (_i, [_vp, _i, _i, _i, _vp]),
    "brev_permute_recursive": (_i, [_vp, _i, _i, _vp]),
    "brev_fft_stages": (_i, [_vp, _vp, _i, _i, _i, _i, _vp]),
    "brev_server_create": (_i, [ctypes.POINTER(ServerConfig), _vp, _u64, ctypes.POINTER(_vp)]),
    "brev_server_destroy": (None, [_vp]),
    "brev_server_run_poisson": (_i, [_vp, _u64, ctypes.c_double, ctypes.c_double, _i, _i, _ip, _i,
                                     _i, ctypes.POINTER(ServerRequest), _u64,
                                     ctypes.POINTER(ServerStats)]),
    "brev_tile_shape": (_i, [_i, _i, _i, _ip, _ip, _ip]),
    "brev_batched_shape": (_i, [_i, _i, _ip]),
    "brev_permute_shape": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "brev_shape_count": (_i, [_i, _i]),
    "brev_shape_at": (_i, [_i, _i, _i, _ip, _ip, _ip]),
    "brev_autotune": (_i, [_i, _i, _i, _cp]),
    "brev_load_tune_cache": (_i, [_cp]),
    "brev_reset_tuning": (None, []),
    "brev_get_device_info": (_i, [ctypes.POINTER(DeviceInfo)]),
    "brev_fp64_fma_tflops": (_i, [ctypes.POINTER(ctypes.c_double)]),
    "brev_host_link_gbs": (_i, [_vp, _vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "brev_launch_count": (_u64, []),
    "brev_workspace_bytes": (_i, [ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "brev_wait_timeouts": (_i, [ctypes.POINTER(_u64)]),
    "brev_status_string": (_cp, [_i]),
    "brev_last_error": (_cp, []),
    "brev_version": (_i, []),
}

_lock = threading.Lock()
_lib = None


class BrevError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{func}: {self.status_name}: {message}")


def lib() -> ctypes.CDLL:
    """Load libbrev.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with "
                    "paper_1708_01873_gb300.build.build_library() (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
            _load_default_tuning(L)
    return _lib


DEFAULT_TUNE_CACHE = os.path.join(_HERE, "tune_gb300.json")


def _load_default_tuning(L) -> None:
    """Tuned tile shapes: $BREV_TUNE_CACHE if set, else the cache shipped
    with the package (ignored by the library unless the device name and SM
    count match the GPU it was tuned on)."""
    path = os.environ.get("BREV_TUNE_CACHE", DEFAULT_TUNE_CACHE)
    if path and os.path.exists(path):
        L.brev_load_tune_cache(path.encode())


def _check(status: int, func: str) -> None:
    if status != BREV_OK:
        msg = lib().brev_last_error().decode(errors="replace")
        raise BrevError(status, func, msg)


def _log2(n: int) -> int:
    if n <= 0 or n & (n - 1):
        raise ValueError(f"element count {n} is not a power of two")
    return n.bit_length() - 1


def _stream_handle(stream, device=None) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _flat(t):
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t


# ------------------------------------------------------------ single --
def brev_permute_to(dst, src, stream=None) -> None:
    """dst[rev(i)] = src[i] (src may be dst: in place)."""
    _flat(dst), _flat(src)
    if dst.element_size() != src.element_size() or dst.numel() != src.numel():
        raise ValueError("dst and src must have the same element size and count")
    k = _log2(src.numel())
    _check(lib().brev_permute_to(dst.data_ptr(), src.data_ptr(), k, src.element_size(),
                                 _stream_handle(stream, src.device)), "brev_permute_to")


def brev_permute(data, in_place: bool = True, stream=None) -> None:
    """in_place: permute ``data`` (2^k elements).  Otherwise ``data`` holds
    [src | dst] (2 * 2^k elements) and the result goes to its second half."""
    _flat(data)
    n = data.numel() if in_place else data.numel() // 2
    if not in_place and data.numel() % 2:
        raise ValueError("[src | dst] buffer needs an even element count")
    k = _log2(n)
    _check(lib().brev_permute(data.data_ptr(), k, data.element_size(), int(bool(in_place)),
                              _stream_handle(stream, data.device)), "brev_permute")


def brev_permute_shape(dst, src, bx: int, bz: int, order: int = 0, stream=None) -> None:
    """Forced tile shape (2^bx x 2^bz; 0, 0 = whole array in one CTA) and
    launch order (0 plain, 1 blocked)."""
    _flat(dst), _flat(src)
    k = _log2(src.numel())
    _check(lib().brev_permute_shape(dst.data_ptr(), src.data_ptr(), k, src.element_size(),
                                    bx, bz, order, _stream_handle(stream, src.device)),
           "brev_permute_shape")


# ----------------------------------------------------------- batched --
def _batch_arrays(tensors: Sequence):
    n = len(tensors)
    ptrs = (ctypes.c_void_p * max(n, 1))()
    ks = (ctypes.c_int * max(n, 1))()
    es = (ctypes.c_int * max(n, 1))()
    for i, t in enumerate(tensors):
        _flat(t)
        ptrs[i] = t.data_ptr()
        ks[i] = _log2(t.numel())
        es[i] = t.element_size()
    return ptrs, ks, es


def brev_permute_batched(tensors: Sequence, stream=None) -> None:
    """Permute every tensor in place in one persistent launch (tensors may
    have different element sizes and lengths)."""
    tensors = list(tensors)
    if not tensors:
        return
    ptrs, ks, es = _batch_arrays(tensors)
    _check(lib().brev_permute_batched_mixed(ptrs, ks, es, len(tensors),
                                            _stream_handle(stream, tensors[0].device)),
           "brev_permute_batched_mixed")


brev_permute_batched_mixed = brev_permute_batched


def brev_permute_batched_noalloc(tensors: Sequence, stream=None) -> None:
    """The batched in-place permutation for callers that cannot allocate
    device memory: its scratch is a fixed array inside the library (at most
    BREV_NOALLOC_MAX_ARRAYS = 1024 arrays per call; calls that overlap on the
    GPU race).  Make the first call on a device before any stream capture."""
    tensors = list(tensors)
    if not tensors:
        return
    ptrs, ks, es = _batch_arrays(tensors)
    _check(lib().brev_permute_batched_noalloc(ptrs, ks, es, len(tensors),
                                              _stream_handle(stream, tensors[0].device)),
           "brev_permute_batched_noalloc")


class BrevPlan:
    """A captured batch (brev_plan_create); ``launch`` replays it."""

    def __init__(self, tensors: Iterable):
        self.tensors = list(tensors)  # keeps the storage alive
        ptrs, ks, es = _batch_arrays(self.tensors)
        h = ctypes.c_void_p()
        _check(lib().brev_plan_create(ptrs, ks, es, 0, len(self.tensors), ctypes.byref(h)),
               "brev_plan_create")
        self._h = h

    def launch(self, stream=None) -> None:
        dev = self.tensors[0].device if self.tensors else None
        _check(lib().brev_plan_launch(self._h, _stream_handle(stream, dev)), "brev_plan_launch")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            lib().brev_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def brev_plan_create(tensors: Iterable) -> BrevPlan:
    return BrevPlan(tensors)


# ---------------------------------------------------- transpositions --
def brev_transpose(dst, src, log2_rows: int, log2_cols: int, stream=None) -> None:
    """dst (2^cols x 2^rows) = transpose of src (2^rows x 2^cols), both
    flat and row-major; dst may be src for square matrices."""
    _flat(dst), _flat(src)
    if src.numel() != 1 << (log2_rows + log2_cols) or dst.numel() != src.numel():
        raise ValueError("tensor sizes do not match the matrix shape")
    _check(lib().brev_transpose(dst.data_ptr(), src.data_ptr(), log2_rows, log2_cols,
                                src.element_size(), _stream_handle(stream, src.device)),
           "brev_transpose")


# ------------------------------------------------- one array, G ranks --
def brev_dist_plan(log2n: int, log2_ranks: int, elem_bytes: int, rank: int):
    """(send_offsets, recv_offsets, segment_elems) of the exchange on rank
    `rank` (offsets in elements, one per peer); host-only."""
    G = 1 << log2_ranks
    so, ro, seg = (ctypes.c_uint64 * G)(), (ctypes.c_uint64 * G)(), ctypes.c_uint64()
    _check(lib().brev_dist_plan(log2n, log2_ranks, elem_bytes, rank, so, ro, ctypes.byref(seg)),
           "brev_dist_plan")
    return list(so), list(ro), seg.value


def brev_dist_pack(send, block, log2n: int, log2_ranks: int, stream=None) -> None:
    """Step 1 of the permutation over 2^log2_ranks ranks (send may be block)."""
    _flat(send), _flat(block)
    _check(lib().brev_dist_pack(send.data_ptr(), block.data_ptr(), log2n, log2_ranks,
                                block.element_size(), _stream_handle(stream, block.device)),
           "brev_dist_pack")


def brev_dist_finish(block, recv, log2n: int, log2_ranks: int, stream=None) -> None:
    """Step 3 of the permutation over 2^log2_ranks ranks."""
    _flat(block), _flat(recv)
    _check(lib().brev_dist_finish(block.data_ptr(), recv.data_ptr(), log2n, log2_ranks,
                                  block.element_size(), _stream_handle(stream, block.device)),
           "brev_dist_finish")


def dist_steps(block, recv, log2n: int, log2_ranks: int, rank: int, pack, exchange, finish):
    """The three steps on one rank, with the local passes and the exchange
    passed in: pack(block) permutes the block in place into send order,
    exchange(recv, send, seg_elems) moves segment q of every rank's send
    buffer to segment p = sender of rank q's receive buffer (equal
    segments, offsets from brev_dist_plan), finish(block, recv) writes the
    result.  brev_permute_distributed passes the library's kernels and
    torch.distributed's all-to-all."""
    E = block.element_size()
    so, ro, seg = brev_dist_plan(log2n, log2_ranks, E, rank)
    G = 1 << log2_ranks
    if so != [q * seg for q in range(G)] or ro != so:
        raise RuntimeError("exchange plan is not one of equal consecutive segments")
    pack(block)
    exchange(recv, block, seg)
    finish(block, recv)


def brev_permute_distributed(block, recv=None, group=None, stream=None) -> None:
    """Permute one array spread over the ranks of `group` (a power of two of
    them, one GPU each), rank p holding the p-th consecutive block: on
    return every rank's block holds its part of the permuted array.  recv
    is a scratch tensor like block (allocated when None).  The exchange is
    torch.distributed's all-to-all (NCCL on GPUs)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    g = _log2(world)
    rank = dist.get_rank(group)
    log2n = _log2(block.numel()) + g
    if recv is None:
        recv = torch.empty_like(block)

    def exchange(r, s, seg):
        dist.all_to_all_single(r.view(torch.uint8), s.view(torch.uint8), group=group)

    dist_steps(block, recv, log2n, g, rank,
               pack=lambda b: brev_dist_pack(b, b, log2n, g, stream),
               exchange=exchange,
               finish=lambda b, r: brev_dist_finish(b, r, log2n, g, stream))


def brev_shard_batch(log2n: Sequence[int], elem_bytes: Sequence[int], world: int) -> list[int]:
    """Owner rank of each array of a batch split across `world` ranks by
    array (largest first, to the least-loaded rank); host-only."""
    n = len(log2n)
    ks = (ctypes.c_int * n)(*log2n)
    es = (ctypes.c_int * n)(*elem_bytes)
    own = (ctypes.c_int * n)()
    _check(lib().brev_shard_batch(ks, es, n, world, own), "brev_shard_batch")
    return list(own)


def brev_even_odd(dst, src, stream=None) -> None:
    """Even-indexed elements, then odd-indexed ones (the Stockham step)."""
    _flat(dst), _flat(src)
    _check(lib().brev_even_odd(dst.data_ptr(), src.data_ptr(), _log2(src.numel()),
                               src.element_size(), _stream_handle(stream, src.device)),
           "brev_even_odd")


def brev_perfect_shuffle(dst, src, stream=None) -> None:
    """The two halves interleaved (inverse of brev_even_odd)."""
    _flat(dst), _flat(src)
    _check(lib().brev_perfect_shuffle(dst.data_ptr(), src.data_ptr(), _log2(src.numel()),
                                      src.element_size(), _stream_handle(stream, src.device)),
           "brev_perfect_shuffle")


def brev_permute_segments(data, log2_segments: int, stream=None) -> None:
    """Bit-reverse each of 2^log2_segments equal contiguous segments in place."""
    _flat(data)
    k = _log2(data.numel())
    if log2_segments > k:
        raise ValueError("more segments than elements")
    _check(lib().brev_permute_segments(data.data_ptr(), log2_segments, k - log2_segments,
                                       data.element_size(),
                                       _stream_handle(stream, data.device)),
           "brev_permute_segments")


def brev_permute_recursive(data, stream=None) -> None:
    """In-place permutation by the paper's recursive method (multi-pass)."""
    _flat(data)
    _check(lib().brev_permute_recursive(data.data_ptr(), _log2(data.numel()),
                                        data.element_size(), _stream_handle(stream, data.device)),
           "brev_permute_recursive")


def brev_fft_stages(dst, src, stages: int, inverse: bool = False, stream=None) -> None:
    """dst = first `stages` radix-2 DIT FFT stages of the bit-reversed src
    (complex64 or complex128 tensors; dst may be src)."""
    _flat(dst), _flat(src)
    if dst.numel() != src.numel() or dst.element_size() != src.element_size():
        raise ValueError("dst and src must match")
    _check(lib().brev_fft_stages(dst.data_ptr(), src.data_ptr(), _log2(src.numel()),
                                 src.element_size(), stages, int(bool(inverse)),
                                 _stream_handle(stream, src.device)), "brev_fft_stages")


# ----------------------------------------------------------- serving --
def brev_server_run_poisson(arena, seed: int, rate_per_s: float, seconds: float,
                            k_range=(10, 24), elem_sizes=(4, 8, 16), max_slots: int = 256,
                            max_batch: int = 256, n_streams: int = 4,
                            hold_results: bool = False, trace: bool = False,
                            resident: bool = False, idle_stop_ms: int = 0):
    """Run the native serving loop over the device tensor ``arena`` for a
    seeded Poisson stream; returns (stats dict, trace list or None).
    resident: one kernel fed through page-locked host memory instead of a
    launch per batch."""
    cfg = ServerConfig(max_slots, max_batch, n_streams, int(bool(resident)), idle_stop_ms)
    h = ctypes.c_void_p()
    _check(lib().brev_server_create(ctypes.byref(cfg), arena.data_ptr(),
                                    arena.numel() * arena.element_size(), ctypes.byref(h)),
           "brev_server_create")
    try:
        es = (ctypes.c_int * len(elem_sizes))(*elem_sizes)
        cap = int(rate_per_s * seconds * 1.2 + 1000) if trace else 0
        tr = (ServerRequest * cap)() if trace else None
        st = ServerStats()
        _check(lib().brev_server_run_poisson(h, seed, rate_per_s, seconds, k_range[0],
                                             k_range[1], es, len(elem_sizes),
                                             int(bool(hold_results)), tr, cap,
                                             ctypes.byref(st)), "brev_server_run_poisson")
    finally:
        lib().brev_server_destroy(h)
    stats = {f: getattr(st, f) for f, _ in ServerStats._fields_}
    recs = None
    if trace:
        recs = [{"offset": r.offset, "log2n": r.log2n, "elem_bytes": r.elem_bytes,
                 "batch": r.batch, "arrival_us": r.arrival_us, "launch_us": r.launch_us,
                 "done_us": r.done_us, "seen_us": r.seen_us}
                for r in tr[:st.offered]]
    return stats, recs


# -------------------------------------------------------------- host --
def brev_permute_host(dst, src, stream=None) -> None:
    """Host (CPU, ideally pinned) tensors: copy in, permute on the GPU, copy
    out; returns when the result is in ``dst``."""
    _flat(dst), _flat(src)
    k = _log2(src.numel())
    import torch
    s = _stream_handle(stream, torch.device("cuda", torch.cuda.current_device()))
    _check(lib().brev_permute_host(dst.data_ptr(), src.data_ptr(), k, src.element_size(), s),
           "brev_permute_host")


# ------------------------------------------------------------ tuning --
def brev_tile_shape(log2n: int, elem_bytes: int, in_place: bool) -> tuple[int, int, int]:
    """(bx, bz, order) the library uses; (0, 0, 0) = whole array in one CTA."""
    bx, bz, order = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().brev_tile_shape(log2n, elem_bytes, int(bool(in_place)), ctypes.byref(bx),
                                 ctypes.byref(bz), ctypes.byref(order)), "brev_tile_shape")
    return bx.value, bz.value, order.value


def brev_batched_shape(log2n: int, elem_bytes: int) -> int:
    """Tile exponent b the batched kernel uses for such an array (0 = the
    whole array staged as one unit); BrevError if it runs as a single-array
    launch inside a batch."""
    b = ctypes.c_int()
    _check(lib().brev_batched_shape(log2n, elem_bytes, ctypes.byref(b)), "brev_batched_shape")
    return b.value


def brev_shapes(elem_bytes: int, in_place: bool) -> list[tuple[int, int, int]]:
    """Compiled 16-byte-path (bx, bz, order) triples."""
    out = []
    for i in range(lib().brev_shape_count(elem_bytes, int(bool(in_place)))):
        bx, bz, order = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().brev_shape_at(elem_bytes, int(bool(in_place)), i, ctypes.byref(bx),
                                   ctypes.byref(bz), ctypes.byref(order)), "brev_shape_at")
        out.append((bx.value, bz.value, order.value))
    return out


def brev_autotune(k_min: int, k_max: int, elem_bytes: int, cache_path: str | None) -> None:
    p = cache_path.encode() if cache_path else None
    _check(lib().brev_autotune(k_min, k_max, elem_bytes, p), "brev_autotune")


def brev_load_tune_cache(path: str) -> None:
    _check(lib().brev_load_tune_cache(path.encode()), "brev_load_tune_cache")


def brev_reset_tuning() -> None:
    lib().brev_reset_tuning()


def brev_get_device_info() -> dict:
    info = DeviceInfo()
    _check(lib().brev_get_device_info(ctypes.byref(info)), "brev_get_device_info")
    return {"name": info.name.decode(), "sm_count": info.sm_count, "l2_bytes": info.l2_bytes,
            "mem_clock_khz": info.mem_clock_khz, "mem_bus_bits": info.mem_bus_bits,
            "nominal_gbs": info.nominal_gbs, "max_smem_per_block": info.max_smem_per_block}


def brev_fp64_fma_tflops() -> float:
    """Measured FP64 fused multiply-add rate of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(lib().brev_fp64_fma_tflops(ctypes.byref(v)), "brev_fp64_fma_tflops")
    return v.value


def brev_host_link_gbs(dst_host, src_host) -> float:
    """Measured rate (GB/s, read + write) of an SM-driven copy between two
    page-locked host tensors of the same size: the host path's ceiling."""
    v = ctypes.c_double()
    nbytes = src_host.numel() * src_host.element_size()
    if dst_host.numel() * dst_host.element_size() != nbytes:
        raise ValueError("host tensors differ in size")
    _check(lib().brev_host_link_gbs(dst_host.data_ptr(), src_host.data_ptr(), nbytes,
                                    ctypes.byref(v)), "brev_host_link_gbs")
    return v.value


def brev_launch_count() -> int:
    return int(lib().brev_launch_count())


def brev_workspace_bytes() -> tuple[int, int]:
    """(reserved, used) bytes of the library's workspace pool on the
    current device."""
    r, u = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().brev_workspace_bytes(ctypes.byref(r), ctypes.byref(u)), "brev_workspace_bytes")
    return r.value, u.value


def brev_wait_timeouts() -> int:
    """Bounded waits of the batched kernel that gave up on the current
    device (0 on a healthy device; synchronises the device)."""
    v = _u64(0)
    _check(lib().brev_wait_timeouts(ctypes.byref(v)), "brev_wait_timeouts")
    return int(v.value)


def brev_status_string(status: int) -> str:
    return lib().brev_status_string(status).decode()


def brev_last_error() -> str:
    return lib().brev_last_error().decode(errors="replace")


def brev_version() -> int:
    return int(lib().brev_version())
