"""The C ABI without a GPU: the library loads, exports every symbol that
include/brev.h declares, and its host-only logic (argument checks, tile-shape
choice, tuning-cache parsing, status strings) behaves as documented.  No call
here launches or touches device memory."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "brev.h")


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"BREV_API\s+[\w\s\*]*?\b(brev_\w+)\s*\(", text)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("brev_permute", "brev_permute_to", "brev_permute_batched",
                     "brev_permute_batched_mixed", "brev_plan_create", "brev_plan_launch",
                     "brev_plan_destroy", "brev_autotune", "brev_status_string",
                     "brev_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(brev_lib):
    L = ctypes.CDLL(brev_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers the same names
    assert set(declared_functions()) <= set(brev_lib.SIGNATURES)


def test_version_and_status_strings(brev_lib):
    assert brev_lib.brev_version() == 1000
    for s, name in brev_lib.STATUS_NAMES.items():
        assert brev_lib.brev_status_string(s) == name
    assert brev_lib.brev_status_string(42) == "BREV_ERR_UNKNOWN"


def test_argument_checks_before_any_device_call(brev_lib):
    L = brev_lib.lib()
    assert L.brev_permute_to(None, None, 3, 4, None) == 1
    assert "NULL" in brev_lib.brev_last_error()
    assert L.brev_permute_to(64, 64, 3, 3, None) == 1         # elem_bytes
    assert L.brev_permute_to(64, 64, 35, 4, None) == 1        # k
    assert L.brev_permute_to(66, 66, 3, 4, None) == 2         # alignment
    assert L.brev_permute_to(64, 4098, 3, 4, None) == 2       # source misaligned
    assert L.brev_permute_to(1024, 1040, 3, 4, None) == 3     # partial overlap
    assert L.brev_permute_batched(None, None, -1, 4, None) == 1
    assert L.brev_permute_batched(None, None, 0, 4, None) == 0  # empty batch
    assert L.brev_permute_batched_noalloc(None, None, None, 1025, None) == 1
    assert "exceeds" in brev_lib.brev_last_error()
    assert L.brev_permute_shape(64, 64, 10, 8, 4, 5, 0, None) == 1  # in place needs square
    assert L.brev_autotune(5, 3, 8, None) == 1
    assert L.brev_autotune(0, 10, 7, None) == 1
    h = ctypes.c_void_p()
    assert L.brev_plan_create(None, None, None, 8, -1, ctypes.byref(h)) == 1
    assert L.brev_plan_launch(None, None) == 1


def test_tile_shape_choice(brev_lib):
    brev_lib.brev_reset_tuning()
    b_min = {16: 3, 8: 4, 4: 5, 2: 6, 1: 7}
    for E in (16, 8, 4, 2, 1):
        for k in range(0, 35):
            for ip in (False, True):
                bx, bz, order = brev_lib.brev_tile_shape(k, E, ip)
                if k < 2 * b_min[E]:
                    assert (bx, bz, order) == (0, 0, 0)   # whole array in one CTA
                else:
                    assert bx + bz <= k and bx >= b_min[E] and bz >= b_min[E]
                    assert (E << bz) >= 128 and (E << bx) >= 128
                    if ip:
                        assert bx == bz
                    assert (bx, bz, order) in brev_lib.brev_shapes(E, ip)
    # defaults (no tuning): 512-byte rows for 16-byte elements at large k
    assert brev_lib.brev_tile_shape(28, 16, False) == (5, 5, 0)
    # every 16-byte shape is compiled in both launch orders
    for E in (16, 8, 4, 2, 1):
        for ip in (False, True):
            shapes = brev_lib.brev_shapes(E, ip)
            assert {(bx, bz, 1) for bx, bz, o in shapes if o == 0} == \
                {s for s in shapes if s[2] == 1}


def test_tune_cache_round_trip_host_only(brev_lib, tmp_path):
    p = tmp_path / "t.json"
    entries = [
        {"elem_bytes": 8, "log2n": 20, "in_place": 0, "bx": 5, "bz": 6, "order": 1, "gbs": 1.0},
        {"elem_bytes": 8, "log2n": 20, "in_place": 1, "bx": 4, "bz": 4, "gbs": 1.0},
        # invalid entries are ignored: non-square in place, shape not compiled,
        # tile larger than the array
        {"elem_bytes": 8, "log2n": 21, "in_place": 1, "bx": 4, "bz": 5, "gbs": 1.0},
        {"elem_bytes": 8, "log2n": 22, "in_place": 0, "bx": 3, "bz": 3, "gbs": 1.0},
        {"elem_bytes": 16, "log2n": 9, "in_place": 0, "bx": 5, "bz": 5, "gbs": 1.0},
    ]
    p.write_text(json.dumps({"format": "brev-tune-1", "device": "any", "sm_count": 1,
                             "entries": entries}))
    brev_lib.brev_reset_tuning()
    brev_lib.brev_load_tune_cache(str(p))
    assert brev_lib.brev_tile_shape(20, 8, False) == (5, 6, 1)
    assert brev_lib.brev_tile_shape(20, 8, True) == (4, 4, 0)   # no "order" key: plain
    brev_lib.brev_reset_tuning()
    d21 = brev_lib.brev_tile_shape(21, 8, True)
    brev_lib.brev_load_tune_cache(str(p))
    assert brev_lib.brev_tile_shape(21, 8, True) == d21
    assert brev_lib.brev_tile_shape(9, 16, False)[:2] != (5, 5)
    brev_lib.brev_reset_tuning()
    with pytest.raises(brev_lib.BrevError):
        brev_lib.brev_load_tune_cache(str(tmp_path / "missing.json"))


def test_batched_shape_choice(brev_lib):
    """Built-in batched tile exponents: 16 KiB tiles with 256-512-byte rows
    at large k, smaller tiles for short arrays, whole-array staging below
    2 b_min, single-array launches for 1- and 2-byte elements."""
    brev_lib.brev_reset_tuning()
    b_min = {16: 3, 8: 4, 4: 5}
    pref = {16: 5, 8: 5, 4: 6}
    for E in (16, 8, 4):
        for k in range(2, 35):
            b = brev_lib.brev_batched_shape(k, E)
            if k < 2 * b_min[E]:
                assert b == 0
            else:
                assert b == min(pref[E], k // 2) and b >= b_min[E]
    for E, k in ((16, 0), (16, 1), (2, 20), (1, 20)):
        with pytest.raises(brev_lib.BrevError):
            brev_lib.brev_batched_shape(k, E)


def test_batched_tune_cache_round_trip_host_only(brev_lib, tmp_path):
    p = tmp_path / "b.json"
    entries = [
        {"elem_bytes": 16, "log2n": 14, "batched_b": 4, "gbs": 1.0},
        {"elem_bytes": 8, "log2n": 11, "batched_b": 0, "gbs": 1.0},    # 16 KiB staged whole
        # invalid: b too large for k, shape not in the batched kernel, whole
        # array too large to stage
        {"elem_bytes": 16, "log2n": 7, "batched_b": 4, "gbs": 1.0},
        {"elem_bytes": 4, "log2n": 20, "batched_b": 4, "gbs": 1.0},
        {"elem_bytes": 16, "log2n": 20, "batched_b": 0, "gbs": 1.0},
    ]
    p.write_text(json.dumps({"format": "brev-tune-1", "device": "any", "sm_count": 1,
                             "entries": entries}))
    brev_lib.brev_reset_tuning()
    d = {(k, E): brev_lib.brev_batched_shape(k, E) for k, E in ((7, 16), (20, 4), (20, 16))}
    brev_lib.brev_load_tune_cache(str(p))
    assert brev_lib.brev_batched_shape(14, 16) == 4
    assert brev_lib.brev_batched_shape(11, 8) == 0
    for (k, E), b in d.items():
        assert brev_lib.brev_batched_shape(k, E) == b
    brev_lib.brev_reset_tuning()
    assert brev_lib.brev_batched_shape(14, 16) == 5


def test_shipped_tune_cache_is_valid(brev_lib):
    d = json.load(open(brev_lib.DEFAULT_TUNE_CACHE))
    assert d["format"] == "brev-tune-1" and d["sm_count"] > 0
    for e in d["entries"]:
        if "batched_b" in e:
            b = e["batched_b"]
            assert b == 0 or (2 * b <= e["log2n"] and e["elem_bytes"] in (4, 8, 16))
            continue
        assert (e["bx"], e["bz"], e.get("order", 0)) in \
            brev_lib.brev_shapes(e["elem_bytes"], bool(e["in_place"]))
        assert e["bx"] + e["bz"] <= e["log2n"]


def test_concurrent_builds_compile_once(monkeypatch, tmp_path):
    """Ranks started together all call the build.  The build takes a file
    lock and re-checks staleness under it, so one caller compiles and the
    others find the library up to date; no two compilations overlap.  The
    compiler is replaced by a recorder here, so nothing is compiled."""
    import threading
    import time

    from paper_1708_01873_gb300 import build as B

    monkeypatch.setattr(B, "BUILD", str(tmp_path))
    state = {"built": False, "active": 0, "max_active": 0, "compiles": 0}
    guard = threading.Lock()

    def fake_compile(verbose):
        with guard:
            state["active"] += 1
            state["compiles"] += 1
            state["max_active"] = max(state["max_active"], state["active"])
        time.sleep(0.2)
        with guard:
            state["active"] -= 1
            state["built"] = True
        return B.LIB

    monkeypatch.setattr(B, "is_stale", lambda: not state["built"])
    monkeypatch.setattr(B, "_compile_and_link", fake_compile)
    threads = [threading.Thread(target=B.build_library) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert state["compiles"] == 1 and state["max_active"] == 1
