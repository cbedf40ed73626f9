"""Autotune the tile shapes on the current GPU and write the JSON cache.

    python -m paper_1708_01873_gb300.tune --out paper_1708_01873_gb300/tune_gb300.json

For every element size and k, brev_autotune times each compiled 16-byte
tile shape out-of-place and in-place (L2 flushed between repetitions,
median of several runs) and keeps the fastest; for 4-, 8- and 16-byte
elements it also times the batched kernel's tile exponent b per k on a
batch of equal arrays.  The library loads the
cache at import when the device name and SM count match (or the file named
by BREV_TUNE_CACHE).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "tune_gb300.json"))
    ap.add_argument("--kmin", type=int, default=6)
    ap.add_argument("--kmax", type=int, default=30)
    ap.add_argument("--elem", type=int, nargs="*", default=[16, 8, 4, 2, 1])
    a = ap.parse_args(argv)
    from paper_1708_01873_gb300 import brev
    brev.lib()
    brev.brev_reset_tuning()  # time every shape, not the previous cache's choice
    for E in a.elem:
        brev.brev_autotune(a.kmin, a.kmax, E, a.out)
        print(f"tuned E={E}", flush=True)
    with open(a.out) as f:
        d = json.load(f)
    print(json.dumps({"device": d["device"], "entries": len(d["entries"])}))


if __name__ == "__main__":
    main()
