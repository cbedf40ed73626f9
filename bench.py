#!/usr/bin/env python3
"""Benchmark of the GB300 bit-reversed permutation library.

Default workload (one "step"): the single-array sweep
k = 10..28 x {uint32, float32, complex<float>, complex<double>} x
{out-of-place, in-place} -- 152 permutations of seeded synthetic arrays
held in 34 GiB, 64 GiB moved per step.  ``value`` is bit-reverse GB/s counting read + write
(2 n E bytes per permutation) over the whole step.  The same JSON line also
carries the batched workload (4096 arrays, k in [8, 20], mixed
complex<float>/complex<double>: one captured-graph persistent launch vs a
loop of per-array launches), the roofline of the dominant kernel, the
end-to-end host-buffer path and the CPU-oracle baseline.

``--impl reference`` times the CPU oracle on the host cores instead (the
paper has no GPU code to run), on a bounded sample of the same sweep.

Multi-GPU (torchrun, one rank per GPU): every rank runs the same workload on
its own GPU (replicas; the permutation of one array needs no exchange at
these sizes), timing takes the max over ranks, value sums all ranks' bytes.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP_KS = list(range(10, 29))
SWEEP_KINDS = [("u32", 4), ("f32", 4), ("c64", 8), ("c128", 16)]
FALLBACK_PEAK_GBS = 6800.0
# what the timed path moves: whole elements of the sweep's kinds, as opaque
# bytes (nothing is computed or narrowed)
DTYPE_LABEL = "opaque 4/8/16-byte elements (exact)"
# FP64 FMA thread-instructions per SM per cycle on GB300 (ncu's issue peak,
# sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 over
# 152 SMs)
FP64_FMA_PER_SM_CLK = 2


# ------------------------------------------------------------- helpers --
def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="brev", choices=["brev", "reference"])
    ap.add_argument("--kmax", type=int, default=28, help="largest k of the sweep")
    ap.add_argument("--kinds", default="u32,f32,c64,c128",
                    help="element kinds of the sweep (comma separated)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="total oracle time budget of --impl reference")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-kmax", type=int, default=20)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-next", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-midsize", action="store_true")
    ap.add_argument("--no-serve-sweep", action="store_true")
    ap.add_argument("--sweep-seconds", type=float, default=2.0,
                    help="seconds of arrivals per point of the serving rate sweep")
    ap.add_argument("--points-out", default=None,
                    help="write per-point median times of the sweep to this JSON file")
    ap.add_argument("--next-k", type=int, default=28,
                    help="array size (log2) of the transposition / FFT-stage measurements")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's time (the whole job ends when it does)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank: float, world: int, seconds_max: float) -> float:
    """Aggregate throughput: every rank's bytes over the slowest rank's time
    (weak scaling: each rank runs the full per-GPU workload)."""
    return world * bytes_per_rank / seconds_max / 1e9


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_PEAK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during timed regions."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []  # (t, sm, max, power, flags)
        self.windows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                self.samples.append((time.time(), float(parts[1]), float(parts[2]),
                                     float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                                     parts[5:9]))
            except ValueError:
                pass

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.proc = None

    # nvidia-smi's polling stalls CUDA calls of the serving loop's host
    # thread (one stall of 50-80 ms per run of a few seconds, measured on
    # GB300), so the latency sections run with the sampler stopped.
    pause = stop
    resume = start

    def summary(self):
        inside = [s for s in self.samples
                  if any(a - 0.05 <= s[0] <= b + 0.05 for a, b in self.windows)]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"],
                    "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i, v in enumerate(s[4])
                          if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(s[1] for s in inside),
                "sm_max_mhz": max(s[2] for s in inside), "reasons": reasons,
                "samples": len(inside), "power_w_max": max(s[3] for s in inside)}


def shape_name(brev, k, E, inplace):
    bx, bz, order = brev.brev_tile_shape(k, E, inplace)
    if bx == 0:
        return f"small_E{E}"
    return (f"tile_{'inplace' if inplace else 'oop'}_E{E}_{bx}x{bz}"
            + ("_blocked" if order == 1 else ""))


# ------------------------------------------------------------ the sweep --
def make_sweep(torch, inputs, kmax, device, kinds=None):
    pts = []
    for kind, E in SWEEP_KINDS:
        if kinds and kind not in kinds:
            continue
        for k in range(SWEEP_KS[0], kmax + 1):
            n = 1 << k
            src = torch.empty(n * E, dtype=torch.uint8, device=device)
            inputs.fill_torch(src, 100 + k, kind)
            dst = torch.empty_like(src)
            pts.append({"kind": kind, "E": E, "k": k, "src": src, "dst": dst,
                        "bytes": 2 * n * E})
    return pts


def sweep_order(pts):
    """All out-of-place launches (ascending k), then all in-place ones: every
    buffer is touched again only after far more than L2 of other traffic."""
    seq = [(p, False) for p in pts] + [(p, True) for p in pts]
    return seq


def sweep_config(kmax, kinds, ws, l2_mib):
    """The sweep's `config`, shared by both arms: every kind's k = 10..kmax,
    out of place then in place, 2 n E bytes per point."""
    sel = [(kind, E) for kind, E in SWEEP_KINDS if kind in kinds.split(",")]
    names = {"u32": "uint32", "f32": "float32", "c64": "complex<float>", "c128": "complex<double>"}
    step_bytes = 2 * sum(2 * (1 << k) * E for _, E in sel for k in range(SWEEP_KS[0], kmax + 1))
    return {"workload": "single-array sweep k=%d..%d x {%s} x {out-of-place, in-place}"
                        % (SWEEP_KS[0], kmax, ", ".join(names[kd] for kd, _ in sel)),
            "points_per_step": 2 * len(sel) * (kmax - SWEEP_KS[0] + 1),
            "bytes_per_step": step_bytes,
            "l2": ("no flush: %.0f GiB moved per step, every buffer re-touched only after "
                   ">= 1 GiB of other traffic (L2 = %s MiB)"
                   % (step_bytes / 2 ** 30, l2_mib if l2_mib is not None else "?"))
                  if kmax >= 26 else
                  "no flush: a reduced sweep of %.1f MiB per step, whose buffers can stay in L2"
                  % (step_bytes / 2 ** 20),
            "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"}


def launch_point(brev, p, inplace, stream):
    if inplace:
        brev.lib().brev_permute_to(p["dst"].data_ptr(), p["dst"].data_ptr(), p["k"], p["E"],
                                   stream)
    else:
        brev.lib().brev_permute_to(p["dst"].data_ptr(), p["src"].data_ptr(), p["k"], p["E"],
                                   stream)


def run_brev(args):
    import torch
    import torch.distributed as dist
    from __graft_entry__ import build
    from paper_1708_01873_gb300 import brev, inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=device)
    build()
    info = brev.brev_get_device_info()
    peak, peak_src = measured_peak()
    # all work on one non-default stream (graph capture needs one)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    def reduce_max(x):
        return max_over_ranks(x, ws, device)

    pts = make_sweep(torch, inputs, args.kmax, device, args.kinds.split(","))
    seq = sweep_order(pts)
    step_bytes = sum(p["bytes"] for p, _ in seq)
    if step_bytes != sweep_config(args.kmax, args.kinds, ws, None)["bytes_per_step"]:
        raise RuntimeError("sweep bytes disagree with the reported config")
    names = [shape_name(brev, p["k"], p["E"], ip) for p, ip in seq]
    L = brev.lib()
    # Warm-up.  Its last steps bracket every launch with CUDA events: the
    # per-kernel shares, the per-point table and the choice of the dominant
    # kernel come from them, so that the timed steps carry events around the
    # dominant kernel's launches only.
    prof_steps = min(args.warmup, 2)
    per_kernel = {}
    per_point = {}
    for w in range(args.warmup):
        prof = w >= args.warmup - prof_steps
        evw = []
        for p, ip in seq:
            if prof:
                ea = torch.cuda.Event(enable_timing=True)
                eb = torch.cuda.Event(enable_timing=True)
                ea.record(stream)
            launch_point(brev, p, ip, sh)
            if prof:
                eb.record(stream)
                evw.append((ea, eb))
        torch.cuda.synchronize(device)
        for i, ((p, ip), (ea, eb)) in enumerate(zip(seq, evw)):
            ms = ea.elapsed_time(eb)
            per_kernel[names[i]] = per_kernel.get(names[i], 0.0) + ms
            key = f"{p['kind']}_{'ip' if ip else 'oop'}_k{p['k']}"
            per_point.setdefault(key, {"ms": [], "bytes": p["bytes"], "k": p["k"], "E": p["E"],
                                       "mode": "ip" if ip else "oop", "kernel": names[i],
                                       "seq": i})
            per_point[key]["ms"].append(ms)
    total_kernel_ms = sum(per_kernel.values())
    # dominant kernel = most device time; its roofline is read at its
    # largest launch configuration (one fixed size per launch)
    dom_name = max(per_kernel, key=per_kernel.get)
    dom_pts = [v for v in per_point.values() if v["kernel"] == dom_name]
    dom = max(dom_pts, key=lambda v: (v["k"], sum(v["ms"])))
    dom_i = dom["seq"]

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)

    # timed steps: events only around the dominant launch configuration
    dom_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    c0 = L.brev_launch_count()
    w0 = time.time()
    t_start.record(stream)
    for s in range(args.steps):
        ea, eb = dom_evs[s]
        for i, (p, ip) in enumerate(seq):
            if i == dom_i:
                ea.record(stream)
                launch_point(brev, p, ip, sh)
                eb.record(stream)
            else:
                launch_point(brev, p, ip, sh)
    t_end.record(stream)
    barrier()
    w1 = time.time()
    sampler.window(w0, w1)
    launches = L.brev_launch_count() - c0
    ms_total = reduce_max(t_start.elapsed_time(t_end))
    ms_per_step = ms_total / args.steps
    value = whole_job_gbs(step_bytes * args.steps, ws, ms_total * 1e-3)
    dom_ms = statistics.mean(ea.elapsed_time(eb) for ea, eb in dom_evs)
    achieved = dom["bytes"] / (dom_ms * 1e-3) / 1e9
    traffic = load_traffic(dom_name, dom["k"], dom["E"], dom["mode"])
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": dom_name,
                "launch": f"k={dom['k']} E={dom['E']} {dom['mode']}",
                "bytes_per_launch": dom["bytes"],
                "avg_launch_ms": round(dom_ms, 4),
                "launches_timed": args.steps,
                "peak_source": f"{peak_src} (copy bandwidth)",
                "kernel_share_of_step": round(per_kernel[dom_name] / total_kernel_ms, 3),
                "shares_from": f"{prof_steps} warm-up steps with events around every launch",
                "nominal_gbs": round(info["nominal_gbs"], 1),
                "frac_nominal": round(achieved / info["nominal_gbs"], 4)}
    if args.points_out and rank == 0:
        with open(args.points_out, "w") as fh:
            json.dump({key: {"k": v["k"], "E": v["E"], "mode": v["mode"], "kernel": v["kernel"],
                             "median_ms": statistics.median(v["ms"]),
                             "gbs": v["bytes"] / (statistics.median(v["ms"]) * 1e-3) / 1e9}
                       for key, v in per_point.items()}, fh, indent=0)
    large = {}
    for key, v in per_point.items():
        if v["k"] >= 26:
            large[key] = round(v["bytes"] / (statistics.median(v["ms"]) * 1e-3) / 1e9, 1)

    # The sections after the sweep report an error in their place rather
    # than ending the run: the sweep's line is printed whatever they do.
    def section(name, fn):
        try:
            return fn()
        except Exception as exc:  # noqa: BLE001 -- reported in the JSON line
            import traceback
            traceback.print_exc()
            return {"error": f"{name}: {type(exc).__name__}: {exc}"}

    # ---------------------------------------------------- batched (cfg 4)
    batched = None
    if not args.no_batched:
        batched = section("batched", lambda: bench_batched(
            torch, brev, inputs, device, stream, sampler, reduce_max, barrier,
            count=args.batch_count, kmax=args.batch_kmax, ws=ws, rank=rank))

    # ------------------------------------- large single arrays (cfg 3)
    large_cfg = None
    if not args.no_large:
        large_cfg = section("large", lambda: bench_large(
            torch, brev, inputs, device, stream, sampler, reduce_max, barrier, peak,
            info["nominal_gbs"]))

    # ----------------------- mid-size arrays, back to back (cfg 2 detail)
    midsize = None
    if not args.no_midsize:
        midsize = section("midsize", lambda: bench_midsize(
            torch, brev, device, stream, sampler, reduce_max, barrier, peak,
            info["l2_bytes"]))

    # -------------------------------------------- widened rows (NEXT)
    next_rows = None
    if not args.no_next:
        next_rows = section("next", lambda: bench_next(
            torch, brev, inputs, device, stream, sampler, reduce_max, barrier, peak,
            k=args.next_k))

    # ---------- one array over all ranks (N > 1), or its local passes (N = 1)
    distributed = None
    if ws > 1:
        distributed = section("distributed", lambda: bench_distributed(
            torch, brev, device, stream, sampler, reduce_max, barrier, ws, rank))
    elif not args.no_next:
        distributed = section("distributed local passes", lambda: bench_dist_local(
            torch, brev, device, stream, sampler, barrier, peak))

    # ------------------------------------------------------------ e2e
    e2e = None
    if not args.no_e2e:
        e2e = section("e2e", lambda: bench_e2e(
            torch, brev, inputs, pts, seq, args.e2e_steps, stream, sampler, reduce_max,
            barrier, ws))
    # ---------------------------------------------------- serving (cfg 5)
    serving = None
    if not args.no_serve:
        from paper_1708_01873_gb300.serve import serve_poisson
        for p in pts:  # release the sweep's buffers for the serving pool
            p["src"] = p["dst"] = None
        torch.cuda.empty_cache()
        sampler.pause()
        arena = torch.empty(16 << 30, dtype=torch.uint8, device=device)
        native = section("serving", lambda: traced_run(brev, arena, resident=False,
                                                       seconds=args.serve_seconds))
        resident = section("resident serving", lambda: traced_run(
            brev, arena, resident=True, seconds=args.serve_seconds))
        rate_sweep = None
        if not args.no_serve_sweep:
            rate_sweep = section("serving rate sweep", lambda: serving_rate_sweep(
                brev, arena, args.sweep_seconds))
        del arena
        torch.cuda.empty_cache()
        py = section("python serving", lambda: serve_poisson(
            seconds=min(args.serve_seconds, 5.0), rate=20000.0, seed=5, pool_bytes=16 << 30,
            device=local))
        sampler.resume()
        serving = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in native.items()}
        serving["loop"] = "native C++ (brev_server_run_poisson)"
        serving["workload"] = ("Poisson arrivals, mean 50 us apart (20k req/s), k uniform in "
                               "[10,24], E uniform in {4,8,16}, seed 5; arena 16 GiB, 256 "
                               "slots, 4 streams; latency = completion seen by the serving "
                               "thread - arrival (device-clock figures: device_p50_us, "
                               "device_p99_us)")
        serving["clock_sampling"] = "paused (nvidia-smi polling stalls the host loop)"
        serving["resident"] = {
            "loop": "one resident kernel fed through a page-locked request ring (no launch "
                    "per request)",
            **{k: (round(v, 1) if isinstance(v, float) else v) for k, v in resident.items()
               if k in ("completed", "p50_us", "p99_us", "max_us", "mean_us", "queue_p99_us",
                        "gbs", "launches", "max_inflight", "peak_pool_bytes", "error",
                        "by_size")}}
        serving["rate_sweep"] = rate_sweep
        serving["python_loop"] = {k: py[k] for k in ("completed", "p50_us", "p99_us", "gbs",
                                                     "mean_batch", "error") if k in py}
    sampler.stop()
    clocks = sampler.summary()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = section("cpu baseline", lambda: cpu_baseline(args.cpu_seconds))

    for p in pts:
        p["src"] = p["dst"] = None
    if rank == 0:
        line = {
            "metric": "bit-reverse GB/s (read+write) & % of HBM peak; batched vs looped launches",
            "value": round(value, 1), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_LABEL,
            "data": "synthetic (seeded SplitMix64: uint32, float32 U[-1,1), complex<float>, "
                    "complex<double>)",
            "config": sweep_config(args.kmax, args.kinds, ws, info["l2_bytes"] >> 20),
            "roofline": roofline,
            "frac_of_peak": round(value / ws / peak, 4),
            "frac_of_nominal": round(value / ws / info["nominal_gbs"], 4),
            "large_arrays_gbs": large,
            "large_arrays_from": "warm-up steps with CUDA events around every launch",
            "batched": batched,
            "serving": serving,
            "large_single_arrays": large_cfg,
            "midsize_back_to_back": midsize,
            "distributed_single_array": distributed,
            "transpositions_and_recursive": next_rows,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "device": info["name"],
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def kernel_source_hash() -> str:
    """Hash of the tile-kernel sources; a recorded ncu traffic figure is
    used only while it matches."""
    import hashlib
    h = hashlib.sha256()
    for f in ("brev_device.cuh", "brev_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1708_01873_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel_name, k, E, mode):
    """DRAM read + write bytes of one launch of ``kernel_name`` at (k, E,
    mode), from profiles/traffic.txt (an ncu capture of that launch), or
    None if none was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    h = kernel_source_hash()
    with open(p) as fh:
        for line in fh:
            parts = line.split()
            # kernel k E mode source_hash dram_read dram_write
            if (len(parts) >= 7 and not line.startswith("#") and parts[0] == kernel_name
                    and parts[1] == str(k) and parts[2] == str(E) and parts[3] == mode
                    and parts[4] == h):
                return int(float(parts[5]) + float(parts[6]))
    return None


def event_timer(torch, stream, sampler, reduce_max, barrier, reps, warm):
    """timed(fn): `warm` untimed calls, then the mean of `reps` calls on
    `stream` between two CUDA events (barrier on both sides, max over
    ranks); the clock sampler's window covers the timed calls."""
    def timed(fn):
        for _ in range(warm):
            fn()
        barrier()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        ea.record(stream)
        for _ in range(reps):
            fn()
        eb.record(stream)
        barrier()
        sampler.window(w0, time.time())
        return reduce_max(ea.elapsed_time(eb)) / reps
    return timed


def bench_large(torch, brev, inputs, device, stream, sampler, reduce_max, barrier, peak,
                nominal, reps=5, warm=2):
    """The large single arrays: k = 30 float32 in place (4 GiB), k = 28
    complex<double> in place (4 GiB), k = 29 complex<float> out of place
    (odd k, 4 GiB -> 4 GiB).  Arrays far larger than L2, so no flush."""
    L = brev.lib()
    sh = stream.cuda_stream
    timed = event_timer(torch, stream, sampler, reduce_max, barrier, reps, warm)
    out = {}
    for kind, E, k, inplace in (("f32", 4, 30, True), ("c128", 16, 28, True),
                                ("c64", 8, 29, False)):
        src = torch.empty((1 << k) * E, dtype=torch.uint8, device=device)
        inputs.fill_torch(src, 30 + k, kind, chunk=1 << 26)
        dst = src if inplace else torch.empty_like(src)
        ms = timed(lambda: L.brev_permute_to(dst.data_ptr(), src.data_ptr(), k, E, sh))
        gbs = 2 * src.numel() / (ms * 1e-3) / 1e9
        bx, bz, order = brev.brev_tile_shape(k, E, inplace)
        out[f"{kind}_k{k}_{'in_place' if inplace else 'out_of_place'}"] = {
            "ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
            "frac_nominal": round(gbs / nominal, 4), "tile": [bx, bz, order]}
        del src, dst
    torch.cuda.empty_cache()
    return out


def _graph_of(torch, stream, fns):
    """A CUDA graph of the launches fns() enqueue on `stream`."""
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        for f in fns:
            f()
    return g


def _replay_ms(torch, stream, g, reps=3):
    """Mean time of one replay of graph g (two warm-up replays first)."""
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bench_midsize(torch, brev, device, stream, sampler, reduce_max, barrier, peak, l2_bytes,
                  ks=range(18, 26), kinds=(("f32", 4), ("c64", 8), ("c128", 16))):
    """Single arrays of k = 18..25 timed as R back-to-back launches captured
    in one CUDA graph (no event between launches).  cold: the launches
    rotate over buffer sets whose footprint together exceeds 3x L2, so every
    launch reads its input from HBM; warm: one buffer set (out of place
    ping-pong), L2-resident when it fits; copy: torch's device copy of the
    same bytes, timed the same way -- the per-launch ceiling any kernel of
    that size meets.  Beside them, C equal arrays of about 1 GiB in all: the
    loop of C single launches (one graph) against one batched launch (a
    plan)."""
    L = brev.lib()
    sh = stream.cuda_stream
    out = {"method": "R launches per CUDA graph replay; GB/s = 2 n E x R / replay time; "
                     "cold rotates buffers totalling > 3x L2, warm reuses one set",
           "points": {}, "batched_vs_loop": {}}
    w0 = time.time()
    for kind, E in kinds:
        for k in ks:
            nb = E << k
            for ip in (False, True):
                foot = nb if ip else 2 * nb
                M = max(1, min(-(-3 * l2_bytes // foot), (6 << 30) // foot))
                bufs = [torch.empty(nb, dtype=torch.uint8, device=device)
                        for _ in range(M if ip else 2 * M)]
                for b_ in bufs:
                    b_.fill_(0x5A)
                sets = ([(b_, b_) for b_ in bufs] if ip else
                        [(bufs[2 * i + 1], bufs[2 * i]) for i in range(M)])
                R = max(8, min(256, int(4e-3 / (2 * nb / 6.5e12))))

                def launch(d, s_):
                    return lambda: L.brev_permute_to(d.data_ptr(), s_.data_ptr(), k, E, sh)
                cold = [launch(*sets[r % M]) for r in range(R)]
                d0, s0 = sets[0]
                warm = [launch(d0, s0) if (ip or r % 2 == 0) else launch(s0, d0)
                        for r in range(R)]
                rec = {}
                for name, fns in (("cold", cold), ("warm", warm)):
                    g = _graph_of(torch, stream, fns)
                    ms = _replay_ms(torch, stream, g) / R
                    rec[f"{name}_gbs"] = round(2 * nb / (ms * 1e-3) / 1e9, 1)
                    del g
                if not ip:
                    f32 = [(d.view(torch.float32), s_.view(torch.float32)) for d, s_ in sets]
                    g = _graph_of(torch, stream,
                                  [lambda d=f32[r % M][0], s_=f32[r % M][1]: d.copy_(s_)
                                   for r in range(R)])
                    ms = _replay_ms(torch, stream, g) / R
                    rec["copy_cold_gbs"] = round(2 * nb / (ms * 1e-3) / 1e9, 1)
                    del g
                rec["cold_frac"] = round(rec["cold_gbs"] / peak, 4)
                rec["tile"] = list(brev.brev_tile_shape(k, E, ip))
                out["points"][f"{kind}_{'ip' if ip else 'oop'}_k{k}"] = rec
                del bufs, sets, cold, warm
                torch.cuda.empty_cache()
        for k in range(18, 25):
            nb = E << k
            C = max(2, min(512, (1 << 30) // nb))
            arrs = [torch.full((nb,), 3, dtype=torch.uint8, device=device) for _ in range(C)]
            views = [a.view({4: torch.float32, 8: torch.complex64, 16: torch.complex128}[E])
                     for a in arrs]
            g = _graph_of(torch, stream,
                          [lambda a=a: L.brev_permute_to(a.data_ptr(), a.data_ptr(), k, E, sh)
                           for a in arrs])
            loop_ms = _replay_ms(torch, stream, g)
            del g
            plan = brev.BrevPlan(views)
            for _ in range(2):
                plan.launch(stream)
            torch.cuda.synchronize()
            ea = torch.cuda.Event(enable_timing=True)
            eb = torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            for _ in range(8):
                plan.launch(stream)
            eb.record(stream)
            torch.cuda.synchronize()
            plan_ms = ea.elapsed_time(eb) / 8
            plan.close()
            tot = 2 * nb * C
            out["batched_vs_loop"][f"{kind}_k{k}_x{C}"] = {
                "loop_gbs": round(tot / (loop_ms * 1e-3) / 1e9, 1),
                "batched_gbs": round(tot / (plan_ms * 1e-3) / 1e9, 1),
                "speedup": round(loop_ms / plan_ms, 3)}
            del arrs, views
            torch.cuda.empty_cache()
    sampler.window(w0, time.time())
    return out


def bench_distributed(torch, brev, device, stream, sampler, reduce_max, barrier, ws, rank,
                      log2_block=27, reps=5, warm=2):
    """One complex<double> array of ws x 2^27 elements (2 GiB per rank)
    spread over the ranks: pack (local pass), all-to-all (NCCL), finish
    (local pass), timed on the launch stream with a barrier on both sides,
    max over ranks.  Runs only with a power-of-two number of ranks."""
    import torch.distributed as dist
    g = ws.bit_length() - 1
    if ws != 1 << g:
        return {"skipped": f"{ws} ranks is not a power of two"}
    E = 16
    k = log2_block + g
    block = torch.empty((1 << log2_block) * E, dtype=torch.uint8, device=device)
    block.fill_(rank & 0xFF)
    recv = torch.empty_like(block)
    blk = block.view(torch.complex128)
    rcv = recv.view(torch.complex128)
    L = brev.lib()
    sh = stream.cuda_stream

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        brev.brev_dist_pack(blk, blk, k, g, stream)
        if ev:
            ev[1].record(stream)
        dist.all_to_all_single(recv, block)
        if ev:
            ev[2].record(stream)
        brev.brev_dist_finish(blk, rcv, k, g, stream)
        if ev:
            ev[3].record(stream)

    for _ in range(warm):
        step()
    barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    w0 = time.time()
    for e in evs:
        step(e)
    barrier()
    sampler.window(w0, time.time())
    tot = reduce_max(evs[0][0].elapsed_time(evs[-1][3])) / reps
    pack = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    a2a = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    fin = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    nbytes = 2 * (E << k)  # the whole array read and written once
    return {"workload": f"complex<double>, k={k} over {ws} ranks (2^{log2_block} elements each)",
            "ms_per_step": round(tot, 4), "gbs": round(nbytes / (tot * 1e-3) / 1e9, 1),
            "rank0_pack_ms": round(pack, 4), "rank0_all_to_all_ms": round(a2a, 4),
            "rank0_finish_ms": round(fin, 4),
            "exchange": "torch.distributed.all_to_all_single (NCCL), equal segments"}


def bench_dist_local(torch, brev, device, stream, sampler, barrier, peak, log2_block=27,
                     reps=5, warm=2):
    """One GPU: the two local passes of the permutation spread over G = 2, 4,
    8, 16 ranks, on one rank's block of 2^27 complex<double> (2 GiB) --
    the pack (a (k-g)-bit permutation in place) and the finish (a 2^g x
    2^(k-2g) transposition with bit-reversed rows, out of place) -- each
    timed back to back with CUDA events.  The exchange between them needs
    several GPUs and is not run here."""
    E = 16
    blk = torch.empty((1 << log2_block) * E, dtype=torch.uint8, device=device)
    blk.fill_(0x3C)
    rcv = torch.empty_like(blk)
    b = blk.view(torch.complex128)
    r = rcv.view(torch.complex128)
    nbytes = 2 * blk.numel()
    timed = event_timer(torch, stream, sampler, lambda x: x, barrier, reps, warm)
    out = {"block": f"2^{log2_block} complex<double> (2 GiB) per rank"}
    for g in (1, 2, 3, 4):
        k = log2_block + g
        pack = timed(lambda: brev.brev_dist_pack(b, b, k, g, stream))
        fin = timed(lambda: brev.brev_dist_finish(b, r, k, g, stream))
        out[f"G{1 << g}"] = {"pack_ms": round(pack, 4),
                             "pack_gbs": round(nbytes / (pack * 1e-3) / 1e9, 1),
                             "finish_ms": round(fin, 4),
                             "finish_gbs": round(nbytes / (fin * 1e-3) / 1e9, 1),
                             "finish_frac": round(nbytes / (fin * 1e-3) / 1e9 / peak, 4)}
    del blk, rcv
    torch.cuda.empty_cache()
    return out


def bench_next(torch, brev, inputs, device, stream, sampler, reduce_max, barrier, peak,
               reps=5, warm=2, k=28):
    """The widened rows: transpositions (square and narrow: the even-odd step
    and the perfect shuffle) and the paper's recursive method (three passes)
    against the one-pass tile kernel, all on 4 GiB arrays."""
    L = brev.lib()
    sh = stream.cuda_stream
    timed = event_timer(torch, stream, sampler, reduce_max, barrier, reps, warm)

    out = {}
    E = 16
    h = k // 2
    src = torch.empty((1 << k) * E, dtype=torch.uint8, device=device)
    inputs.fill_torch(src, 28, "c128", chunk=1 << 26)
    dst = torch.empty_like(src)
    nbytes = 2 * src.numel()
    for name, a, c in ((f"transpose_{1 << h}x{1 << (k - h)}_c128", h, k - h),
                       (f"even_odd_c128_k{k}", k - 1, 1), (f"perfect_shuffle_c128_k{k}", 1, k - 1)):
        ms = timed(lambda: L.brev_transpose(dst.data_ptr(), src.data_ptr(), a, c, E, sh))
        out[name] = {"ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}
    ms = timed(lambda: L.brev_transpose(dst.data_ptr(), dst.data_ptr(), h, h, E, sh))
    out[f"transpose_in_place_{1 << h}x{1 << h}_c128"] = {
        "ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
        "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}
    one = timed(lambda: L.brev_permute_to(dst.data_ptr(), dst.data_ptr(), k, E, sh))
    rec = timed(lambda: L.brev_permute_recursive(dst.data_ptr(), k, E, sh))
    out[f"recursive_vs_one_pass_c128_k{k}"] = {
        "one_pass_ms": round(one, 4), "recursive_ms": round(rec, 4),
        "ratio": round(rec / one, 3),
        "one_pass_gbs": round(nbytes / (one * 1e-3) / 1e9, 1),
        "recursive_hbm_passes": 3}
    # bit reversal fused with the first DIT FFT stages vs the plain permutation.
    # complex<double> stages are bound by the FP64 pipe: the peak is measured
    # on this GPU in the same run (brev_fp64_fma_tflops: independent FMA
    # chains on every SM); beside it the figure derived from the SM count,
    # 2 FP64 FMA per SM per cycle (the issue peak ncu reports for GB300),
    # 2 flops and the maximum SM clock nvidia-smi reports.
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    max_mhz = max((smp[2] for smp in sampler.samples), default=None)
    fp64_derived = sm_count * FP64_FMA_PER_SM_CLK * 2 * max_mhz * 1e6 / 1e12 if max_mhz else None
    w0 = time.time()
    fp64_peak = brev.brev_fp64_fma_tflops()
    sampler.window(w0, time.time())
    for kind, E, S in (("c64", 8, 6), ("c128", 16, 5)):
        k2 = k
        x = torch.empty((1 << k2) * E, dtype=torch.uint8, device=device)
        inputs.fill_torch(x, 29, kind, chunk=1 << 26)
        y = torch.empty_like(x)
        nb = 2 * x.numel()
        plain = timed(lambda: L.brev_permute_to(y.data_ptr(), x.data_ptr(), k2, E, sh))
        fused = timed(lambda: L.brev_fft_stages(y.data_ptr(), x.data_ptr(), k2, E, S, 0, sh))
        fused_ip = timed(lambda: L.brev_fft_stages(y.data_ptr(), y.data_ptr(), k2, E, S, 0, sh))
        flops = 5.0 * (1 << k2) * S  # radix-2 butterfly stage: 5 n flops
        out[f"fft_stages_{kind}_k{k2}_S{S}"] = {
            "permute_ms": round(plain, 4), "fused_ms": round(fused, 4),
            "fused_in_place_ms": round(fused_ip, 4),
            "fused_gbs": round(nb / (fused * 1e-3) / 1e9, 1),
            "fused_frac": round(nb / (fused * 1e-3) / 1e9 / peak, 4),
            "fused_gflops": round(flops / (fused * 1e-3) / 1e9, 1),
            "stages_cost_vs_permute": round(fused / plain, 3)}
        if E == 16 and fp64_peak:
            ach = flops / (fused * 1e-3) / 1e12
            out[f"fft_stages_{kind}_k{k2}_S{S}"]["roofline"] = {
                "bound": "alu", "unit": "TFLOP/s", "achieved": round(ach, 3),
                "peak": round(fp64_peak, 3), "frac": round(ach / fp64_peak, 4),
                "counted": "5 n flops per radix-2 stage",
                "peak_source": "measured in this run: FP64 FMA chains on every SM "
                               "(brev_fp64_fma_tflops), 2 flops per FMA",
                "derived_peak": round(fp64_derived, 3) if fp64_derived else None,
                "derived_from": (f"{sm_count} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA/SM/cycle x "
                                 f"2 flops x {max_mhz:.0f} MHz") if max_mhz else None}
        del x, y
    del src, dst
    return out


SIZE_CLASSES = ((10, 16), (17, 20), (21, 22), (23, 24))


def latency_by_size(trace):
    """Per-request latency (completion seen by the serving thread -
    arrival, from the trace) by array size class: count, p50, p99 and the
    share of the run's slowest 1 % that the class holds."""
    import numpy as np
    trace = [r for r in (trace or []) if r["seen_us"] > 0]
    if not trace:
        return None
    lat = np.array([r["seen_us"] - r["arrival_us"] for r in trace])
    ks = np.array([r["log2n"] for r in trace])
    cut = np.percentile(lat, 99)
    slow = lat >= cut
    out = {}
    for lo, hi in SIZE_CLASSES:
        m = (ks >= lo) & (ks <= hi)
        if not m.any():
            continue
        out[f"k{lo}-{hi}"] = {"count": int(m.sum()),
                              "p50_us": round(float(np.percentile(lat[m], 50)), 1),
                              "p99_us": round(float(np.percentile(lat[m], 99)), 1),
                              "share_of_slowest_1pct": round(float((slow & m).sum() / slow.sum()), 3)}
    return out


def traced_run(brev, arena, resident, seconds, rate=20000.0):
    """The 20k req/s headline run of one serving mode, with the per-request
    trace summarised by size class."""
    st, tr = brev.brev_server_run_poisson(arena, seed=5, rate_per_s=rate, seconds=seconds,
                                          resident=resident, trace=True)
    st["by_size"] = latency_by_size(tr)
    return st


def serving_rate_sweep(brev, arena, seconds):
    """Poisson arrival rates of 20k..200k req/s for three servers -- the
    launch loop with one request per launch, the loop with continuous
    batching (up to 256 requests per launch), and the resident kernel -- on
    the configured mix (k 10..24) and on small requests (k 10..16), E in
    {4, 8, 16}.  Each point reports the sustained completions per second,
    GB/s and latency; a server that cannot keep up completes fewer requests
    per second than offered and its latency grows with the backlog."""
    servers = (("launch_one_per_launch", dict(resident=False, max_batch=1)),
               ("launch_batched", dict(resident=False, max_batch=256)),
               ("resident", dict(resident=True)))
    out = {"seconds_per_point": seconds, "points": {}}
    for mix, kr in (("mix_k10-24", (10, 24)), ("small_k10-16", (10, 16))):
        for rate in (20000.0, 50000.0, 100000.0, 200000.0):
            for name, kw in servers:
                st, _ = brev.brev_server_run_poisson(arena, seed=6, rate_per_s=rate,
                                                     seconds=seconds, k_range=kr, **kw)
                out["points"][f"{mix}_{int(rate / 1000)}k_{name}"] = {
                    "offered_req_per_s": rate,
                    "completed_req_per_s": round(st["req_per_s"], 1),
                    "gbs": round(st["gbs"], 1),
                    "p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1),
                    "max_us": round(st["max_us"], 1),
                    "mean_batch": round(st["completed"] / max(1, st["batches"]), 2),
                    "launches": st["launches"]}
    return out


def bench_batched(torch, brev, inputs, device, stream, sampler, reduce_max, barrier,
                  reps=10, warm=3, count=4096, kmax=20, ws=1, rank=0):
    """The 4096-array batch: one persistent launch (as a captured plan, and
    per call) against a loop of single-array launches (plain and captured).
    With several ranks the batch is split across them by array
    (brev_shard_batch: strong scaling, each rank launches its share) and
    GB/s counts the whole batch over the slowest rank's time."""
    import numpy as np
    rng = np.random.default_rng(4)
    ks = rng.integers(8, kmax + 1, size=count)
    Es = rng.choice([8, 16], size=count)
    owner = (brev.brev_shard_batch([int(x) for x in ks], [int(x) for x in Es], ws)
             if ws > 1 else [0] * count)
    arrays = []
    kept = []
    for i in range(count):
        if owner[i] != rank:
            continue
        E = int(Es[i])
        a = torch.empty((1 << int(ks[i])) * E, dtype=torch.uint8, device=device)
        inputs.fill_torch(a, 40000 + i, "c64" if E == 8 else "c128", chunk=1 << 26)
        arrays.append(a.view(torch.complex64 if E == 8 else torch.complex128))
        kept.append(i)
    total = sum(2 * (int(E) << int(k)) for k, E in zip(ks, Es))  # the whole batch
    ks = ks[kept]
    Es = Es[kept]
    L = brev.lib()
    sh = stream.cuda_stream
    plan = brev.BrevPlan(arrays)
    ptrs = [a.data_ptr() for a in arrays]
    kk = [int(x) for x in ks]
    ee = [int(x) for x in Es]

    def loop():
        for p, k, E in zip(ptrs, kk, ee):
            L.brev_permute_to(p, p, k, E, sh)

    def one_batched():
        brev.brev_permute_batched(arrays, stream=stream)

    def graph_replay():
        plan.launch(stream)

    # the loop of single launches captured into a CUDA graph too
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device)
    torch.cuda.synchronize(device)
    c0 = L.brev_launch_count()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="thread_local"):
        for p, k, E in zip(ptrs, kk, ee):
            L.brev_permute_to(p, p, k, E, cap.cuda_stream)
    loop_launches = L.brev_launch_count() - c0

    def loop_graph():
        g.replay()

    out = {}
    for name, fn in (("persistent_graph", graph_replay), ("persistent", one_batched),
                     ("loop", loop), ("loop_graph", loop_graph)):
        for _ in range(warm):
            fn()
        barrier()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        ea.record(stream)
        for _ in range(reps):
            fn()
        eb.record(stream)
        barrier()
        sampler.window(w0, time.time())
        ms = reduce_max(ea.elapsed_time(eb)) / reps
        out[name] = {"ms": round(ms, 3), "gbs": round(total / (ms * 1e-3) / 1e9, 1)}
    plan.close()
    tuned_b = sorted({(E, k, brev.brev_batched_shape(k, E)) for E in (8, 16)
                      for k in range(8, kmax + 1)})
    res = {"workload": f"{count} arrays, k uniform in [8,{kmax}], E uniform in {{8,16}} "
                       "(seed 4), in place; persistent = one launch per batch",
           "sharding": (f"{ws} ranks by array (brev_shard_batch), strong scaling: "
                        f"{len(kept)} arrays on rank 0") if ws > 1 else "1 GPU",
           "tile_exponent_b": {f"E{E}_k{k}": b for E, k, b in tuned_b},
           "tile_exponent_from": "autotuned table (brev_autotune, tune_gb300.json)",
           "bytes_per_batch": total, "launches_in_loop": int(loop_launches), **out,
           "speedup_persistent_graph_vs_loop": round(out["loop"]["ms"] /
                                                     out["persistent_graph"]["ms"], 2),
           "speedup_persistent_graph_vs_loop_graph": round(out["loop_graph"]["ms"] /
                                                           out["persistent_graph"]["ms"], 2)}
    del arrays
    return res


def bench_e2e(torch, brev, inputs, pts, seq, steps, stream, sampler, reduce_max, barrier,
              ws):
    """The sweep through brev_permute_host, every point every step, timed on
    the host clock around the calls (each returns with its result in host
    memory).  The buffers are page-locked, so the tile kernel reads each
    input from host memory and writes each result to host memory over
    NVLink-C2C: every step moves all inputs host -> device and all results
    device -> host, with no device copy in between."""
    L = brev.lib()
    sh = stream.cuda_stream
    kinds = {}
    for p in pts:
        kinds[p["kind"]] = max(kinds.get(p["kind"], 0), p["src"].numel())
    host_src = {}
    for kind, nbytes in kinds.items():
        h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        # the prefix of a seeded array is the seeded array of that length
        inputs.fill_torch(h, 100, kind, chunk=1 << 26)
        host_src[kind] = h
    host_dst = torch.empty(max(kinds.values()), dtype=torch.uint8, pin_memory=True)
    h2d = sum(p["src"].numel() for p, _ in seq)

    def step():
        for p, ip in seq:
            nb = p["src"].numel()
            s = host_src[p["kind"]]
            d = s if ip else host_dst
            rc = L.brev_permute_host(d.data_ptr(), s.data_ptr(), p["k"], p["E"], sh)
            if rc != 0:
                raise RuntimeError(brev.brev_last_error())

    step()  # warm-up (pool growth)
    # in-place steps change host_src; restore for a clean next run is not
    # needed for timing (content does not affect the permutation's cost)
    barrier()
    w0 = time.time()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    barrier()
    el = reduce_max(time.perf_counter() - t0)
    sampler.window(w0, time.time())
    step_bytes = sum(p["bytes"] for p, _ in seq)
    value = ws * step_bytes * steps / el / 1e9
    # the link's ceiling for the same traffic, measured the same way: every
    # point's input copied host -> device on one stream while its size in
    # results goes device -> host on another (cudaMemcpyAsync through torch,
    # page-locked buffers), host clock around each step
    s_in = torch.cuda.Stream(stream.device)
    s_out = torch.cuda.Stream(stream.device)

    def link_step():
        with torch.cuda.stream(s_in):
            for p, _ in seq:
                nb = p["src"].numel()
                p["dst"].copy_(host_src[p["kind"]][:nb], non_blocking=True)
        with torch.cuda.stream(s_out):
            for p, _ in seq:
                nb = p["src"].numel()
                host_dst[:nb].copy_(p["src"], non_blocking=True)
        s_in.synchronize()
        s_out.synchronize()

    link_step()
    barrier()
    w0 = time.time()
    t0 = time.perf_counter()
    for _ in range(steps):
        link_step()
    barrier()
    el_link = reduce_max(time.perf_counter() - t0)
    sampler.window(w0, time.time())
    ce = ws * step_bytes * steps / el_link / 1e9
    # the route the permutation itself takes: SMs reading and writing
    # page-locked host memory, measured as a plain copy kernel over the
    # largest pair of buffers (4 GiB)
    big = max(host_src, key=lambda kd: host_src[kd].numel())
    w0 = time.time()
    link = brev.brev_host_link_gbs(host_dst, host_src[big][:host_dst.numel()])
    sampler.window(w0, time.time())
    return {"value": round(value, 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d, "steps": steps,
            "api": "brev_permute_host on page-locked host buffers: the kernel reads each "
                   "input from and writes each result to host memory over NVLink-C2C, "
                   "every point every step, host clock around the calls",
            "link_gbs": round(link, 1), "frac": round(value / link, 4),
            "link_from": "copy kernel reading and writing page-locked host memory over "
                         "NVLink-C2C (brev_host_link_gbs, 4 GiB, read + write bytes, events)",
            "copy_engine_gbs": round(ce, 1),
            "copy_engine_from": "the same bytes moved by concurrent host->device and "
                                "device->host cudaMemcpyAsync (two streams, page-locked "
                                "buffers), host clock"}


# --------------------------------------------------------- CPU baseline --
def oracle_points(k):
    from paper_1708_01873_gb300 import inputs
    return [(kind, E, k, inputs.array_np(100 + k, 1 << k, kind)) for kind, E in SWEEP_KINDS]


def time_oracle(points):
    """Run the plain oracle out-of-place and in-place on every point; returns
    (algorithmic bytes, seconds spent inside the oracle)."""
    import oracle
    nbytes, secs = 0, 0.0
    for kind, E, k, src in points:
        t0 = time.perf_counter()
        oracle.brev_oop(src, k, E)
        secs += time.perf_counter() - t0
        b = src.copy()
        t0 = time.perf_counter()
        oracle.brev_inplace(b, k, E)
        secs += time.perf_counter() - t0
        nbytes += 2 * (2 * (1 << k) * E)
    return nbytes, secs


def largest_k_within(budget_s):
    """Largest sweep k such that the sweep truncated at k takes about
    budget_s seconds of oracle time (each k costs about twice the previous)."""
    import oracle
    oracle.build()
    done_s, last_k, pts_all = 0.0, SWEEP_KS[0], []
    for k in SWEEP_KS:
        if done_s and done_s * 2.2 > budget_s:
            break
        pts = oracle_points(k)
        _, t = time_oracle(pts)
        done_s += t
        last_k = k
        pts_all += pts
    return last_k, pts_all


def time_oracle_mt(points, threads):
    """The oracle's threaded out-of-place copy (index range split over
    ``threads`` host threads) on every point; returns (algorithmic bytes,
    seconds, threads actually used)."""
    import oracle
    nbytes, secs, used = 0, 0.0, 1
    for kind, E, k, src in points:
        t0 = time.perf_counter()
        _, u = oracle.brev_oop_mt(src, k, E, threads)
        secs += time.perf_counter() - t0
        used = max(used, u)
        nbytes += 2 * (1 << k) * E
    return nbytes, secs, used


def cpu_baseline(budget_s):
    """The plain single-thread oracle timed on the host cores over the sweep
    truncated at the largest k that fits about ``budget_s`` seconds; beside
    it, the oracle's threaded out-of-place copy on the same points with every
    host thread."""
    kmax, pts = largest_k_within(budget_s / 2)
    nbytes, secs = time_oracle(pts)
    threads = os.cpu_count() or 1
    mt_bytes, mt_secs, used = time_oracle_mt(pts, threads)
    return {"value": round(nbytes / secs / 1e9, 3), "unit": "GB/s", "cores": 1,
            "kind": "oracle",
            "sample": f"sweep k=10..{kmax} x {{u32,f32,c64,c128}} x {{oop,in-place}}, "
                      f"plain single-thread C oracle, {secs:.1f} s timed",
            "seconds": round(secs, 2),
            "threaded": {"value": round(mt_bytes / mt_secs / 1e9, 3), "unit": "GB/s",
                         "cores": used, "host_threads": threads,
                         "sample": f"the same points, out of place only, index range split "
                                   f"over {used} threads, {mt_secs:.2f} s timed"}}


def reference_l2_mib():
    """L2 size for the shared config line, if a GPU is visible (the oracle
    itself needs none)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_properties(0).L2_cache_size >> 20
    except Exception:  # noqa: BLE001 -- informational only
        pass
    return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # size each step so that the whole run stays within about 90 s
    budget = max(0.02, args.ref_seconds / max(1, args.steps + args.warmup))
    kmax, pts = largest_k_within(budget)
    for _ in range(args.warmup):
        time_oracle(pts)
    tot_bytes, secs = 0, 0.0
    for _ in range(args.steps):
        b, t = time_oracle(pts)
        tot_bytes += b
        secs += t
    value = tot_bytes / secs / 1e9
    line = {"metric": "bit-reverse GB/s (read+write) & % of HBM peak; batched vs looped launches",
            "impl": "reference", "value": round(value, 3), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_LABEL,
            "data": "synthetic (seeded SplitMix64)",
            "config": sweep_config(args.kmax, args.kinds, ws, reference_l2_mib()),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"bounded sample of that sweep: each step the points "
                                       f"k=10..{kmax} of every kind, out of place and in "
                                       f"place, on the plain single-thread C oracle"},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_brev(args)


if __name__ == "__main__":
    main()
