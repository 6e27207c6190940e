#!/usr/bin/env python3
"""Benchmark: compact cell-updates/s of the life step on the Sierpinski
triangle F^{3,2} at r = 20 (3.49e9 compact cells, Bernoulli(0.3) seed 3,
B3/S23) on one GB300, with its HBM roofline fraction, next to the
bounding-box step at r = 16 (the largest level whose box fits), the
end-to-end call from host buffers, and the CPU oracle on the host cores.

One benchmark step is one generation of the whole hot path over the whole
state: for every compact cell lambda, the Moore probe, nu and the rule
(one launch of the tiled step kernel).  Inputs are already resident in HBM
when the timed region starts; the state (3.49 GB per buffer) is far larger
than the 129 MB L2, so no flush is needed between iterations of the
headline; the r = 16 compact comparison fits in L2 and is timed with an L2
flush between generations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compact cell-updates/s (Sierpinski triangle r=20, B3/S23) and % HBM roofline vs bounding box on 1 GB300"
UNIT = "cell-updates/s"
KERNEL_SRC = os.path.join(ROOT, "paper_2110_12952_gb300", "csrc", "step.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--r", type=int, default=20, help="triangle level of the headline workload")
    ap.add_argument("--bb-r", type=int, default=16, help="level of the compact-vs-BB comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-bb", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--no-maps", action="store_true")
    ap.add_argument("--maps-only", action="store_true", help="run the maps leg alone and print it")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-plain-requests", type=int, default=600)
    ap.add_argument("--serve-chunk", type=int, default=16)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tile-levels", type=int, default=-1, help="tile depth L (-1: library choice)")
    ap.add_argument("--stages", type=int, default=-1, help="input pipeline stages with --tile-levels (-1: default)")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1 GPUs: one independent instance per GPU instead of one instance sharded")
    ap.add_argument("--shard", action="store_true", help="run the sharded path even on one GPU")
    ap.add_argument("--shard-tile-levels", type=int, default=9, help="tile depth of the sharded instance")
    return ap.parse_args()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy kernel)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 copy measurement)"


def kernel_sources(top: str = KERNEL_SRC) -> list:
    """The step kernel's source and every file it includes with #include "...",
    followed transitively."""
    import re
    seen, todo = [], [os.path.normpath(top)]
    while todo:
        path = todo.pop(0)
        if path in seen or not os.path.exists(path):
            continue
        seen.append(path)
        with open(path) as fh:
            for m in re.finditer(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), re.M):
                todo.append(os.path.normpath(os.path.join(os.path.dirname(path), m.group(1))))
    return seen


def kernel_hash() -> str:
    h = hashlib.sha256()
    for path in kernel_sources():
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; None otherwise."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        if d.get("kernel_hash") != kernel_hash() or d.get("workload") != workload:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_ready(self, timeout=5.0):
        """Wait for the first sample (nvidia-smi takes a moment to start)."""
        t_end = time.monotonic() + timeout
        while self.proc is not None and not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)

    def window(self, t0, t1):
        """Keep only the samples taken between t0 and t1 (monotonic clock)."""
        self.lines = [(t, l) for t, l in self.lines if t0 <= t <= t1]

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        rows = []
        for _, l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ CPU oracle

def oracle_sample(r: int, target_s: float, seed: int, p: float):
    """Time the oracle's compact step on the first 3^L cells of the level-r
    triangle (one level-L subtree; its neighbours lie in the first 3^(L+1)
    cells, which are initialised from the same seeded generator).  L is
    chosen from a short calibration so that the sample takes ~target_s."""
    import numpy as np
    import oracle
    from paper_2110_12952_gb300 import workloads as W
    fam = W.TRIANGLE
    o = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
    st = np.zeros(o.cells, dtype=np.uint8)   # untouched pages stay unmapped
    out = np.zeros(o.cells, dtype=np.uint8)
    Lc = min(11, r - 1)
    o.init_bernoulli(seed, p, 0, 3 ** (Lc + 1), out=st)
    t0 = time.perf_counter()
    o.step_range(st, 0, 3 ** Lc, out=out)
    rate = 3 ** Lc / max(time.perf_counter() - t0, 1e-6)
    L = Lc
    while L + 1 < r and 3 ** (L + 1) / rate <= target_s:
        L += 1
    o.init_bernoulli(seed, p, 0, 3 ** (L + 1), out=st)

    def run():
        t = time.perf_counter()
        o.step_range(st, 0, 3 ** L, out=out)
        return time.perf_counter() - t

    return o, L, run


def cpu_baseline(r, target_s, seed, p):
    import oracle
    o, L, run = oracle_sample(r, target_s, seed, p)
    dt = run()
    return {"value": 3 ** L / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"one generation of the first 3^{L} = {3 ** L} compact cells (one level-{L} "
                      f"subtree) of the triangle r={r}, seed {seed}, p={p}; {dt:.1f} s"}


def run_reference(args, rank, world):
    """The oracle timed on the host cores on the same workload and metric."""
    import oracle
    from paper_2110_12952_gb300 import workloads as W
    inst = W.TRI_R20 if args.r == 20 else W.Instance(W.TRIANGLE, args.r, 0.3, 3, 1000)
    if rank != 0:
        return None
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    o, L, run = oracle_sample(inst.r, per_step, inst.seed, inst.p)
    for _ in range(args.warmup):
        run()
    total = sum(run() for _ in range(args.steps))
    value = 3 ** L * args.steps / total
    sample = (f"each step: one generation of the first 3^{L} = {3 ** L} compact cells (a level-{L} "
              f"subtree) of the triangle r={inst.r}")
    return {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": workload_config(inst),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def workload_config(inst):
    return {"workload": f"sierpinski_triangle_F32_r{inst.r}", "fractal": "F^{3,2} offsets (0,0),(1,0),(0,1)",
            "r": inst.r, "cells": 3 ** inst.r, "p": inst.p, "seed": inst.seed, "rule": "B3/S23",
            "generations_per_step": 1,
            "l2": "state per buffer larger than the 129 MB L2; no flush needed"}


# ------------------------------------------------------------------- GPU

def time_steps(fn, steps, warmup, flush=None):
    """Per-iteration CUDA-event times (ms) on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    st = torch.cuda.current_stream()
    for _ in range(steps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def aggregate_ranks(ms_local, units_local, world, dist, device):
    """Whole-job throughput of independent replicas (one per rank, the same
    units each): the slowest rank's time (MAX over ranks) and the units of
    all ranks divided by it.  Returns (ms_max, units per second)."""
    import torch
    ms_max = float(ms_local)
    if dist is not None:
        t = torch.tensor([ms_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, units_local * world / (ms_max / 1e3)


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    from paper_2110_12952_gb300 import Fractal, build, workloads as W

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    inst = W.TRI_R20 if args.r == 20 else W.Instance(W.TRIANGLE, args.r, 0.3, 3, 1000)
    fam = inst.family
    g = Fractal.from_family(fam, inst.r)
    a = g.init_bernoulli(inst.seed + rank, inst.p)
    b = torch.empty_like(a)
    if args.tile_levels >= 0:
        g.tile_levels = args.tile_levels
        g.pipeline_stages = args.stages
    else:
        g.autotune(a, b)   # picks the tile depth; untimed
    bufs = [a, b]
    cur = [0]

    def one_generation():
        g.step(bufs[cur[0]], out=bufs[1 - cur[0]], steps=1)
        cur[0] ^= 1

    # warm-up, then exactly K timed generations bracketed by barrier + sync;
    # the clock sampler starts before the warm-up and keeps only the samples
    # taken inside the timed region
    with ClockSampler(dev.index) as clocks:
        for _ in range(args.warmup):
            one_generation()
        torch.cuda.synchronize()
        clocks.wait_ready()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t_start = time.monotonic()
        ev0.record(stream)
        for _ in range(args.steps):
            one_generation()
        ev1.record(stream)
        torch.cuda.synchronize()
        t_end = time.monotonic()
    clocks.window(t_start, t_end)
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max, value = aggregate_ranks(ms, g.cells * args.steps, world, dist, dev)
    ms_per_step = ms_max / args.steps

    # roofline of the step kernel: 2 algorithmic bytes per compact update
    peak, peak_src = measured_peak()
    alg_bytes = 2.0 * g.cells
    achieved = alg_bytes / (ms / args.steps / 1e3) / 1e9
    workload = workload_config(inst)["workload"]
    plan = g.plan_info()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_per_launch(workload),
            "kernel": f"step_tma_kernel<2,{plan['policy']},false> ({plan['policy_name']} policy)",
            "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_src,
            "tile_levels": plan["tile_levels"], "launch": {k: plan[k] for k in
                                                           ("block", "grid", "smem_bytes", "stages", "blocks_per_sm")}}

    extra = {}
    # end-to-end through the public API from pinned host buffers
    if not args.no_e2e:
        host_in = torch.empty(g.cells, dtype=torch.uint8).pin_memory()
        host_out = torch.empty(g.cells, dtype=torch.uint8).pin_memory()
        host_in.copy_(bufs[cur[0]])
        e2e_steps = max(1, min(args.steps, 5))
        g.run_host(host_in, host_out, steps=1)
        torch.cuda.synchronize()
        calls = []
        for _ in range(e2e_steps):   # each call synchronises before it returns
            t0 = time.perf_counter()
            g.run_host(host_in, host_out, steps=1)
            calls.append(time.perf_counter() - t0)
        dt = statistics.median(calls)
        # the host link alone: one pinned copy of the state each way
        dev_tmp = bufs[cur[0]]

        def copy_ms(fn):
            fn()
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t) * 1e3

        h2d_ms = copy_ms(lambda: dev_tmp.copy_(host_in, non_blocking=True))
        d2h_ms = copy_ms(lambda: host_out.copy_(dev_tmp, non_blocking=True))
        extra["e2e"] = {"value": g.cells / dt, "unit": UNIT, "h2d_bytes_per_step": g.cells,
                        "d2h_bytes_per_step": g.cells, "ms_per_step": dt * 1e3,
                        "call": "fractal_run_host (H2D, 1 generation, D2H, sync; chunks of tiles with "
                                "the two copy directions overlapped)",
                        "link_h2d_gbs": g.cells / h2d_ms / 1e6, "link_d2h_gbs": g.cells / d2h_ms / 1e6,
                        "sequential_copies_ms": h2d_ms + d2h_ms,
                        "calls_ms": [c * 1e3 for c in calls], "timing": "median of the individually timed calls"}
        del host_in, host_out
    del a, b, bufs
    g.close()
    torch.cuda.empty_cache()

    # the maps alone, CUDA cores vs tensor cores
    if not args.no_maps and rank == 0:
        extra["maps"] = maps_compare(args, W)
    # compact vs bounding box at equal r
    if not args.no_bb and rank == 0:
        extra["bb_compare"] = bb_compare(args, W)
    # the other NBB fractals of the paper's Table 1 workloads
    if not args.no_others and rank == 0:
        extra["other_fractals"] = others_compare(args, W)
    # many uneven instances: batched graph vs one instance per launch
    if not args.no_batch and rank == 0:
        extra["batched"] = batched_compare(args, W)
    # open-loop Poisson requests: continuous-batching server vs one request at a time
    if not args.no_serve and rank == 0:
        extra["served"] = serve_compare(args, W)

    gpu_launches = args.steps  # one step-kernel launch per generation
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": dict(workload_config(inst), parallelism=f"replicas{world}"),
            "roofline": roof, "gpu_launches": gpu_launches}
    cs = clocks.summary()
    line["clocks"] = cs
    line.update(extra)
    return line


def run_sharded(args, rank, world, dist):
    """One triangle instance of level --r split over the N ranks (one shard
    per GPU, contiguous tile ranges): each generation every rank gathers the
    tiles its peers need, exchanges them with NCCL send/recv straight into the
    peers' halo regions, and steps its own tiles.  Strong scaling: the
    instance is the same at every N."""
    import torch
    from paper_2110_12952_gb300 import Fractal, build, workloads as W
    from paper_2110_12952_gb300.shard import ShardPlan, exchange_dist

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    inst = W.TRI_R20 if args.r == 20 else W.Instance(W.TRIANGLE, args.r, 0.3, 3, 1000)
    fam, L = inst.family, args.shard_tile_levels
    g = Fractal.from_family(fam, inst.r)
    plan = ShardPlan.from_family(fam, inst.r, L, world, rank)
    plan.attach(g)
    a = torch.zeros(plan.buffer_cells, dtype=torch.uint8, device=dev)
    full = g.init_bernoulli(inst.seed, inst.p)         # the same instance on every rank
    a[: plan.local_cells].copy_(full[plan.first_cell: plan.first_cell + plan.local_cells])
    del full
    torch.cuda.empty_cache()
    b = torch.zeros_like(a)
    bufs = [a, b]
    cur = [0]
    peers_with_data = sum(1 for q in range(world) if q != rank and len(plan.sends(q)[0]))
    halo_bytes = plan.buffer_cells - plan.local_cells

    def one_generation():
        exchange_dist(plan, bufs[cur[0]], dist)
        plan.step(bufs[cur[0]], bufs[1 - cur[0]])
        cur[0] ^= 1

    with ClockSampler(dev.index) as clocks:
        for _ in range(args.warmup):
            one_generation()
        torch.cuda.synchronize()
        clocks.wait_ready()
        dist.barrier()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t_start = time.monotonic()
        ev0.record(stream)
        for _ in range(args.steps):
            one_generation()
        ev1.record(stream)
        torch.cuda.synchronize()
        t_end = time.monotonic()
    clocks.window(t_start, t_end)
    dist.barrier()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    cells = fam.k ** inst.r
    value = cells * args.steps / (ms_max / 1e3)
    # end to end: the rank's own cells from pinned host memory, one
    # generation (exchange + step), its own cells back, every step
    hin = torch.empty(plan.local_cells, dtype=torch.uint8).pin_memory()
    hout = torch.empty(plan.local_cells, dtype=torch.uint8).pin_memory()
    hin.copy_(bufs[cur[0]][: plan.local_cells])
    e2e_steps = max(1, min(args.steps, 5))
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bufs[cur[0]][: plan.local_cells].copy_(hin, non_blocking=True)
        one_generation()
        hout.copy_(bufs[cur[0]][: plan.local_cells], non_blocking=True)
        torch.cuda.synchronize()
    dt = torch.tensor([(time.perf_counter() - t0) / e2e_steps], dtype=torch.float64, device=dev)
    dist.all_reduce(dt, op=dist.ReduceOp.MAX)
    e2e = {"value": cells / float(dt.item()), "unit": UNIT, "h2d_bytes_per_step": plan.local_cells,
           "d2h_bytes_per_step": plan.local_cells, "ms_per_step": float(dt.item()) * 1e3,
           "call": "per rank: own cells H2D, halo exchange + fractal_shard_step, own cells D2H, sync",
           "bytes_note": "per rank; every rank moves its own cells"}
    peak, peak_src = measured_peak()
    per_rank_alg = 2.0 * plan.local_cells
    achieved = per_rank_alg / (ms / args.steps / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": dict(workload_config(inst), parallelism=f"shards{world}", tile_levels=L,
                           halo_bytes_per_rank=halo_bytes, own_cells_rank0=plan.local_cells),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "step_tma_kernel<2,10,false> over the shard's tiles (rank 0) plus its halo gathers",
                         "algorithmic_bytes_per_launch": per_rank_alg, "peak_source": peak_src},
            "gpu_launches": args.steps * (1 + peers_with_data), "e2e": e2e}
    line["clocks"] = clocks.summary()
    plan.close()
    g.close()
    return line


def maps_compare(args, W):
    """The maps alone (the batch API): lambda of 2^25 seeded compact indices
    of the triangle at r = 20 and nu / compact coordinate of their
    coordinates, on the CUDA cores (fractal_lambda, fractal_nu + fractal_nu2d)
    and with the level sums on the tensor cores (fractal_lambda_tc,
    fractal_nu_tc).  Inputs are resident; the median of 10 timed calls each."""
    import torch
    from paper_2110_12952_gb300 import Fractal
    g = Fractal.from_family(W.TRIANGLE, 20)
    n = 1 << 25
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    w = torch.randint(0, g.cells, (n,), dtype=torch.int64, device="cuda", generator=gen)
    c = g.lam(w)
    out = {}
    for name, fn in (("lambda_cuda_core", lambda: g.lam(w, out=c)),
                     ("lambda_tensor_core", lambda: g.lam_tc(w, out=c)),
                     ("nu_and_compact_cuda_core", lambda: (g.nu(c), g.nu2d(c))),
                     ("nu_and_compact_tensor_core", lambda: g.nu_tc(c, compact=True))):
        ms = statistics.median(time_steps(fn, 10, 3))
        out[name] = {"ms": ms, "maps_per_s": n / (ms / 1e3)}
    same = torch.equal(g.lam_tc(w), g.lam(w))
    om, c2 = g.nu_tc(c, compact=True)
    same = same and torch.equal(om, g.nu(c)) and torch.equal(c2, g.nu2d(c))
    out["workload"] = "triangle r=20, 2^25 uniform compact indices (seed 11) and their coordinates"
    out["tensor_core_equals_cuda_core"] = bool(same)
    del w, c
    g.close()
    torch.cuda.empty_cache()
    return out


def bb_compare(args, W):
    import torch
    from paper_2110_12952_gb300 import Fractal
    r = args.bb_r
    inst = W.Instance(W.TRIANGLE, r, 0.3, 2, 1000)
    g = Fractal.from_family(inst.family, r)
    peak, _ = measured_peak()
    flush_buf = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")

    def flush():
        flush_buf.fill_(1)

    st = g.init_bernoulli(inst.seed, inst.p)
    out = torch.empty_like(st)
    g.autotune(st, out)
    n = max(5, min(args.steps, 20))
    ct = time_steps(lambda: g.step(st, out=out, steps=1), n, 3, flush=flush)
    box = g.scatter(st)
    box_out = torch.empty_like(box)
    bt = time_steps(lambda: g.bb_step(box, out=box_out, steps=1), n, 3)
    c_ms, b_ms = statistics.median(ct), statistics.median(bt)
    # the paper's own approaches at the same level (Sec. 4): lambda(omega) on
    # the box and nu(omega) on blocked rho x rho storage, rho = 2 .. 32
    paper = {}
    for l in range(1, 6):
        rho = 2 ** l
        lt = time_steps(lambda: g.lambda_box_step(box, l, out=box_out, steps=1), max(3, n // 2), 2)
        blk = g.blocked_pack(st, l)
        blk_out = torch.empty_like(blk)
        kt = time_steps(lambda: g.blocked_step(blk, l, out=blk_out, steps=1), max(3, n // 2), 2,
                        flush=flush if 2 * blk.numel() < 4 * 129 * 2**20 else None)
        lm, km = statistics.median(lt), statistics.median(kt)
        paper[f"rho{rho}"] = {"lambda_box_ms": lm, "blocked_nu_ms": km, "blocked_bytes": blk.numel(),
                              "speedup_vs_bb_lambda": b_ms / lm, "speedup_vs_bb_blocked_nu": b_ms / km}
        del blk, blk_out
    res = {"workload": f"sierpinski_triangle_F32_r{r}", "cells": g.cells, "box_cells": g.box_cells,
           "compact_updates_per_s": g.cells / (c_ms / 1e3),
           "compact_ms_per_generation": c_ms,
           "compact_hbm_frac": 2.0 * g.cells / (c_ms / 1e3) / 1e9 / peak,
           "compact_note": "state 43 MB per buffer fits in L2; L2 flushed (512 MB write) before each timed generation",
           "bb_ms_per_generation": b_ms,
           "bb_compact_updates_per_s": g.cells / (b_ms / 1e3),
           "bb_box_updates_per_s": g.box_cells / (b_ms / 1e3),
           "bb_hbm_frac": 2.0 * g.box_cells / (b_ms / 1e3) / 1e9 / peak,
           "speedup_compact_vs_bb": b_ms / c_ms,
           "memory_ratio_bb_vs_compact": g.box_cells / g.cells,
           "generations_timed": n,
           "paper_approaches": paper,
           "paper_approaches_note": "lambda_box: the paper's lambda(omega) (box storage, compact grid of "
                                    "rho x rho blocks); blocked_nu: its nu(omega) on blocked rho x rho storage "
                                    "(mini box staged in shared memory, maps per block); speedups vs this BB kernel"}
    del st, out, box, box_out, flush_buf
    g.close()
    torch.cuda.empty_cache()
    return res


def batched_compare(args, W):
    """4096 uneven independent instances (triangle r 6..14, carpet r 3..8,
    Vicsek r 3..9, p ~ U[0.2, 0.6], seeds from master seed 7), 200 generations
    each: the batched graph-replayed run against the loop of one
    fractal_step call per instance."""
    import torch
    from paper_2110_12952_gb300 import Batch, Fractal
    mix = W.batched_mix(args.batch_instances, master_seed=7, steps=args.batch_steps)
    handles = {}
    states = []
    for inst in mix:
        key = (inst.family.name, inst.r)
        if key not in handles:
            handles[key] = Fractal.from_family(inst.family, inst.r)
        g = handles[key]
        x = g.init_bernoulli(inst.seed, inst.p)
        states.append((g, x, torch.empty_like(x)))
    for g in handles.values():   # tile depth per fractal and level (untimed)
        x = g.init_bernoulli(1, 0.5)
        g.autotune(x, torch.empty_like(x))
        del x
    batch = Batch()
    for (g, x, y), inst in zip(states, mix):
        batch.add(g, x, y, inst.steps)
    batch.run()                    # builds tables and graph; untimed
    for g in handles.values():     # the plain path's scratch buffers; untimed
        x = g.init_bernoulli(1, 0.5)
        g.step(x, steps=2)
        del x
    torch.cuda.synchronize()
    updates, launches = batch.stats()
    st = torch.cuda.current_stream()
    # one timed run of each path, after its untimed warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    batch.run()
    e1.record(st)
    e1.synchronize()
    best_b = e0.elapsed_time(e1)
    ref = [y.clone() for (_, _, y) in states[:64]]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(st)
    for (g, x, y), inst in zip(states, mix):
        g.step(x, out=y, steps=inst.steps)
    e1.record(st)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    plain_wall = time.perf_counter() - t0
    same = all(torch.equal(a, y) for a, (_, _, y) in zip(ref, states[:64]))
    total_cells = sum(i.cells for i in mix)
    res = {"workload": f"{len(mix)} instances (triangle r6-14, carpet r3-8, vicsek r3-9), "
                       f"{args.batch_steps} generations each, master seed 7",
           "total_cells": total_cells, "cell_updates": updates,
           "batched_ms": best_b, "batched_updates_per_s": updates / (best_b / 1e3),
           "timing": "one run of each path after an untimed warm-up of each",
           "batched_launches_in_graph": launches, "graph_launches_per_run": 1,
           "plain_ms": plain_ms, "plain_wall_s": plain_wall,
           "plain_updates_per_s": updates / (plain_ms / 1e3),
           "plain_launches": sum(i.steps for i in mix),
           "speedup_batched_vs_plain": plain_ms / best_b,
           "batched_equals_plain_on_sample": bool(same)}
    batch.close()
    del states, ref
    for g in handles.values():
        g.close()
    torch.cuda.empty_cache()
    return res


def temporal_compare(g, x, y, single_ms, peak):
    """Temporal blocking on the carpet: one pass = 9 generations
    (fractal_set_temporal_blocking(9), automatic tile depth).  Bytes per
    update are reported next to the 2-byte single-generation figure: per
    tile of k^L cells a pass reads the tile and the level-2 units of the
    neighbouring tiles that touch it, and writes the tile."""
    gens = 9
    g.set_temporal_blocking(gens)
    times = time_steps(lambda: g.step(x, out=y, steps=gens), 10, 3)
    g.set_temporal_blocking(0)
    ms = statistics.median(times)
    L = next(l for l in range(5, 1, -1) if l <= g.r and _tb_smem(l) <= 100 * 1024)
    tile = 8 ** L
    halo_units = 4 * 3 ** (L - 2) + 4
    bytes_per_pass = g.cells // tile * (2 * tile + 64 * halo_units)
    return {"generations_per_pass": gens, "tile_levels": L, "ms_per_pass": ms,
            "updates_per_s": g.cells * gens / (ms / 1e3),
            "speedup_vs_single_generation": single_ms * gens / ms,
            "hbm_bytes_per_update": bytes_per_pass / (g.cells * gens),
            "achieved_gbs": bytes_per_pass / (ms / 1e3) / 1e9, "peak_gbs": peak,
            "note": "bytes per update are (tile + halo units + tile) / (cells x generations); "
                    "the roofline of single generations is 2 B per update"}


def multigen_compare(g, x, y, ms_single, gens=50):
    """One call of `gens` generations (bit3 policy: the state stays bit-packed
    between the first and the last generation), timed three times."""
    import torch
    g.step(x, out=y, steps=gens)
    ts = time_steps(lambda: g.step(x, out=y, steps=gens), 3, 1)
    ms = statistics.median(ts)
    return {"generations_per_call": gens, "ms_per_call": ms, "ms_per_generation": ms / gens,
            "updates_per_s": g.cells * gens / (ms / 1e3), "speedup_vs_single_generation": ms_single / (ms / gens),
            "note": "first generation bytes -> bit-packed tile states, the ones between states -> states, "
                    "the last states -> bytes; per-generation bytes are not comparable with the 2 B/update roofline"}


def _tb_smem(L):
    # shared memory of the temporal-blocking plan at tile depth L (carpet)
    r16 = lambda v: (v + 15) // 16 * 16
    nus = 3 ** (L - 2)
    W_ = 9 * nus + 18
    RS = (W_ + 31) // 32 + 2
    nring = 4 * nus + 4
    off = r16(8 ** L)
    off = r16(off + 64 * nring + 4)
    off = r16(off + nring + 4)
    return off + 3 * r16(4 * W_ * RS)


def others_compare(args, W):
    """Carpet r=10, Vicsek r=12, Menger r=6 and r=7 (p 0.5, seeds 4-7; Menger
    B5/S45): one generation per timed step after autotuning the tile depth;
    states smaller than L2 are timed with an L2 flush before each generation.
    Bounding boxes of up to 16 GiB (carpet r=10, Menger r=6 and r=7) are
    timed too."""
    import torch
    from paper_2110_12952_gb300 import Fractal
    peak, _ = measured_peak()
    flush_buf = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")
    out = {}
    for inst in (W.CARPET_R10, W.VICSEK_R12, W.MENGER_R6, W.MENGER_R7):
        g = Fractal.from_family(inst.family, inst.r)
        x = g.init_bernoulli(inst.seed, inst.p)
        y = torch.empty_like(x)
        L = g.autotune(x, y)
        small = 2 * g.cells < 4 * 129 * 2**20
        n = max(5, min(args.steps, 20))
        ct = time_steps(lambda: g.step(x, out=y, steps=1), n, 3,
                        flush=(lambda: flush_buf.fill_(1)) if small else None)
        ms = statistics.median(ct)
        res = {"cells": g.cells, "tile_levels": L, "ms_per_generation": ms,
               "updates_per_s": g.cells / (ms / 1e3), "hbm_frac": 2.0 * g.cells / (ms / 1e3) / 1e9 / peak,
               "l2_flush": small}
        if inst.family.name == "carpet":
            res["temporal_blocking"] = temporal_compare(g, x, y, ms, peak)
        if inst.family.name == "menger":
            res["bit_packed_generations"] = multigen_compare(g, x, y, ms)
        if g.box_cells <= 16 * 2**30:
            box = g.scatter(x)
            del x, y
            bo = torch.empty_like(box)
            bt = time_steps(lambda: g.bb_step(box, out=bo, steps=1), max(3, n // 2), 2)
            bms = statistics.median(bt)
            res.update({"bb_box_cells": g.box_cells, "bb_ms_per_generation": bms,
                        "bb_hbm_frac": 2.0 * g.box_cells / (bms / 1e3) / 1e9 / peak,
                        "speedup_compact_vs_bb": bms / ms})
            del box, bo
        out[f"{inst.family.name}_r{inst.r}"] = res
        g.close()
        torch.cuda.empty_cache()
    del flush_buf
    return out


def _pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def serve_compare(args, W):
    """Poisson arrivals (mean --serve-rate req/s for --serve-seconds, master
    seed 8; family uniform over triangle/carpet/Vicsek, r uniform in the
    batched ranges, generations log-uniform in [10, 1000], p ~ U[0.2, 0.6]),
    results reduced to live-cell counts.  The server (continuous batching)
    serves the whole trace; the plain path (one request at a time through
    fractal_step on one stream, FIFO) serves its first --serve-plain-requests
    requests."""
    import torch
    from paper_2110_12952_gb300 import Fractal, Server
    trace = W.poisson_trace(rate_per_s=args.serve_rate, duration_s=args.serve_seconds, master_seed=8)
    handles = {}
    for q in trace:
        key = (q.instance.family.name, q.instance.r)
        if key not in handles:
            handles[key] = Fractal.from_family(q.instance.family, q.instance.r)
    for g in handles.values():     # tables and tile depth before the clock starts
        x = g.init_bernoulli(1, 0.5)
        g.autotune(x, torch.empty_like(x))
        del x
    torch.cuda.synchronize()
    offered = sum(q.instance.cells * q.instance.steps for q in trace)
    srv = Server(hbm_budget_bytes=0, chunk=args.serve_chunk)
    ids = []
    t0 = time.perf_counter()
    t_srv0 = t0
    for q in trace:
        dt = t0 + q.arrival_s - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        i = q.instance
        ids.append(srv.submit(handles[(i.family.name, i.r)], i.seed, i.p, i.steps))
    srv.wait_all()
    t_end = time.perf_counter()
    lats = [srv.poll(rid)[1] for rid in ids]
    st = srv.stats()
    srv.close()
    # plain path on the head of the same trace
    head = trace[: args.serve_plain_requests]
    plain = []
    t0 = time.perf_counter()
    for q in head:
        dt = t0 + q.arrival_s - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        i = q.instance
        g = handles[(i.family.name, i.r)]
        x = g.init_bernoulli(i.seed, i.p)
        y = g.step(x, steps=i.steps)
        int(torch.count_nonzero(y).item())
        plain.append(time.perf_counter() - (t0 + q.arrival_s))
    plain_span = time.perf_counter() - t0
    head_updates = sum(q.instance.cells * q.instance.steps for q in head)
    for g in handles.values():
        g.close()
    torch.cuda.empty_cache()
    served_span = t_end - t_srv0
    return {"workload": f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g} s "
                        f"({len(trace)} requests), master seed 8, results reduced to live-cell counts",
            "requests": len(trace), "offered_updates_per_s": offered / args.serve_seconds,
            "served_updates": st["cell_updates"],
            "served_span_s": served_span,
            "served_updates_per_s": st["cell_updates"] / served_span,
            "served_p50_s": _pct(lats, 50), "served_p99_s": _pct(lats, 99),
            "served_mean_s": sum(lats) / len(lats), "served_launches": st["launches"],
            "chunk": args.serve_chunk,
            "plain_requests": len(head), "plain_p50_s": _pct(plain, 50), "plain_p99_s": _pct(plain, 99),
            "plain_updates_per_s": head_updates / plain_span}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.maps_only:
        import torch
        from paper_2110_12952_gb300 import build, workloads as W
        build.build()
        print(json.dumps({"maps": maps_compare(args, W)}), flush=True)
        return
    sharded = args.shard or (world > 1 and not args.replicas)
    if world > 1 or sharded:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if world == 1:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29533")
            os.environ.setdefault("RANK", "0")
            os.environ.setdefault("WORLD_SIZE", "1")
        tdist.init_process_group("nccl")
        dist = tdist
    if sharded:
        line = run_sharded(args, rank, world, dist)
    else:
        line = run_ours(args, rank, world, dist)
    if rank == 0:
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args.r, args.cpu_seconds, 3, 0.3)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
