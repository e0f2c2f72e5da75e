#!/usr/bin/env python
"""Benchmark of the cell-based Voronoi hot path on GB300.

Workload (the 3D metric's configuration): 1,000,000 points uniform i.i.d. in
a periodic cube of side 100 (unit density, seed 1), 58^3 blocks.  One step is
the whole hot path on one batch, replayed as one captured CUDA graph
(vg_graph_capture / vg_graph_launch): counting sort of the device-resident
points into blocks, the cell kernels (FP32 cuts with FP64 re-test,
sorted-distance prefetch), and the CSR compaction of the faces.  L2 is
flushed between steps (a 256 MB write outside the timed events).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank processes its own
1M-point system (weak scaling, no collective on the data path); value is the
cells of all ranks over the slowest rank's time.

--impl reference times the FP64 CPU oracle (block-grid walk with the radius
bound, OpenMP over cells) on this host's cores, on a bounded sample of the
same workload's cells per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D Voronoi cells/s, 1 GB300, chosen vs plain FP64 form; % of roofline"
N_POINTS = 1_000_000
SIDE = 100.0
GRID = (58, 58, 58)
WORKLOAD = ("uniform1m: 1,000,000 points uniform in a periodic cube of side 100 (seed 1), "
            "58^3 blocks; chosen form = FP32 cuts + FP64 re-test, sorted prefetch")
# FP32 peak derived from unit counts and clock: 152 SMs x 128 FP32 lanes x
# 2 FLOP (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic FLOP counts per unit of work (see the design notes)
FLOP_VTEST, FLOP_CAND, FLOP_NEWV, FLOP_FANTET = 6, 12, 51, 42


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    return ap.parse_args()


def workload(rank: int):
    from paper_2209_11606_gb300 import workloads as W
    return W.uniform(N_POINTS, 3, SIDE, True, seed=1 + rank)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def batched_run(V, torch, stream, flush, steps: int = 5, seed: int = 5):
    """The 256-system batched workload: one container, one graph replay per
    step (one sort over all systems' blocks, one persistent cell launch)."""
    from paper_2209_11606_gb300 import workloads as W
    systems = W.batched_systems(256, 1000, 200_000, seed=seed)
    descs = [V.vg_system(x.lo, x.hi, x.periodic) for x in systems]
    counts = [x.n for x in systems]
    pos = torch.from_numpy(np.concatenate([x.pos for x in systems])).cuda()
    ctx = V.vg_batch_create(3, descs, stream=stream)
    try:
        cfg = V.vg_config_default()
        V.vg_graph_capture(ctx, counts, pos, None, cfg)
        for _ in range(3):
            V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            V.vg_graph_launch(ctx)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        V.vg_graph_sync(ctx)
        ms = [a.elapsed_time(b) for a, b in evs]
        n = int(sum(counts))
        kinds = {}
        for x in systems:
            kinds[x.tag] = kinds.get(x.tag, 0) + 1
        return {"value": n * steps / (sum(ms) / 1000.0), "unit": "cells/s", "steps": steps,
                "ms_per_step": sum(ms) / steps, "cells_per_step": n, "systems": len(systems),
                "mix": kinds, "form": "FP32 cuts + FP64 re-test, sorted prefetch, one graph replay",
                "workload": "256 3D systems, sizes log-uniform in [1000, 200000], uniform / perturbed "
                            "FCC (sigma 0.05 a) / 50 Gaussian blobs (sigma 0.02 side), random "
                            f"periodicity (seed {seed})"}
    finally:
        V.vg_destroy(ctx)


def cpu_baseline(s, cells: int, seed: int = 0):
    """Times the FP64 oracle on a sample of `cells` cells of system s."""
    import oracle
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(s.n, size=min(cells, s.n), replace=False))
    oracle.build()
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=GRID, cells=sample,
                   threads=threads)
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": "cells/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(sample)} random cells of the 1M-point workload (FP64 block-grid "
                      f"walk with the radius bound, OpenMP dynamic over cells)",
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    s = workload(0)
    per_step = 100_000
    for _ in range(args.warmup):
        cpu_baseline(s, 20_000, seed=99)
    total, cells = 0.0, 0
    res = None
    for k in range(args.steps):
        res = cpu_baseline(s, per_step, seed=k)
        total += res["seconds"]
        cells += per_step
    v = cells / total
    line = {"metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD.replace("chosen form = FP32 cuts + FP64 re-test, sorted prefetch",
                                                    "FP64 CPU oracle")},
            "cpu_baseline": {"value": v, "unit": "cells/s", "kind": "oracle", "cores": res["cores"],
                             "sample": f"{per_step} random cells per step of the 1M-point workload"},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2209_11606_gb300 import build as B
    B.build()
    from paper_2209_11606_gb300 import vorogpu as V

    s = workload(rank)
    n = s.n
    stream = torch.cuda.current_stream()
    pos_d = torch.from_numpy(s.pos).cuda()
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, GRID, stream=stream)
    cfg = V.vg_config_default()
    cfg.precision = V.VG_FP32_RETEST
    cfg.order = V.VG_PREFETCH
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step():
        V.vg_insert(ctx, pos_d)
        V.vg_compute(ctx, cfg)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the step as one graph: sort -> cells -> faces, cell kernels timed by
    # event nodes inside the graph
    gcfg = V.vg_config_default()
    gcfg.precision, gcfg.order, gcfg.time_kernels = cfg.precision, cfg.order, 1
    V.vg_graph_capture(ctx, [n], pos_d, None, gcfg)
    for _ in range(max(args.warmup, 3)):
        V.vg_graph_launch(ctx)
    V.vg_graph_sync(ctx)

    # ---- timed region: K steps, L2 flushed between them ----------------------
    V.vg_get_kernel_ms(ctx)  # reset
    l0 = V.vg_get_launches(ctx)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        V.vg_graph_launch(ctx)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    V.vg_graph_sync(ctx)  # input flags and face capacity of the replays
    launches = V.vg_get_launches(ctx) - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    kern_ms, kern_n = V.vg_get_kernel_ms(ctx)
    t_total = sum(step_ms) / 1000.0
    if dist:
        t = torch.tensor([t_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
        dist.barrier()
    value = world * n * args.steps / t_total

    if rank != 0:
        V.vg_destroy(ctx)
        if dist:
            dist.destroy_process_group()
        return

    # ---- work counters -> algorithmic FLOPs of the cell kernels ----------------
    cfg.collect_stats = 1
    step()
    cfg.collect_stats = 0
    w = {k: np.zeros(n, np.int32) for k in ("t", "v", "c", "nv", "r")}
    fb = np.zeros(n, np.uint8)
    V.vg_get_work(ctx, w["t"], w["v"], w["c"], w["nv"], w["r"], fb)
    ne = np.zeros(n, np.int32)
    nf = np.zeros(n, np.int32)
    st = np.zeros(n, np.uint8)
    V.vg_get_cells(ctx, ne=ne, nf=nf, status=st)
    fan = 2 * ne.astype(np.int64) - 2 * nf.astype(np.int64)
    flop = (FLOP_VTEST * w["v"].astype(np.int64).sum() + FLOP_CAND * w["t"].astype(np.int64).sum() +
            FLOP_NEWV * w["nv"].astype(np.int64).sum() + FLOP_FANTET * fan.sum())
    kern_avg_ms = kern_ms / max(kern_n, 1)
    achieved = flop / (kern_avg_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_cells3<float> (cell kernel phase)", "kernel_ms": kern_avg_ms,
            "flop_per_cell": flop / n,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    # ---- the plain FP64 form on the same input (the metric's comparison) -------
    cfg64 = V.vg_config_default()
    cfg64.precision = V.VG_FP64
    cfg64.order = V.VG_WALK
    V.vg_insert(ctx, pos_d)
    V.vg_compute(ctx, cfg64)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot64 = 0.0
    for k in range(reps):
        flush.fill_(k)
        e0.record(stream)
        V.vg_insert(ctx, pos_d)
        V.vg_compute(ctx, cfg64)
        e1.record(stream)
        torch.cuda.synchronize()
        tot64 += e0.elapsed_time(e1) / 1000.0
    plain64 = n * reps / tot64

    # ---- end to end through the public API, host buffers -----------------------
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(s.pos).pin_memory().numpy()
        outs = {"vol": np.float64, "area": np.float64, "nv": np.int32, "ne": np.int32,
                "nf": np.int32, "status": np.uint8}
        host = {k: torch.empty(n, dtype=getattr(torch, np.dtype(t).name)).pin_memory().numpy()
                for k, t in outs.items()}
        cen = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        _, nface = V.vg_get_counts(ctx)
        fo = torch.empty(n + 1, dtype=torch.int64).pin_memory().numpy()
        cap = int(nface * 1.2) + 1024
        ids = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
        img = torch.empty((cap, 3), dtype=torch.int8).pin_memory().numpy()
        fod = torch.empty(cap, dtype=torch.uint8).pin_memory().numpy()
        d2h = 0
        reps = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(reps):
            V.vg_insert(ctx, pos_h)
            V.vg_compute(ctx, cfg)
            _, nface = V.vg_get_counts(ctx)
            V.vg_get_cells(ctx, host["vol"], host["area"], cen, host["nv"], host["ne"], host["nf"],
                           host["status"])
            V.vg_get_faces(ctx, fo, ids[:nface], img[:nface], fod[:nface])
        dt = time.perf_counter() - t0
        d2h = (n * (8 + 8 + 24 + 4 + 4 + 4 + 1) + (n + 1) * 8 + nface * (4 + 3 + 1))
        e2e = {"value": n * reps / dt, "unit": "cells/s", "h2d_bytes_per_step": int(n * 3 * 8),
               "d2h_bytes_per_step": int(d2h)}

    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells_per_step": n * world,
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas{world}"},
            "roofline": roof,
            "step": "one CUDA graph replay: counting sort, cell kernels (3 capacity tiers), face CSR",
            "plain_fp64": {"value": plain64, "unit": "cells/s",
                           "form": "FP64 everywhere, block walk (Sec. 2.1.3)"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "fallback_rate": float(fb.mean()), "retest_per_cell": float(w["r"].mean())}
    if not args.no_batched:
        line["batched"] = batched_run(V, torch, stream, flush)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(s, 100_000).items() if k != "seconds"}
    V.vg_destroy(ctx)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
