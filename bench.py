#!/usr/bin/env python
"""Benchmark of the cell-based Voronoi hot path on GB300.

Default workload (the 3D metric's configuration): 1,000,000 points uniform
i.i.d. in a periodic cube of side 100 (unit density, seed 1), 58^3 blocks.
One step is the whole hot path on one batch, replayed as one captured CUDA
graph (vg_graph_capture / vg_graph_launch): counting sort of the
device-resident points into blocks, the learned per-block preload targets,
the cell kernels (FP32 cuts with FP64 re-test, distance-sorted preload), and
the CSR compaction of the faces.  L2 is flushed between steps (a 256 MB write
outside the timed events).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--split 0|1] [--grid N] [--weinberg]

With N > 1 (torchrun, one rank per GPU) every rank processes its own system
(weak scaling, no collective on the data path); value is the cells of all
ranks over the slowest rank's time.

--workload selects another configuration (no e2e and no batched line there):
slabs102m, the 102.4M-point periodic cube of alternating perturbed-FCC and
uniform slabs; radical2m, 2M radical (power) cells; hex10m, 10M 2D cells;
the paper's cases of Sec. 3.1 in the walled unit cube or square
(homog3d, local3d, local3d_clip, extreme3d, homog2d, local2d, extreme2d);
vorotop102m, 102.4M uniform points in the periodic unit cube (with
--weinberg, VoroTop's case: cells with Weinberg codes).

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
WORKLOADS = {
    "uniform1m": ("uniform1m: 1,000,000 points uniform in a periodic cube of side 100 (seed 1), 58^3 blocks; "
                  "chosen form = FP32 cuts + FP64 re-test, learned distance-sorted preload"),
    "slabs102m": ("slabs102m: 102,400,000 points in a periodic cube of side 296 a (a = 51/32), 8 z-slabs "
                  "alternating perturbed FCC (sigma 0.05 a) and uniform points (seed 6), blocks by the "
                  "n_opt = 4.6 rule; chosen form = FP32 cuts + FP64 re-test, learned distance-sorted preload"),
    "radical2m": ("radical2m: 2,000,000 points uniform in a periodic cube (unit density, seed 4), radii "
                  "log-normal (sigma 0.3) scaled to packing fraction 0.4, blocks by the n_opt = 4.6 rule; "
                  "chosen form = FP32 cuts + FP64 re-test, block walk"),
    "hex10m": ("hex10m: 2D, 10,000,314 points of a perturbed hexagonal lattice (2943 x 3398, sigma 0.05 of the "
               "column spacing, seed 3) in the periodic unit square, blocks by the n_opt = 3.4 rule; "
               "chosen form = FP32 cuts + FP64 re-test, block walk"),
    # the three example cases of Sec. 3.1 (walled unit cube, N = 10^8, grids of
    # Table 3) and the clipped cells of Sec. 3.1.3
    "homog3d": ("homog3d: 10^8 points uniform in the walled unit cube (seed 11), 279^3 blocks (Table 3, "
                "n_opt 4.6); chosen form = FP32 cuts + FP64 re-test, distance-sorted preload (72)"),
    "local3d": ("local3d: the 9,999,326 of 10^8 uniform points (seed 12) inside the central cube of volume 0.1, "
                "walled unit cube, 126^3 blocks (Table 3, n_opt 49); chosen form = FP32 cuts + FP64 re-test, "
                "distance-sorted preload (72), block bound beyond the near shells"),
    "local3d_clip": ("local3d_clip: local3d with every cell clipped by the cube of side 1.5 sqrt(3) d0, "
                     "d0 = (10^8)^(-1/3) (Sec. 3.1.3); chosen form as local3d"),
    "extreme3d": ("extreme3d: 10^8 points, each coordinate 1/2 + 4 (X - 1/2)^3 (seed 13), walled unit cube, "
                  "584^3 blocks (Table 3, n_opt 0.5); chosen form = FP32 cuts + FP64 re-test, "
                  "distance-sorted preload (72)"),
    # VoroTop's case (Sec. 4): cells with Weinberg codes (run with --weinberg)
    "vorotop102m": ("vorotop102m: 102,400,000 points uniform in the periodic unit cube (seed 17), blocks by the "
                    "n_opt = 4.6 rule; chosen form = FP32 cuts + FP64 re-test, distance-sorted preload (72)"),
    # the same three cases in 2D (Table 3 grids)
    "homog2d": ("homog2d: 10^8 points uniform in the walled unit square (seed 14), 5423^2 blocks (Table 3, "
                "n_opt 3.4); chosen form = FP32 cuts + FP64 re-test, block walk"),
    "local2d": ("local2d: the points of 10^8 uniform ones (seed 15) inside the central square of area 0.1, "
                "walled unit square, 1825^2 blocks (Table 3, n_opt 30); chosen form = FP32 cuts + FP64 "
                "re-test, block walk"),
    "extreme2d": ("extreme2d: 10^8 points, each coordinate 1/2 + 4 (X - 1/2)^3 (seed 16), walled unit square, "
                  "14142^2 blocks (Table 3, n_opt 0.5); chosen form = FP32 cuts + FP64 re-test, block walk"),
}
PAPER3D = ("homog3d", "local3d", "local3d_clip", "extreme3d")
PAPER2D = ("homog2d", "local2d", "extreme2d")
METRIC_2D = "2D Voronoi cells/s, 1 GB300, chosen vs plain FP64 form; % of roofline"
# FP32 peak derived from unit counts and clock: 152 SMs x 128 FP32 lanes x
# 2 FLOP (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# GB300's nominal dense FP64 rate (its FP64 units are few; no measured peak)
FP64_PEAK_TFLOPS = 1.25
# algorithmic FLOP per unit of work: a vertex tested against a plane (3 FMA),
# a candidate (offset, |q|^2, plane constant), a new vertex (Cramer's rule on
# three planes), a fan tetrahedron of the statistics (determinant, centroid,
# vector area)
FLOP_VTEST, FLOP_CAND, FLOP_NEWV, FLOP_FANTET = 6, 12, 51, 42
# Counters of the tier-0 FP32 cell kernel from one ncu capture of the
# bench's own workload (profiles/), per workload: DRAM bytes (read + write)
# of one launch, warp instructions per cell, active lanes per instruction,
# issue-active fraction.  An entry is removed whenever the kernel changes
# after its capture, so only counters of the timed build are reported.
CELL_KERNEL_NCU = {
    "uniform1m": {"dram_bytes": 201944576 + 297465856, "warp_inst_per_cell": 12347.4, "lanes_per_inst": 23.26,
                  "issue_active": 0.606, "kernel": "k_cells3<float,2,64,...,HOT> (hot kernel)",
                  "source": "profiles/k_cells3_hot_fp32_uniform1m_ncu.md"},
    "hex10m": {"dram_bytes": 594627584 + 1095686144, "warp_inst_per_cell": 3478.1, "lanes_per_inst": 14.39,
               "issue_active": 0.388, "kernel": "k_cells2<float,8,16> (2D tier 0)",
               "source": "profiles/k_cells2_fp32_hex10m_ncu.md"},
}
MLP_ALPHA, MLP_KMIN, MLP_KMAX = 1.2, 24.0, 1024.0
# peak warp-instruction issue rate: 152 SMs x 4 schedulers x 1 per cycle x 2.07 GHz
ISSUE_PEAK = 152 * 4 * 2.07e9
# algorithmic bytes of the counting sort per particle (FP64 input): read the
# position (24), the block-count atomic (4), write the FP32 offset + radius
# (16) and the input index (4); plus 8 per block for the scan
SORT_BYTES_PER_PARTICLE, SORT_BYTES_PER_BLOCK = 48, 8


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s) and its source."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


PKG = os.path.join(ROOT, "paper_2209_11606_gb300")
MLP_PARAMS = os.path.join(PKG, "mlp_params_gb300.json")
TUNE_CACHE = os.path.join(PKG, "tuned_gb300.json")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform1m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the alternative FP32 forms")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 102.4M-point slabs record of the default run")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison of the GPU outputs with the oracle's")
    ap.add_argument("--grid", type=int, default=0,
                    help="blocks per axis instead of the workload's grid (e.g. a tuned grid)")
    ap.add_argument("--split", type=int, default=1, choices=[0, 1],
                    help="FP32 form: 1 = the kernel built for the common path, handing the rest on "
                         "(3D: to the general kernel; 2D: from 16 to 32 vertices a cell), 0 = the general kernel alone")
    ap.add_argument("--weinberg", action="store_true",
                    help="also time the cells with Weinberg codes (Sec. 4), graph replays")
    return ap.parse_args(argv)


def clip_of(name: str) -> float:
    """Cube side of the clipped cells of Sec. 3.1.3 (0: plain cells)."""
    return 1.5 * math.sqrt(3.0) * 1e8 ** (-1.0 / 3.0) if name == "local3d_clip" else 0.0


def workload(name: str, rank: int):
    """(system, block grid or None for the n_opt rule, chosen order, learned preload)."""
    from paper_2209_11606_gb300 import workloads as W
    if name == "homog3d":
        return W.uniform(100_000_000, 3, 1.0, False, seed=11 + rank), (279,) * 3, "prefetch", False
    if name in ("local3d", "local3d_clip"):
        return W.localized(100_000_000, 3, 0.1, seed=12 + rank), (126,) * 3, "prefetch", False
    if name == "extreme3d":
        return W.extreme_clustering(100_000_000, 3, seed=13 + rank), (584,) * 3, "prefetch", False
    if name == "vorotop102m":
        return W.uniform(102_400_000, 3, 1.0, True, seed=17 + rank), None, "prefetch", False
    if name == "homog2d":
        return W.uniform(100_000_000, 2, 1.0, False, seed=14 + rank), (5423,) * 2, "walk", False
    if name == "local2d":
        return W.localized(100_000_000, 2, 0.1, seed=15 + rank), (1825,) * 2, "walk", False
    if name == "extreme2d":
        return W.extreme_clustering(100_000_000, 2, seed=16 + rank), (14142,) * 2, "walk", False
    if name == "uniform1m":
        return W.uniform(1_000_000, 3, 100.0, True, seed=1 + rank), (58, 58, 58), "prefetch", True
    if name == "slabs102m":
        return W.fcc_uniform_slabs(seed=6 + rank), None, "prefetch", True
    if name == "radical2m":
        return W.radical_uniform(2_000_000, 0.4, 0.3, seed=4 + rank), None, "walk", False
    s = W.hexagonal(2943, 3398, (1.0, 1.0), 0.05, seed=3 + rank)
    return s, None, "walk", False


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


def mlp_params(V, torch):
    """The learned preload's parameters: from the file the last training run
    wrote, else trained here on the labels of the 1M-point configuration
    (uniform and perturbed BCC) by the library's training kernels."""
    if os.path.exists(MLP_PARAMS):
        with open(MLP_PARAMS) as f:
            d = json.load(f)
        return np.asarray(d["params"], dtype=np.float32), d["meta"]
    from paper_2209_11606_gb300 import predictor as P, workloads as W
    t0 = time.perf_counter()
    rows = []
    for name in ("uniform1m", "bcc1m"):
        s = W.workload(name)
        rows.append(P.rows_for_system(s, torch, s.meta["grid"]))
    X = torch.cat([r[0] for r in rows])
    t = torch.cat([r[1] for r in rows])
    params, losses = P.train(X, t, torch, seed=0, steps=1500, lr=3e-3, u=4.0)
    meta = {"trained_on": "k* labels of uniform1m and bcc1m (FP32 form)", "rows": int(X.shape[0]),
            "steps": 1500, "lr": 3e-3, "u": 4.0, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "seconds": time.perf_counter() - t0}
    try:
        with open(MLP_PARAMS, "w") as f:
            json.dump({"meta": meta, "params": [float(x) for x in params]}, f)
    except OSError:
        pass
    return params, meta


def graph_steps(V, torch, ctx, stream, flush, steps):
    """Times `steps` graph replays, L2 flushed before each; returns per-step ms."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        V.vg_graph_launch(ctx)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    V.vg_graph_sync(ctx)
    return [a.elapsed_time(b) for a, b in evs]


def batched_run(V, torch, stream, flush, mlp, steps: int = 5, seed: int = 5):
    """The 256-system batched workload: one container, one graph replay per
    step (one sort over all systems' blocks, one persistent cell launch),
    with N_opt per distribution class and the launch parameters, fixed or
    learned preload targets among them, from the autotuner (cached)."""
    from paper_2209_11606_gb300 import autotune as A, workloads as W
    systems = W.batched_systems(256, 1000, 200_000, seed=seed)
    t0 = time.perf_counter()
    cache = A.Cache(TUNE_CACHE)
    key = "batched256-seed%d-perclass" % seed
    tb = cache.get(key)
    if tb is None:
        tb = A.tune_batch(systems, torch, cache, predictor=mlp, mlp_args=(MLP_ALPHA, MLP_KMIN, MLP_KMAX))
        tb = {"n_opt": tb["n_opt"], "launch": tb["launch"], "classes": tb["classes"]}
        cache.put(key, tb)
    tune_s = time.perf_counter() - t0
    descs = [V.vg_system(x.lo, x.hi, x.periodic, n_opt=v) for x, v in zip(systems, tb["n_opt"])]
    counts = [x.n for x in systems]
    pos = torch.from_numpy(np.concatenate([x.pos for x in systems])).cuda()
    ctx = V.vg_batch_create(3, descs, stream=stream)
    hot = tb["launch"].get("hot_classes")
    try:
        cfg = A.config_from(tb["launch"])
        if cfg.use_mlp:
            V.vg_set_predictor(ctx, mlp, MLP_ALPHA, MLP_KMIN, MLP_KMAX)
        if hot is not None:
            for k, c in enumerate(tb["classes"]):
                V.vg_set_system_split(ctx, k, int(c in hot))
        V.vg_graph_capture(ctx, counts, pos, None, cfg)
        for _ in range(3):
            V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        ms = graph_steps(V, torch, ctx, stream, flush, steps)
        n = int(sum(counts))
        mix = {}
        for x in systems:
            mix[x.tag] = mix.get(x.tag, 0) + 1
        per_class = {}
        for c, v in zip(tb["classes"], tb["n_opt"]):
            per_class[c] = v
        # the same launch on each distribution's systems alone: where the
        # batch's time goes
        by_tag = {}
        for tag in sorted(mix):
            idx = [k for k, x in enumerate(systems) if x.tag == tag]
            sub = V.vg_batch_create(3, [descs[k] for k in idx], stream=stream)
            try:
                pos_t = torch.from_numpy(np.concatenate([systems[k].pos for k in idx])).cuda()
                if cfg.use_mlp:
                    V.vg_set_predictor(sub, mlp, MLP_ALPHA, MLP_KMIN, MLP_KMAX)
                if hot is not None:
                    for j, k in enumerate(idx):
                        V.vg_set_system_split(sub, j, int(tb["classes"][k] in hot))
                V.vg_graph_capture(sub, [counts[k] for k in idx], pos_t, None, cfg)
                V.vg_graph_launch(sub)
                V.vg_graph_sync(sub)
                ms_t = graph_steps(V, torch, sub, stream, flush, 3)
                n_t = int(sum(counts[k] for k in idx))
                by_tag[tag] = {"systems": len(idx), "cells": n_t, "ms_per_step": sum(ms_t) / 3,
                               "cells_per_s": n_t * 3 / (sum(ms_t) / 1000.0)}
            finally:
                V.vg_destroy(sub)
        return {"value": n * steps / (sum(ms) / 1000.0), "unit": "cells/s", "steps": steps,
                "ms_per_step": sum(ms) / steps, "cells_per_step": n, "systems": len(systems),
                "mix": mix, "n_opt_by_class": per_class, "by_distribution": by_tag,
                "launch": {k: tb["launch"].get(k, 0) for k in ("order", "warps_per_cta", "chunk", "use_mlp", "split")}
                | ({"hot_classes": hot} if hot is not None else {}),
                "tuning_seconds": tune_s,
                "form": "FP32 cuts + FP64 re-test, autotuned N_opt, launch and preload (fixed or learned), "
                        "one graph replay",
                "workload": "256 3D systems, sizes log-uniform in [1000, 200000], uniform / perturbed "
                            "FCC (sigma 0.05 a) / 50 Gaussian blobs (sigma 0.02 side), random "
                            f"periodicity (seed {seed})"}
    finally:
        V.vg_destroy(ctx)


def large_run(V, torch, stream, flush, mlp, steps: int = 2, with_oracle: bool = True):
    """The 102.4M-point slabs (perturbed FCC and uniform): the chosen form as
    graph replays (sort, learned preload targets, cells, faces) against the
    plain FP64 form (eager insert + compute, CUDA events on the stream), the
    learned preload's fallback rate, and 2000 sampled cells against the
    oracle."""
    s, grid, _, _ = workload("slabs102m", 0)
    n = s.n
    pos_d = torch.from_numpy(s.pos).cuda()
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, grid, stream=stream)
    try:
        V.vg_set_predictor(ctx, mlp, MLP_ALPHA, MLP_KMIN, MLP_KMAX)
        cfg = V.vg_config_default()
        cfg.precision, cfg.order, cfg.use_mlp, cfg.time_kernels = V.VG_FP32_RETEST, V.VG_PREFETCH, 1, 1
        V.vg_graph_capture(ctx, [n], pos_d, None, cfg)
        V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        V.vg_get_kernel_ms(ctx)
        V.vg_get_sort_ms(ctx)
        ms = graph_steps(V, torch, ctx, stream, flush, steps)
        kern_ms, kern_n = V.vg_get_kernel_ms(ctx)
        sort_ms, sort_n = V.vg_get_sort_ms(ctx)
        chosen = n * steps / (sum(ms) / 1000.0)
        got = V._fetch(ctx, n, 3, False) if with_oracle else None
        # the learned preload's fallbacks (work counters of an eager compute)
        c = V.vg_config_default()
        c.precision, c.order, c.use_mlp, c.collect_stats = V.VG_FP32_RETEST, V.VG_PREFETCH, 1, 1
        V.vg_insert(ctx, pos_d)
        V.vg_compute(ctx, c)
        fb = np.zeros(n, np.uint8)
        pref = np.zeros(n, np.int32)
        V.vg_get_work(ctx, fallback=fb, n_prefetch=pref)
        # the plain FP64 form: sort + cells + faces, eager
        c64 = V.vg_config_default()
        c64.precision, c64.order = V.VG_FP64, V.VG_WALK
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        flush.fill_(1)
        e0.record(stream)
        V.vg_insert(ctx, pos_d)
        V.vg_compute(ctx, c64)
        e1.record(stream)
        torch.cuda.synchronize()
        plain = n / (e0.elapsed_time(e1) / 1000.0)
        rec = {"workload": WORKLOADS["slabs102m"], "cells_per_step": n, "steps": steps,
               "value": chosen, "unit": "cells/s", "ms_per_step": sum(ms) / steps,
               "cell_kernel_ms": kern_ms / max(kern_n, 1), "sort_ms": sort_ms / max(sort_n, 1),
               "plain_fp64": {"value": plain, "unit": "cells/s",
                              "form": "FP64 everywhere, block walk, eager insert + compute"},
               "chosen_vs_plain": chosen / plain,
               "learned_preload": {"shortfall_rate": float((fb > 0).mean()), "walk_rate": float((fb == 1).mean()),
                                   "preload_per_cell": float(pref.mean())},
               "form": "FP32 cuts + FP64 re-test, learned distance-sorted preload, graph replays"}
        if with_oracle:
            import oracle
            rng = np.random.default_rng(7)
            cells = np.sort(rng.choice(n, size=2000, replace=False))
            ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=V.vg_get_grid(ctx, 3), cells=cells,
                                 threads=os.cpu_count() or 1)
            rec["accuracy"] = accuracy(got, ref, cells, 1e-5)
        return rec
    finally:
        V.vg_destroy(ctx)
        del pos_d
        torch.cuda.empty_cache()


def weinberg_run(V, torch, ctx, pos_d, rad_d, cfg, n, stream, flush, reps: int = 3):
    """Cells with and without Weinberg codes (Sec. 4): graph replays of sort,
    cells, codes and face CSR, CUDA events, L2 flushed before each."""
    def timed(weinberg):
        c = V.vg_config_default()
        c.precision, c.order, c.use_mlp, c.clip = cfg.precision, cfg.order, cfg.use_mlp, cfg.clip
        c.weinberg = int(weinberg)
        V.vg_graph_capture(ctx, [n], pos_d, rad_d, c)
        V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        ms = graph_steps(V, torch, ctx, stream, flush, reps)
        return n * reps / (sum(ms) / 1000.0)
    base = timed(False)
    with_codes = timed(True)
    wl, wh, ws = np.zeros(n, np.int32), np.zeros(n, np.uint64), np.zeros(n, np.int32)
    V.vg_get_weinberg(ctx, wl, wh, ws)
    coded = wl > 0
    return {"cells_per_s": with_codes, "without_codes_cells_per_s": base, "unit": "cells/s",
            "coded_fraction": float(coded.mean()), "distinct_codes": int(len(np.unique(wh[coded]))),
            "form": "graph replays with cfg.weinberg = 1 (sort, cells keeping their triangles, a warp per "
                    "cell for its Weinberg code, face CSR), CUDA events, L2 flushed"}


def cpu_baseline(s, grid, cells: int, seed: int = 0, clip: float = 0.0):
    """Times the FP64 oracle on a sample of `cells` cells of system s."""
    import oracle
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(s.n, size=min(cells, s.n), replace=False))
    oracle.build()
    threads = os.cpu_count() or 1
    if grid is None:
        grid = oracle.grid_size(s.n, s.lo, s.hi, 4.6 if s.dim == 3 else 3.4)
    t0 = time.perf_counter()
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, method="grid", nblocks=grid,
                         cells=sample, threads=threads, clip=clip)
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": "cells/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(sample)} random cells of the {s.n}-point workload (FP64 block-grid "
                      f"walk with the radius bound, OpenMP dynamic over cells)",
            "seconds": dt, "cells": sample, "result": ref}


def accuracy(got, ref, cells, rtol):
    """Errors of the GPU outputs against the oracle's on the same cells (the
    parity tests' comparison): topology mismatches and the max / rms
    relative error of volume, area and centroid."""
    from tests.compare import compare
    rep = compare(got, ref, rtol, cells=cells)
    topo = (rep["status_mismatch"] + rep["nv_mismatch"] + rep["ne_mismatch"] + rep["nf_mismatch"] +
            rep["face_mismatch"])
    return {"cells": int(len(cells)), "topology_mismatches": int(topo),
            "vol_max_rel": rep["vol_max_rel"], "vol_rms_rel": rep["vol_rms_rel"],
            "area_max_rel": rep["area_max_rel"], "area_rms_rel": rep["area_rms_rel"],
            "centroid_max_rel": rep["centroid_max_rel"], "centroid_rms_rel": rep["centroid_rms_rel"],
            "bar": rtol, "within_bar": bool(rep["topology_ok"] and rep["values_ok"])}


def job_rate(dist, t_local: float, cells_per_rank: int, steps: int, world: int, device) -> tuple[float, float]:
    """Whole-job cells/s of N replicas: every rank's cells over the slowest
    rank's time (a max-reduce, the only collective).  Returns (rate, time)."""
    t = t_local
    if dist is not None:
        import torch
        v = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
        dist.barrier()
    return world * cells_per_rank * steps / t, t


def run_reference(args, rank, world):
    if rank != 0:
        return
    s, grid, _, _ = workload(args.workload, 0)
    per_step = 100_000
    for _ in range(args.warmup):
        cpu_baseline(s, grid, 20_000, seed=99, clip=clip_of(args.workload))
    total, cells = 0.0, 0
    res = None
    for k in range(args.steps):
        res = cpu_baseline(s, grid, per_step, seed=k, clip=clip_of(args.workload))
        total += res["seconds"]
        cells += per_step
    v = cells / total
    line = {"metric": METRIC if s.dim == 3 else METRIC_2D, "value": v, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload].split(";")[0] + "; FP64 CPU oracle"},
            "cpu_baseline": {"value": v, "unit": "cells/s", "kind": "oracle", "cores": res["cores"],
                             "sample": f"{per_step} random cells per step of the {s.n}-point workload"},
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
    from paper_2209_11606_gb300 import predictor as P, vorogpu as V

    big = args.workload in ("slabs102m", "vorotop102m") + PAPER3D + PAPER2D
    s, grid, chosen_order, learned_on = workload(args.workload, rank)
    if args.grid > 0:
        grid = (args.grid,) * s.dim
    n, dim = s.n, s.dim
    order_code = V.VG_PREFETCH if chosen_order == "prefetch" else V.VG_WALK
    stream = torch.cuda.current_stream()
    pos_d = torch.from_numpy(s.pos).cuda()
    rad_d = None if s.radii is None else torch.from_numpy(s.radii).cuda()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    params, mlp_meta = mlp_params(V, torch)
    mlp = P.predictor(params)
    ctx = V.vg_create(dim, s.lo, s.hi, s.periodic, grid, stream=stream)
    if learned_on:
        V.vg_set_predictor(ctx, mlp, MLP_ALPHA, MLP_KMIN, MLP_KMAX)
    clip = clip_of(args.workload)
    cfg = V.vg_config_default()
    cfg.precision, cfg.order, cfg.use_mlp = V.VG_FP32_RETEST, order_code, int(learned_on)
    cfg.clip = clip
    cfg.split = args.split

    # warm-up through the eager calls, then the step as one graph: sort ->
    # learned preload targets -> cells -> faces, the cell kernels timed by
    # event nodes inside the graph
    for _ in range(max(args.warmup, 3)):
        V.vg_insert(ctx, pos_d, rad_d)
        V.vg_compute(ctx, cfg)
    torch.cuda.synchronize()
    gcfg = V.vg_config_default()
    gcfg.clip = clip
    gcfg.precision, gcfg.order, gcfg.use_mlp, gcfg.time_kernels = cfg.precision, cfg.order, cfg.use_mlp, 1
    gcfg.split = cfg.split
    V.vg_graph_capture(ctx, [n], pos_d, rad_d, gcfg)
    for _ in range(max(args.warmup, 3)):
        V.vg_graph_launch(ctx)
    V.vg_graph_sync(ctx)

    # ---- timed region: K steps, L2 flushed between them ----------------------
    V.vg_get_kernel_ms(ctx)  # reset
    l0 = V.vg_get_launches(ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    step_ms = graph_steps(V, torch, ctx, stream, flush, args.steps)
    clk = clocks.stop()
    launches = V.vg_get_launches(ctx) - l0
    kern_ms, kern_n = V.vg_get_kernel_ms(ctx)
    sort_ms, sort_n = V.vg_get_sort_ms(ctx)
    value, t_total = job_rate(dist, sum(step_ms) / 1000.0, n, args.steps, world, "cuda")

    if rank != 0:
        V.vg_destroy(ctx)
        V.vg_mlp_destroy(mlp)
        if dist:
            dist.destroy_process_group()
        return

    # ---- work counters -> algorithmic FLOPs of the cell kernels ----------------
    def flop_of(w, ne, nf):
        if dim == 3:
            fan = 2 * ne.astype(np.int64) - 2 * nf.astype(np.int64)
            return (FLOP_VTEST * w["v"].astype(np.int64).sum() + FLOP_CAND * w["t"].astype(np.int64).sum() +
                    FLOP_NEWV * w["nv"].astype(np.int64).sum() + FLOP_FANTET * fan.sum())
        # 2D: 4 per vertex test, 8 per candidate, 12 per new vertex, 6 per shoelace term
        return (4 * w["v"].astype(np.int64).sum() + 8 * w["t"].astype(np.int64).sum() +
                12 * w["nv"].astype(np.int64).sum() + 6 * ne.astype(np.int64).sum())

    def work(c):
        c.collect_stats = 1
        V.vg_insert(ctx, pos_d, rad_d)
        V.vg_compute(ctx, c)
        c.collect_stats = 0
        w = {k: np.zeros(n, np.int32) for k in ("t", "v", "c", "nv", "r", "p")}
        fb = np.zeros(n, np.uint8)
        V.vg_get_work(ctx, w["t"], w["v"], w["c"], w["nv"], w["r"], fb, w["p"])
        w["deferred"] = V.vg_get_deferred(ctx)
        return w, fb

    w, fb = work(cfg)
    ne = np.zeros(n, np.int32)
    nf = np.zeros(n, np.int32)
    V.vg_get_cells(ctx, ne=ne, nf=nf)
    flop = flop_of(w, ne, nf)
    kern_avg_ms = kern_ms / max(kern_n, 1)
    achieved = flop / (kern_avg_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS,
            "traffic": None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "kernel": ("k_cells3<float,2,64>" if dim == 3 else "k_cells2<float,8,16>") + " (cell kernel phase, all tiers)",
            "kernel_ms": kern_avg_ms,
            "flop_per_cell": flop / n,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    # the counting sort against HBM bandwidth: its algorithmic bytes (input
    # positions, block counts, sorted offsets and ids, the scan) over its
    # device time inside the replays
    peak_gbs, peak_src = hbm_peak()
    sort_avg_ms = sort_ms / max(sort_n, 1)
    grid_used = V.vg_get_grid(ctx, dim)
    sort_bytes = SORT_BYTES_PER_PARTICLE * n + SORT_BYTES_PER_BLOCK * int(np.prod(grid_used))
    sort_gbs = sort_bytes / (sort_avg_ms / 1000.0) / 1e9 if sort_avg_ms > 0 else None
    roof["sort"] = {"bound": "hbm", "ms": sort_avg_ms, "bytes_per_launch": sort_bytes,
                    "achieved": sort_gbs, "peak": peak_gbs, "unit": "GB/s",
                    "frac": None if sort_gbs is None else sort_gbs / peak_gbs,
                    "peak_source": peak_src,
                    "kernels": "widen (FP32 input), rmax (radical), k_index, scans, k_scatter, k_finalize, "
                               "k_predict (learned preload)"}
    roof["work_per_cell"] = {"candidates_tested": float(w["t"].mean()), "vertex_tests": float(w["v"].mean()),
                             "cuts": float(w["c"].mean()), "new_vertices": float(w["nv"].mean()),
                             "fp64_retests": float(w["r"].mean())}
    if CELL_KERNEL_NCU.get(args.workload):
        prof = CELL_KERNEL_NCU[args.workload]
        ipc = prof["warp_inst_per_cell"]
        roof["traffic"] = prof["dram_bytes"]
        roof["traffic_kernel"] = prof["kernel"]
        roof["issue"] = {"warp_inst_per_cell": ipc,
                         "achieved_inst_per_s": ipc * n / (kern_avg_ms / 1000.0),
                         "peak_inst_per_s": ISSUE_PEAK,
                         "frac": ipc * n / (kern_avg_ms / 1000.0) / ISSUE_PEAK,
                         "lanes_active_per_inst": prof["lanes_per_inst"],
                         "issue_active_ncu": prof["issue_active"],
                         "source": prof["source"]}
    learned = None
    if learned_on:
        c_fixed = V.vg_config_default()
        c_fixed.clip = clip
        w_fixed, fb_fixed = work(c_fixed)
        learned = {"shortfall_rate": float((fb > 0).mean()), "walk_rate": float((fb == 1).mean()),
                   "preload_per_cell": float(w["p"].mean()),
                   "fixed_k_shortfall_rate": float((fb_fixed > 0).mean()),
                   "fixed_k_walk_rate": float((fb_fixed == 1).mean()),
                   "fixed_k_preload_per_cell": float(w_fixed["p"].mean()),
                   "deferred_rate": w["deferred"] / n, "fixed_k_deferred_rate": w_fixed["deferred"] / n,
                   "alpha": MLP_ALPHA, "trained": mlp_meta}

    # ---- the same step in other forms (graph replays) ---------------------------
    def form_rate(order, use_mlp, precision=V.VG_FP32_RETEST, reps=5, kernel_ms=False):
        c2 = V.vg_config_default()
        c2.precision, c2.order, c2.use_mlp = precision, order, use_mlp
        c2.clip = clip
        c2.time_kernels = 1 if kernel_ms else 0
        V.vg_graph_capture(ctx, [n], pos_d, rad_d, c2)
        V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        V.vg_get_kernel_ms(ctx)  # reset
        ms = graph_steps(V, torch, ctx, stream, flush, reps)
        rate = n * reps / (sum(ms) / 1000.0)
        if not kernel_ms:
            return rate
        km, kn = V.vg_get_kernel_ms(ctx)
        return rate, km / max(kn, 1)

    forms = {}
    if not args.no_forms and (learned_on or chosen_order != "walk"):
        forms["fp32_walk"] = form_rate(V.VG_WALK, 0)
    if not args.no_forms and dim == 3 and (learned_on or chosen_order != "prefetch"):
        forms["fp32_prefetch_fixed_k72"] = form_rate(V.VG_PREFETCH, 0)
    plain64, plain_roof = None, None
    if not args.no_plain:
        plain64, plain_ms = form_rate(V.VG_WALK, 0, V.VG_FP64, reps=1 if big else 3, kernel_ms=True)
        if not big:
            # the plain form against the FP64 rate: its own work counters
            cp = V.vg_config_default()
            cp.precision, cp.order, cp.clip = V.VG_FP64, V.VG_WALK, clip
            wp, _ = work(cp)
            nep, nfp = np.zeros(n, np.int32), np.zeros(n, np.int32)
            V.vg_get_cells(ctx, ne=nep, nf=nfp)
            fp = flop_of(wp, nep, nfp)
            ach = fp / (plain_ms / 1000.0) / 1e12
            plain_roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                          "frac": ach / FP64_PEAK_TFLOPS, "kernel_ms": plain_ms, "flop_per_cell": fp / n,
                          "peak_source": "nominal FP64 rate of GB300 (no measured FP64 peak)"}

    # ---- end to end through the public API, host buffers -----------------------
    e2e = None
    if not args.no_e2e and args.workload == "uniform1m":
        pos_h = torch.from_numpy(s.pos).pin_memory().numpy()
        outs = {"vol": np.float64, "area": np.float64, "nv": np.int32, "ne": np.int32,
                "nf": np.int32, "status": np.uint8}
        host = {k: torch.empty(n, dtype=getattr(torch, np.dtype(t).name)).pin_memory().numpy()
                for k, t in outs.items()}
        cen = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        V.vg_insert(ctx, pos_d, rad_d)
        V.vg_compute(ctx, cfg)
        _, nface = V.vg_get_counts(ctx)
        fo = torch.empty(n + 1, dtype=torch.int64).pin_memory().numpy()
        cap = int(nface * 1.2) + 1024
        ids = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
        img = torch.empty((cap, 3), dtype=torch.int8).pin_memory().numpy()
        fod = torch.empty(cap, dtype=torch.uint8).pin_memory().numpy()
        reps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
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

    line = {"metric": METRIC if dim == 3 else METRIC_2D, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "cells_per_step": n * world,
                       "kernel_split": args.split, "grid": list(V.vg_get_grid(ctx, dim)),
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas{world}"},
            "step": "one CUDA graph replay: counting sort, learned preload targets, cell kernels "
                    "(3 capacity tiers), face CSR",
            "roofline": roof,
            "plain_fp64": None if plain64 is None else
            {"value": plain64, "unit": "cells/s", "form": "FP64 everywhere, block walk (Sec. 2.1.3), graph replay",
             "roofline": plain_roof},
            "chosen_vs_plain": None if plain64 is None else value / world / plain64,
            "forms": forms, "learned_preload": learned,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "retest_per_cell": float(w["r"].mean())}
    if args.weinberg and dim == 3:
        line["weinberg"] = weinberg_run(V, torch, ctx, pos_d, rad_d, cfg, n, stream, flush)
    if not args.no_batched and args.workload == "uniform1m":
        line["batched"] = batched_run(V, torch, stream, flush, mlp)
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(s, grid, n if args.workload == "uniform1m" else 100_000, clip=clip)
        line["cpu_baseline"] = {k: v for k, v in cb.items() if k not in ("seconds", "cells", "result")}
        if not args.no_accuracy:
            # every output of the chosen form and of the plain FP64 form against
            # the oracle, on the cells the CPU baseline computed
            acc = {}
            for name, c2, rtol in (("chosen", cfg, 1e-5), ("plain_fp64", None, 1e-12)):
                if c2 is None:
                    c2 = V.vg_config_default()
                    c2.precision, c2.order, c2.clip = V.VG_FP64, V.VG_WALK, clip
                V.vg_insert(ctx, pos_d, rad_d)
                V.vg_compute(ctx, c2)
                got = V._fetch(ctx, n, dim, False)
                acc[name] = accuracy(got, cb["result"], cb["cells"], rtol)
            line["accuracy"] = acc
    if not args.no_large and args.workload == "uniform1m" and world == 1:
        line["large"] = large_run(V, torch, stream, flush, mlp, with_oracle=not args.no_cpu_baseline)
    V.vg_destroy(ctx)
    V.vg_mlp_destroy(mlp)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
