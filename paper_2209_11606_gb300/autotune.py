"""Autotuner of the launch and grid parameters (argument marshalling and
timing around the C ABI; the timed work runs in the library's kernels).

The paper picks the particles-per-block target N_opt and the OpenMP chunk by
hand-run scans and finds that the best N_opt depends strongly on the
particle distribution (Sec. 2.1.4, Table 3, and the chunk scans of Sec. 3.1).
Here the scan is automatic: for a system, every combination of

* N_opt in {1, 2, 3, 4.6, 6, 8, 12, 16} (block counts by the rule of
  Sec. 2.1.4; the paper's best values span 0.5 to 49 across distributions),
* warps per CTA in {1, 2, 4} (one warp per cell, so CTA sizes 32..128),
* candidate order in {sorted prefetch, block walk},
* cells per work-queue ticket in {1, 2, 4},
* for the sorted prefetch, a fixed preload target or the learned one (when
  a predictor is given: per-block targets from the MLP of Sec. 2.1.3's
  candidate count, computed at insert),

is timed on a seeded random sample of the cells (vg_compute_subset, CUDA
events around the cell kernels), and the fastest is kept.  Results are cached
in a JSON file keyed by (dimension, radical, size bucket, distribution class),
the class read from the spread of the block counts.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import vorogpu as V

N_OPT = (1.0, 2.0, 3.0, 4.6, 6.0, 8.0, 12.0, 16.0, 24.0, 32.0, 48.0)
WARPS = (1, 2, 4)
ORDERS = ("prefetch", "walk")
CHUNKS = (1, 2, 4)


def distribution_class(pos, lo, hi, periodic=None) -> str:
    """'lattice', 'uniform' or 'clustered' from the coefficient of variation
    of the block counts on a grid of about 5 particles per block (a Poisson
    set gives about 0.45, a perturbed lattice far less, clusters far more)."""
    pos = np.asarray(pos, dtype=np.float64)
    n, d = pos.shape
    if n < 50:
        return "small"
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    lam = (n / (5.0 * np.prod(L))) ** (1.0 / d)
    nb = np.maximum(1, np.floor(lam * L).astype(np.int64))
    idx = np.clip(np.floor((pos - lo) / (L / nb)).astype(np.int64), 0, nb - 1)
    key = idx[:, 0]
    mul = nb[0]
    for a in range(1, d):
        key = key + mul * idx[:, a]
        mul *= nb[a]
    c = np.bincount(key, minlength=int(np.prod(nb))).astype(np.float64)
    cv = c.std() / max(c.mean(), 1e-12)
    if cv < 0.3:
        return "lattice"
    if cv < 0.8:
        return "uniform"
    return "clustered"


def cache_key(dim: int, radical: bool, n: int, cls: str) -> str:
    return f"d{dim}-r{int(bool(radical))}-n2^{int(math.log2(max(n, 1)))}-{cls}"


class Cache:
    """JSON file of tuned parameters."""

    def __init__(self, path: str):
        self.path = path
        self.data = {}
        if os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, key):
        return self.data.get(key)

    def put(self, key, value):
        self.data[key] = value
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _cfg(order: str, warps: int, chunk: int, use_mlp: int = 0, split: int = 1):
    cfg = V.vg_config_default()
    cfg.order = V.VG_WALK if order == "walk" else V.VG_PREFETCH
    cfg.warps_per_cta = warps
    cfg.chunk = chunk
    cfg.use_mlp = int(use_mlp)
    cfg.split = int(split)
    return cfg


def _time_subset(ctx, sample, cfg, reps: int) -> float:
    V.vg_compute_subset(ctx, sample, cfg)            # warm-up
    cfg.time_kernels = 1
    V.vg_get_kernel_ms(ctx)
    for _ in range(reps):
        V.vg_compute_subset(ctx, sample, cfg)
    ms, cnt = V.vg_get_kernel_ms(ctx)
    cfg.time_kernels = 0
    return ms / max(cnt, 1)


def tune_system(s, torch, sample_frac: float = 0.05, min_sample: int = 20000, seed: int = 0,
                reps: int = 2, n_opts=N_OPT, warps=WARPS, orders=ORDERS, chunks=CHUNKS,
                fixed_grid=None) -> dict:
    """Times every combination on a sample of s's cells; returns the best
    and the full table.  With `fixed_grid` the block counts are not tuned."""
    n = s.n
    rng = np.random.default_rng(seed)
    m = min(n, max(int(sample_frac * n), min_sample))
    sample = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    pos = torch.from_numpy(np.ascontiguousarray(s.pos)).cuda()
    rad = None if s.radii is None else torch.from_numpy(np.ascontiguousarray(s.radii)).cuda()
    table = []
    grids = [("fixed", fixed_grid)] if fixed_grid is not None else [(v, None) for v in n_opts]
    for nopt, nb in grids:
        ctx = V.vg_create(s.dim, s.lo, s.hi, s.periodic, nb, 0.0 if nb is not None else nopt)
        try:
            V.vg_insert(ctx, pos, rad)
            grid = V.vg_get_grid(ctx, s.dim)
            for order in orders:
                if order == "prefetch" and s.dim != 3:
                    continue
                for w in warps:
                    for ch in chunks:
                        ms = _time_subset(ctx, sample, _cfg(order, w, ch), reps)
                        table.append({"n_opt": nopt, "grid": list(grid), "order": order,
                                      "warps_per_cta": w, "chunk": ch, "ms": ms,
                                      "cells_per_s": m / (ms / 1000.0)})
        finally:
            V.vg_destroy(ctx)
    best = min(table, key=lambda r: r["ms"])
    return {"best": best, "table": table, "sample": m}


def tuned(s, torch, cache: Cache | None = None, cls: str | None = None, **kw) -> dict:
    """The cached best parameters for s's class, tuning on a miss."""
    cls = cls or distribution_class(s.pos, s.lo, s.hi)
    key = cache_key(s.dim, s.radii is not None, s.n, cls)
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            return hit
    res = tune_system(s, torch, **kw)
    best = dict(res["best"])
    best["class"] = cls
    best["key"] = key
    best["sample"] = res["sample"]
    if cache is not None:
        cache.put(key, best)
    return best


def config_from(best: dict):
    """vg_config of a tuned entry."""
    return _cfg(best["order"], int(best["warps_per_cta"]), int(best["chunk"]), int(best.get("use_mlp", 0)),
                int(best.get("split", 1)))


def tune_batch(systems, torch, cache: Cache | None = None, sample_frac: float = 0.05, seed: int = 0,
               reps: int = 2, predictor=None, mlp_args=(1.2, 24.0, 1024.0)) -> dict:
    """Parameters for a batch of systems: N_opt per distribution class (tuned
    on the class's largest system with the default launch), then the launch
    parameters (order, warps per CTA, chunk, the hot/general kernel split of
    the prefetch form, for the whole batch or per distribution class
    (`launch["hot_classes"]`: the classes on the hot kernel), and with a
    `predictor` handle fixed or learned preload targets, `mlp_args` =
    (alpha, kmin, kmax)) on a sample of the whole batch with those grids.  Returns {"n_opt": [...],
    "launch": {...}, "classes": [...]}."""
    classes = [distribution_class(x.pos, x.lo, x.hi) for x in systems]
    n_opt_of = {}
    for cls in sorted(set(classes)):
        rep = max((x for x, c in zip(systems, classes) if c == cls), key=lambda x: x.n)
        key = cache_key(rep.dim, rep.radii is not None, rep.n, cls) + "-grid"
        hit = cache.get(key) if cache is not None else None
        if hit is None:
            res = tune_system(rep, torch, sample_frac=sample_frac, seed=seed, reps=reps,
                              orders=("prefetch",) if rep.dim == 3 else ("walk",), warps=(4,), chunks=(2,))
            hit = {"n_opt": res["best"]["n_opt"], "class": cls, "sample": res["sample"]}
            if cache is not None:
                cache.put(key, hit)
        n_opt_of[cls] = float(hit["n_opt"])
    n_opts = [n_opt_of[c] for c in classes]
    descs = [V.vg_system(x.lo, x.hi, x.periodic, n_opt=v) for x, v in zip(systems, n_opts)]
    counts = [x.n for x in systems]
    n = int(sum(counts))
    pos = torch.from_numpy(np.concatenate([x.pos for x in systems])).cuda()
    radical = systems[0].radii is not None
    rad = torch.from_numpy(np.concatenate([x.radii for x in systems])).cuda() if radical else None
    rng = np.random.default_rng(seed)
    m = min(n, max(int(sample_frac * n), 20000))
    sample = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    ctx = V.vg_batch_create(systems[0].dim, descs)
    table = []
    try:
        if predictor is not None:
            V.vg_set_predictor(ctx, predictor, *mlp_args)
        V.vg_batch_insert(ctx, counts, pos, rad)
        for order in ORDERS:
            if order == "prefetch" and systems[0].dim != 3:
                continue
            mlps = (0, 1) if order == "prefetch" and predictor is not None else (0,)
            splits = (1, 0) if order == "prefetch" or systems[0].dim == 2 else (1,)
            for w in WARPS:
                for ch in CHUNKS:
                    for um in mlps:
                        for sp in splits:
                            ms = _time_subset(ctx, sample, _cfg(order, w, ch, um, sp), reps)
                            table.append({"order": order, "warps_per_cta": w, "chunk": ch, "use_mlp": um,
                                          "split": sp, "ms": ms})
        # 3D prefetch: the kernel split per distribution class (some classes
        # on the kernel built for the common path, the rest on the general
        # one), at the best launch so far
        best = min(table, key=lambda r: r["ms"])
        cls_set = sorted(set(classes))
        if best["order"] == "prefetch" and systems[0].dim == 3 and len(cls_set) > 1:
            for mask in range(1, (1 << len(cls_set)) - 1):
                hot = [c for b, c in enumerate(cls_set) if (mask >> b) & 1]
                for k, c in enumerate(classes):
                    V.vg_set_system_split(ctx, k, int(c in hot))
                cfg = _cfg("prefetch", best["warps_per_cta"], best["chunk"], best["use_mlp"], 1)
                ms = _time_subset(ctx, sample, cfg, reps)
                table.append({"order": "prefetch", "warps_per_cta": best["warps_per_cta"], "chunk": best["chunk"],
                              "use_mlp": best["use_mlp"], "split": 1, "hot_classes": hot, "ms": ms})
    finally:
        V.vg_destroy(ctx)
    launch = min(table, key=lambda r: r["ms"])
    return {"n_opt": n_opts, "classes": classes, "launch": launch, "table": table, "sample": m}
