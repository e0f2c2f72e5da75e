"""Autotuner: the distribution classes (CPU) and, on a GPU, that the chosen
parameters are the fastest of those timed, that the cache returns them, and
that the tuned configuration computes the same cells."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import autotune as A
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare


def test_distribution_classes():
    assert A.distribution_class(*_sys(W.uniform(20000, 3, 1.0, True, seed=1))) == "uniform"
    assert A.distribution_class(*_sys(W.bcc(20, 1.25, 0.02, seed=2))) == "lattice"
    assert A.distribution_class(*_sys(W.blobs(20000, 27.0, 50, 0.02, True, 3))) == "clustered"
    assert A.distribution_class(*_sys(W.uniform(10, 3, 1.0, True, seed=4))) == "small"


def _sys(s):
    return s.pos, s.lo, s.hi


def test_cache_roundtrip(tmp_path):
    c = A.Cache(str(tmp_path / "tune.json"))
    k = A.cache_key(3, False, 1_000_000, "uniform")
    assert k == "d3-r0-n2^19-uniform"
    c.put(k, {"n_opt": 4.6, "order": "prefetch", "warps_per_cta": 4, "chunk": 2})
    c2 = A.Cache(str(tmp_path / "tune.json"))
    assert c2.get(k)["n_opt"] == 4.6


@pytest.mark.gpu
def test_tuner_picks_the_fastest_and_caches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()
    s = W.uniform(60000, 3, 60000 ** (1 / 3), True, seed=5)
    res = A.tune_system(s, torch, sample_frac=0.2, n_opts=(2.0, 4.6), warps=(2, 4), chunks=(1, 2))
    assert len(res["table"]) == 2 * 2 * 2 * 2
    assert res["best"]["ms"] == min(r["ms"] for r in res["table"])
    cache = A.Cache(str(tmp_path / "t.json"))
    b1 = A.tuned(s, torch, cache, sample_frac=0.2, n_opts=(2.0, 4.6), warps=(2, 4), chunks=(1, 2))
    b2 = A.tuned(s, torch, cache)  # a cache hit: no timing
    assert b1 == b2 and b1["class"] == "uniform"


@pytest.mark.gpu
def test_tuned_batch_computes_the_same_cells():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build, vorogpu as V
    from tests.test_gpu_batch import slice_system
    build.build()
    systems = W.batched_systems(nsys=6, nmin=2000, nmax=8000, seed=21)
    tb = A.tune_batch(systems, torch, sample_frac=0.3)
    assert len(tb["n_opt"]) == 6 and all(v in A.N_OPT for v in tb["n_opt"])
    descs = [V.vg_system(x.lo, x.hi, x.periodic, n_opt=v) for x, v in zip(systems, tb["n_opt"])]
    cfg = A.config_from(tb["launch"])
    got = V.compute_batch_host(descs, [x.pos for x in systems],
                               order="walk" if tb["launch"]["order"] == "walk" else "prefetch",
                               warps_per_cta=cfg.warps_per_cta, chunk=cfg.chunk)
    base = 0
    for k, x in enumerate(systems):
        ref = oracle.compute(x.pos, x.lo, x.hi, x.periodic, nblocks=got["grids"][k])
        rep = compare(slice_system(got, base, x.n), ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], (k, rep)
        base += x.n
