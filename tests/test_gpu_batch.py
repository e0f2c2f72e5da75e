"""Batched containers: many independent systems sorted and computed in one
pass (one counting sort over all systems' blocks, one persistent cell launch
fed by one work queue).  Every system's cells must equal the oracle's for
that system alone, and equal the single-system library call bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare

pytestmark = pytest.mark.gpu

FORMS = [("fp64", "walk", 1e-12), ("fp32", "walk", 1e-5), ("fp32", "prefetch", 1e-5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()


def vg():
    from paper_2209_11606_gb300 import vorogpu
    return vorogpu


def slice_system(out, base, n):
    """System k's part of a batched result, neighbour ids made local."""
    fo = out["face_off"]
    a, b = int(fo[base]), int(fo[base + n])
    ids = out["nbr_id"][a:b].astype(np.int64).copy()
    ids[ids >= 0] -= base
    return {
        "vol": out["vol"][base:base + n], "area": out["area"][base:base + n],
        "centroid": out["centroid"][base:base + n], "nv": out["nv"][base:base + n],
        "ne": out["ne"][base:base + n], "nf": out["nf"][base:base + n],
        "status": out["status"][base:base + n], "face_off": fo[base:base + n + 1] - a,
        "nbr_id": ids, "nbr_img": out["nbr_img"][a:b], "face_order": out["face_order"][a:b],
    }


def run_batch(systems, precision, order, radical=False, **kw):
    v = vg()
    descs = [v.vg_system(s.lo, s.hi, s.periodic, n_opt=0.0) for s in systems]
    radii = [s.radii for s in systems] if radical else None
    return v.compute_batch_host(descs, [s.pos for s in systems], radii, precision=precision,
                                order=order, **kw)


def check_batch(systems, precision, order, rtol, radical=False):
    got = run_batch(systems, precision, order, radical)
    base = 0
    for k, s in enumerate(systems):
        nb = got["grids"][k]
        ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii if radical else None,
                             nblocks=nb)
        part = slice_system(got, base, s.n)
        rep = compare(part, ref, rtol)
        assert rep["topology_ok"], (k, s.tag, rep)
        assert rep["values_ok"], (k, s.tag, rep)
        base += s.n
    return got


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_batch_mixed_systems_match_oracle(precision, order, rtol):
    systems = W.batched_systems(nsys=12, nmin=40, nmax=2500, seed=11)
    check_batch(systems, precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS[::2])
def test_batch_equals_single_system_calls(precision, order, rtol):
    systems = W.batched_systems(nsys=6, nmin=200, nmax=3000, seed=12)
    got = run_batch(systems, precision, order)
    base = 0
    for k, s in enumerate(systems):
        one = vg().compute_host(s.pos, s.lo, s.hi, s.periodic, nblocks=got["grids"][k],
                                precision=precision, order=order)
        part = slice_system(got, base, s.n)
        for key in ("vol", "area", "centroid", "nv", "ne", "nf", "status", "face_off",
                    "nbr_id", "nbr_img", "face_order"):
            assert np.array_equal(np.asarray(part[key]), np.asarray(one[key])), (k, key)
        base += s.n


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_batch_radical_per_system_rmax(precision, order, rtol):
    # systems with very different radius spreads: each stop test must use
    # its own system's largest radius
    systems = []
    for k, sig in enumerate((0.05, 0.3, 0.6)):
        s = W.radical_uniform(1500 + 500 * k, packing=0.4, sigma=sig, seed=20 + k)
        if k == 1:
            s.periodic = (False, True, False)
        systems.append(s)
    check_batch(systems, precision, order, rtol, radical=True)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_2d(precision, rtol):
    systems = [W.uniform(1200, 2, 1.0, True, seed=31), W.uniform(700, 2, 3.0, False, seed=32),
               W.hexagonal(12, 10, (1.0, 1.0), 0.03, seed=33)]
    check_batch(systems, precision, "walk", rtol)


def test_batch_with_empty_and_tiny_systems():
    systems = [W.uniform(500, 3, 1.0, True, seed=41), W.uniform(0, 3, 1.0, False, seed=42),
               W.uniform(1, 3, 2.0, False, seed=43), W.uniform(2, 3, 1.0, True, seed=44),
               W.uniform(800, 3, 5.0, False, seed=45)]
    check_batch(systems, "fp32", "prefetch", 1e-5)
    check_batch(systems, "fp64", "walk", 1e-12)


def test_batch_api_errors():
    v = vg()
    s = W.uniform(100, 3, 1.0, True, seed=50)
    ctx = v.vg_batch_create(3, [v.vg_system(s.lo, s.hi, s.periodic)] * 2)
    try:
        with pytest.raises(v.VgError) as e:
            v.vg_insert(ctx, s.pos)
        assert e.value.code == 7  # VG_ERR_STATE: batched containers take vg_batch_insert
        with pytest.raises(ValueError):
            v.vg_batch_insert(ctx, [60, 60], s.pos)
        v.vg_batch_insert(ctx, [40, 60], s.pos)
        v.vg_compute(ctx)
        assert v.vg_get_counts(ctx)[0] == 100
    finally:
        v.vg_destroy(ctx)
    with pytest.raises(v.VgError):
        v.vg_batch_create(3, [])
