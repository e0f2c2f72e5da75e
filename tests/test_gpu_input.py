"""FP32 input (vg_insert / vg_batch_insert / vg_graph_capture with dtype
VG_F32): the library widens the values to FP64 on the device before the
sort, so its cells must be the oracle's cells of the same FP32 values read
as FP64 -- topology bit-exact, volumes, areas and centroids within the
form's bar."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare
from tests.test_gpu_batch import slice_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()
    return torch


def _fetch(ctx, n, d):
    from paper_2209_11606_gb300 import vorogpu as V
    return V._fetch(ctx, n, d, False)


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_fp32_points_match_the_oracle_on_the_rounded_points(torch_dev, where, precision, rtol):
    from paper_2209_11606_gb300 import vorogpu as V
    torch = torch_dev
    s = W.uniform(4000, 3, 4000 ** (1 / 3), True, seed=61)
    p32 = s.pos.astype(np.float32)
    ref = oracle.compute(p32.astype(np.float64), s.lo, s.hi, s.periodic, nblocks=(9, 9, 9))
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, (9, 9, 9))
    try:
        V.vg_insert(ctx, p32 if where == "host" else torch.from_numpy(p32).cuda())
        cfg = V._make_cfg(precision, "walk" if precision == "fp64" else "prefetch", False, {})
        V.vg_compute(ctx, cfg)
        got = _fetch(ctx, s.n, 3)
    finally:
        V.vg_destroy(ctx)
    rep = compare(got, ref, rtol)
    assert rep["topology_ok"] and rep["values_ok"], rep


def test_fp32_radii_and_batch(torch_dev):
    """Radical cells from FP32 positions and radii in a batched container."""
    from paper_2209_11606_gb300 import vorogpu as V
    a = W.radical_uniform(1500, 0.4, 0.3, seed=62)
    b = W.uniform(700, 3, 3.0, False, seed=63)
    b.radii = np.full(b.n, 0.2)
    systems = [a, b]
    descs = [V.vg_system(x.lo, x.hi, x.periodic, (6, 6, 6)) for x in systems]
    pos32 = np.concatenate([x.pos for x in systems]).astype(np.float32)
    rad32 = np.concatenate([x.radii for x in systems]).astype(np.float32)
    ctx = V.vg_batch_create(3, descs)
    try:
        V.vg_batch_insert(ctx, [x.n for x in systems], pos32, rad32)
        V.vg_compute(ctx, V._make_cfg("fp32", "walk", False, {}))
        got = _fetch(ctx, pos32.shape[0], 3)
    finally:
        V.vg_destroy(ctx)
    base = 0
    for x in systems:
        p = pos32[base:base + x.n].astype(np.float64)
        r = rad32[base:base + x.n].astype(np.float64)
        ref = oracle.compute(p, x.lo, x.hi, x.periodic, radii=r, nblocks=(6, 6, 6))
        rep = compare(slice_system(got, base, x.n), ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], rep
        base += x.n


def test_fp32_graph_replay_equals_eager(torch_dev):
    from paper_2209_11606_gb300 import vorogpu as V
    torch = torch_dev
    s = W.uniform(5000, 3, 5000 ** (1 / 3), True, seed=64)
    p32 = torch.from_numpy(s.pos.astype(np.float32)).cuda()
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, (10, 10, 10))
    try:
        cfg = V._make_cfg("fp32", "prefetch", False, {})
        V.vg_insert(ctx, p32)
        V.vg_compute(ctx, cfg)
        eager = _fetch(ctx, s.n, 3)
        V.vg_graph_capture(ctx, [s.n], p32, None, cfg)
        V.vg_graph_launch(ctx)
        V.vg_graph_sync(ctx)
        replay = _fetch(ctx, s.n, 3)
    finally:
        V.vg_destroy(ctx)
    for k in ("vol", "area", "centroid", "nf", "nbr_id", "face_off"):
        assert np.array_equal(eager[k], replay[k]), k
