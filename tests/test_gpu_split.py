"""The two kernels of the 3D FP32 prefetch form (`vg_config.split`).

With split = 1 a kernel built for the common path (distance-sorted preload,
FP32 cuts with the FP64 re-test, FP32 statistics) computes every cell it
can and hands the rest to the general kernel, which computes those cells
from the start: the walk after both preloads, FP64 statistics (degenerate
or ill-conditioned vertices), plane slots used up, more than 32 faces.  With split = 0 the general kernel
computes every cell.  Both settings give the oracle's cells (topology
bit-exact, values within the FP32 form's 1e-5), and the hand-over count
(`vg_get_deferred`) is small on uniform points, every cell on an exact
FCC lattice (degree-4 vertices: FP64 statistics), and zero with split = 0.
"""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()


def run(s, nb, split):
    from paper_2209_11606_gb300 import vorogpu as V
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, nb)
    try:
        V.vg_insert(ctx, np.ascontiguousarray(s.pos, dtype=np.float64))
        cfg = V._make_cfg("fp32", "prefetch", False, {"split": split})
        V.vg_compute(ctx, cfg)
        out = V._fetch(ctx, s.n, 3, False)
        out["deferred"] = V.vg_get_deferred(ctx)
        out["grid"] = V.vg_get_grid(ctx, 3)
        return out
    finally:
        V.vg_destroy(ctx)


CASES = {
    # (points, blocks, bounds on the share of cells handed over with split = 1)
    "uniform": (lambda: W.uniform(20_000, 3, 20_000 ** (1 / 3), True, seed=61), (16, 16, 16), (0.0, 0.02)),
    "fcc_exact": (lambda: W.fcc(4, 1.0), (4, 4, 4), (0.99, 1.0)),
    # surface cells of a cluster reach the walls: the walk after the preloads
    "localized": (lambda: W.localized(50_000, 3, 0.1, seed=62), (17, 17, 17), (0.001, 0.5)),
    "clustered": (lambda: W.extreme_clustering(20_000, 3, seed=63), (34, 34, 34), (0.001, 1.0)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_split_gives_the_oracles_cells(name):
    make, nb, (lo_share, hi_share) = CASES[name]
    s = make()
    hot = run(s, nb, 1)
    gen = run(s, nb, 0)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=hot["grid"])
    for got in (hot, gen):
        rep = compare(got, ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], (name, rep)
    assert gen["deferred"] == 0
    share = hot["deferred"] / s.n
    assert lo_share <= share <= hi_share, (name, hot["deferred"], s.n)


def test_per_system_split_in_a_batch():
    # a batch of three systems with the middle one marked for the general
    # kernel: all of its cells are handed over, every system's cells equal
    # the oracle's, and the whole batch equals the all-hot one bit for bit
    from paper_2209_11606_gb300 import vorogpu as V
    from tests.test_gpu_batch import slice_system
    systems = [W.uniform(6000, 3, 6000 ** (1 / 3), True, seed=64),
               W.extreme_clustering(4000, 3, seed=65),
               W.fcc(6, 1.0, 0.05, seed=66)]
    descs = [V.vg_system(s.lo, s.hi, s.periodic, n_opt=4.6) for s in systems]
    pos = np.ascontiguousarray(np.concatenate([s.pos for s in systems]))
    counts = [s.n for s in systems]
    outs = []
    for marks in ((1, 1, 1), (1, 0, 1)):
        ctx = V.vg_batch_create(3, descs)
        try:
            for k, m in enumerate(marks):
                V.vg_set_system_split(ctx, k, m)
            V.vg_batch_insert(ctx, counts, pos)
            V.vg_compute(ctx, V._make_cfg("fp32", "prefetch", False, {"split": 1}))
            out = V._fetch(ctx, pos.shape[0], 3, False)
            out["deferred"] = V.vg_get_deferred(ctx)
            out["grids"] = [V.vg_get_system_grid(ctx, k, 3) for k in range(3)]
            outs.append(out)
        finally:
            V.vg_destroy(ctx)
    assert outs[1]["deferred"] >= systems[1].n
    base = 0
    for k, s in enumerate(systems):
        ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=outs[1]["grids"][k])
        rep = compare(slice_system(outs[1], base, s.n), ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], (k, rep)
        base += s.n
    for key in ("nv", "ne", "nf", "status", "face_off", "nbr_id", "face_order"):
        np.testing.assert_array_equal(outs[0][key], outs[1][key])
    with pytest.raises(V.VgError):
        _bad_split(V, descs)


def _bad_split(V, descs):
    ctx = V.vg_batch_create(3, descs)
    try:
        V.vg_set_system_split(ctx, 3, 1)  # no system 3
    finally:
        V.vg_destroy(ctx)
