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
