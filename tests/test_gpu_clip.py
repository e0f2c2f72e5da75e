"""Clipped cells (Sec. 3.1.3) on the GPU against the oracle with the same
clip: each cell starts from the box intersected with the cube (2D: square)
of side h centred on its particle.  Topology bit-exact, values within 1e-12
(FP64 form) and 1e-5 (FP32 form with FP64 re-test)."""
import math

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


def check(s, nb, precision, order, rtol, clip):
    from paper_2209_11606_gb300 import vorogpu
    got = vorogpu.compute_host(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, nblocks=nb,
                               precision=precision, order=order, clip=clip)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, method="grid",
                         nblocks=got["grid"], clip=clip)
    rep = compare(got, ref, rtol)
    assert rep["topology_ok"], rep
    assert rep["values_ok"], rep
    return got, ref


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_localized_3d_clipped_like_the_paper(precision, order, rtol):
    # the paper's test scaled down: N' candidates, those in the central cube
    # of volume 0.1 kept, cube side h = 1.5 sqrt(3) d0 with d0 = N'^(-1/3)
    n_cand = 200_000
    s = W.localized(n_cand, 3, 0.1, seed=21)
    h = 1.5 * math.sqrt(3) * n_cand ** (-1 / 3)
    got, _ = check(s, None, precision, order, rtol, h)
    # cells deep inside the cluster stay unclipped; the outer ones are cut
    walls = got["nbr_id"] < 0
    assert 0 < walls.sum() < len(walls)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_periodic_clip_smaller_than_cells(precision, order, rtol):
    s = W.uniform(3000, 3, 1.0, True, seed=22)
    check(s, (8, 8, 8), precision, order, rtol, 0.08)


@pytest.mark.parametrize("precision,order,rtol", FORMS[:2])
def test_localized_2d_clipped(precision, order, rtol):
    n_cand = 100_000
    s = W.localized(n_cand, 2, 0.1, seed=23)
    check(s, None, precision, order, rtol, 1.5 * math.sqrt(2) * n_cand ** (-1 / 2))


def test_bcc_clipped_closed_form():
    # V = 0.7^3 - 8 (0.3^3 / 6) for BCC with a = 1 and a cube of side 0.7
    s = W.bcc(6, 1.0)
    got, _ = check(s, (6, 6, 6), "fp32", "prefetch", 1e-5, 0.7)
    np.testing.assert_allclose(got["vol"], 0.7 ** 3 - 8 * 0.3 ** 3 / 6, rtol=1e-6)
    assert np.all(got["nf"] == 14)


def test_radical_clipped():
    s = W.radical_uniform(4000, 0.4, 0.3, seed=24)
    d0 = (np.prod(np.asarray(s.hi) - np.asarray(s.lo)) / s.n) ** (1 / 3)
    check(s, None, "fp32", "walk", 1e-5, 1.2 * d0)


def test_clip_rejects_bad_values():
    from paper_2209_11606_gb300 import vorogpu
    s = W.uniform(100, 3, 1.0, False, seed=25)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(vorogpu.VgError):
            vorogpu.compute_host(s.pos, s.lo, s.hi, s.periodic, nblocks=(2, 2, 2), clip=bad)
