"""Parity of the CUDA path with the FP64 oracle, element by element.

Tolerances: topology (status, V/E/F, neighbour ids and images, face orders)
bit-exact; volume, area and centroid within 1e-12 relative for the FP64
form and 1e-5 for the FP32 form with FP64 re-test."""
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


def run(s, nb, precision, order, **kw):
    from paper_2209_11606_gb300 import vorogpu
    return vorogpu.compute_host(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, nblocks=nb,
                                precision=precision, order=order, **kw)


def check(s, nb, precision, order, rtol, method="grid"):
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, method=method, nblocks=nb)
    got = run(s, nb, precision, order)
    rep = compare(got, ref, rtol)
    assert rep["topology_ok"], rep
    assert rep["values_ok"], rep
    return got, ref, rep


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_unit_cube_1000_walled(precision, order, rtol):
    s = W.workload("unit1000")
    check(s, (6, 6, 6), precision, order, rtol, method="brute")


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_uniform_periodic(precision, order, rtol):
    s = W.uniform(3000, 3, 3000 ** (1 / 3), True, seed=7)
    check(s, (8, 8, 8), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_mixed_periodicity_ragged_grid(precision, order, rtol):
    s = W.uniform(2500, 3, 1.0, False, seed=8)
    s.periodic = (True, False, True)
    check(s, (7, 5, 6), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_bcc_exact_lattice(precision, order, rtol):
    s = W.bcc(4, 1.25)
    got, _, _ = check(s, (4, 4, 4), precision, order, rtol)
    assert np.all(got["nf"] == 14) and np.all(got["nv"] == 24)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_fcc_exact_lattice_degree4(precision, order, rtol):
    s = W.fcc(3, 1.0)
    got, _, _ = check(s, (3, 3, 3), precision, order, rtol)
    assert np.all(got["nf"] == 12) and np.all(got["nv"] == 14) and np.all(got["ne"] == 24)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_perturbed_bcc(precision, order, rtol):
    s = W.bcc(6, 1.25, 0.02, seed=2)
    got, _, _ = check(s, (6, 6, 6), precision, order, rtol)
    for i in range(s.n):
        a, b = got["face_off"][i], got["face_off"][i + 1]
        assert sorted(got["face_order"][a:b].tolist()) == [4] * 6 + [6] * 8


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_tiny_systems(precision, order, rtol):
    for n, per in ((1, True), (1, False), (2, False), (5, True)):
        s = W.uniform(n, 3, 1.0, per, seed=10 + n)
        check(s, (2, 2, 2), precision, order, rtol, method="brute")


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_uniform_periodic_20k_all_cells(precision, order, rtol):
    # large enough that walks span several windows of blocks
    s = W.uniform(20000, 3, 20000 ** (1 / 3), True, seed=17)
    check(s, (16, 16, 16), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_uniform_walled_fine_grid(precision, order, rtol):
    # small blocks (about one particle each): long walks over many blocks
    s = W.uniform(8000, 3, 1.0, False, seed=18)
    check(s, (20, 20, 20), precision, order, rtol)


# ---------------------------------------------------------------- 2D
FORMS2 = [("fp64", "walk", 1e-12), ("fp32", "walk", 1e-5)]


@pytest.mark.parametrize("precision,order,rtol", FORMS2)
def test_2d_uniform_walled_and_periodic(precision, order, rtol):
    for per, seed in ((False, 21), (True, 22)):
        s = W.uniform(5000, 2, 1.0, per, seed=seed)
        check(s, (37, 29), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS2)
def test_2d_square_lattice_degree4(precision, order, rtol):
    s = W.square(12, 0.25)
    got, _, _ = check(s, (6, 6), precision, order, rtol)
    assert np.all(got["nv"] == 4)


@pytest.mark.parametrize("precision,order,rtol", FORMS2)
def test_2d_perturbed_hexagonal(precision, order, rtol):
    s = W.hexagonal(60, 70, (1.0, 1.0), 0.05, seed=3)
    got, _, _ = check(s, (30, 30), precision, order, rtol)
    assert got["nv"].sum() == 6 * s.n  # torus: mean 6 edges


@pytest.mark.parametrize("precision,order,rtol", FORMS2)
def test_2d_tiny(precision, order, rtol):
    for n, per in ((1, True), (1, False), (2, False), (4, True)):
        s = W.uniform(n, 2, 1.0, per, seed=30 + n)
        check(s, (2, 2), precision, order, rtol, method="brute")


# ------------------------------------------------------------ radical
@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_radical_3d(precision, order, rtol):
    s = W.radical_uniform(3000, packing=0.4, sigma=0.3, seed=41)
    got, ref, _ = check(s, (7, 7, 7), precision, order, rtol)
    np.testing.assert_allclose(got["vol"].sum(), np.prod(s.hi), rtol=rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_radical_3d_empty_cells(precision, order, rtol):
    s = W.radical_uniform(2000, packing=0.4, sigma=0.8, seed=42)
    got, ref, _ = check(s, (6, 6, 6), precision, order, rtol)
    assert (ref["status"] == 1).sum() > 0  # the case holds empty cells


@pytest.mark.parametrize("precision,order,rtol", FORMS2)
def test_radical_2d(precision, order, rtol):
    s = W.uniform(3000, 2, 1.0, True, seed=43)
    s.radii = W.radii_lognormal(3000, 1.0, 0.4, dim=2, sigma=0.3, seed=44)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, nblocks=(25, 25))
    got = run(s, (25, 25), precision, order)
    rep = compare(got, ref, rtol)
    assert rep["topology_ok"], rep
    assert rep["vol_max_rel"] <= rtol and rep["centroid_max_rel"] <= rtol, rep
    # perimeters of radical polygons with nearly parallel edges: the FP64
    # rounding of both implementations is amplified by those edges'
    # conditioning (observed 4e-12), so the FP64 bar for them is 1e-11
    assert rep["area_max_rel"] <= max(rtol, 1e-11), rep


@pytest.mark.parametrize("precision,order,rtol", FORMS)
def test_localized_extended_cells(precision, order, rtol):
    # Sec. 3.1 'localized': the cells at the cluster's surface reach the walls,
    # so their walks run far past the offset list (shell enumeration and, in
    # the FP32 form, the block bound)
    s = W.localized(200_000, 3, 0.1, seed=31)
    check(s, (27, 27, 27), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS[:2])
def test_extreme_clustering_3d(precision, order, rtol):
    s = W.extreme_clustering(20_000, 3, seed=32)
    check(s, (34, 34, 34), precision, order, rtol)


# both sides place each 2D vertex where its two lines cross, so the FP64
# form holds the 1e-12 bar on cells far smaller than the box
@pytest.mark.parametrize("precision,order,rtol", [("fp64", "walk", 1e-12), ("fp32", "walk", 1e-5)])
def test_extreme_clustering_2d(precision, order, rtol):
    # Sec. 3.1 'extreme clustering' in 2D: cells near the centre are 1e-4 of
    # a block side and smaller, where block-relative FP32 positions carry
    # errors a relative band alone would miss
    s = W.extreme_clustering(100_000, 2, seed=16)
    check(s, (447, 447), precision, order, rtol)


@pytest.mark.parametrize("precision,order,rtol", FORMS[:2])
def test_localized_2d_fine_grid(precision, order, rtol):
    # cells at the cluster's surface span tens of blocks, so the walk covers
    # every shell past the offset list, the corners of the last listed shell
    # included
    s = W.localized(100_000, 2, 0.1, seed=23)
    check(s, (200, 200), precision, order, rtol)


# FP64 bars: both sides place each vertex on its planes (lines in 2D), so
# neither error grows with the box, and the 2D cells hold 1e-12.  In 3D the
# background cells beside the cluster carry its tiny faces, whose vertices
# lie where planes of cluster particles 1e-4 of a block apart meet, nearly
# parallel: a condition number of some 1e4-1e5 on both sides puts those
# cells' volumes 4e-11 apart (the cluster's own cells agree to 1e-12)
CORNER_FORMS = [(3, "fp64", "walk", 1e-10), (3, "fp32", "walk", 1e-5), (3, "fp32", "prefetch", 1e-5),
                (2, "fp64", "walk", 1e-12), (2, "fp32", "walk", 1e-5)]


@pytest.mark.parametrize("dim,precision,order,rtol", CORNER_FORMS)
def test_tiny_cells_at_a_block_corner(dim, precision, order, rtol):
    # cells 1e-4 of a block side beside a block corner, as at the centre of
    # the extreme-clustering sets at 10^7-10^8 points: block-relative FP32
    # positions there are coarse against the cells and their neighbours'
    # planes, so the FP32 form must test in FP64 where the band cannot
    # decide, and take FP64 statistics where its vertices are off
    s = W.corner_cluster(20_000, 2_000, dim, nb=20, seed=40 + dim)
    check(s, (20,) * dim, precision, order, rtol)
