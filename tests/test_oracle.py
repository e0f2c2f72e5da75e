"""Pins for the FP64 oracle: values and properties fixed by the paper or by
geometry, none of them computed by the oracle itself.

* closed-form cells of square, hexagonal, simple cubic, BCC and FCC lattices;
* a box split by one bisector (N=2, plain and radical), the whole box (N=1);
* qhull (scipy.spatial.Voronoi) on the same points plus their periodic
  images or wall reflections -- an independent Voronoi construction;
* Monte-Carlo nearest-site / least-power-distance assignment;
* partition of the box (the cells tile the container), Euler's formula,
  degree-3 vertices, neighbour symmetry, 2D torus mean of 6 edges;
* the paper's worked example (mean perimeter 0.01265 at N=10^5) and the
  Table 3 grid sizes;
* the grid walk (radius bound) equals the brute-force definition.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def faces_of(r, i):
    a, b = r["face_off"][i], r["face_off"][i + 1]
    return r["nbr_id"][a:b], r["nbr_img"][a:b], r["face_order"][a:b]


def neighbour_set(r, i):
    ids, imgs, _ = faces_of(r, i)
    return {(int(j), tuple(int(x) for x in m)) for j, m in zip(ids, imgs)}


# ---------------------------------------------------------------- lattices

def test_square_lattice_cells_are_squares():
    s = W.square(5, 0.5)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    assert np.all(r["status"] == 0)
    np.testing.assert_allclose(r["vol"], 0.25, rtol=1e-13)
    np.testing.assert_allclose(r["area"], 2.0, rtol=1e-13)      # perimeter 4d
    assert np.all(r["nv"] == 4) and np.all(r["nf"] == 4)
    np.testing.assert_allclose(r["centroid"], 0.0, atol=1e-13)


def test_hexagonal_lattice_cells_are_regular_hexagons():
    d = 0.25
    s = W.hexagonal(4, 4, (4 * d, 4 * d * math.sqrt(3) / 2))
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], math.sqrt(3) / 2 * d * d, rtol=1e-12)
    np.testing.assert_allclose(r["area"], 2 * math.sqrt(3) * d, rtol=1e-12)
    assert np.all(r["nv"] == 6)


def test_simple_cubic_cells_are_cubes():
    s = W.simple_cubic(3, 1.5)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], 1.5 ** 3, rtol=1e-13)
    np.testing.assert_allclose(r["area"], 6 * 1.5 ** 2, rtol=1e-13)
    assert np.all(r["nv"] == 8) and np.all(r["ne"] == 12) and np.all(r["nf"] == 6)


def test_bcc_cells_are_truncated_octahedra():
    a = 1.25
    s = W.bcc(3, a)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], a ** 3 / 2, rtol=1e-13)
    np.testing.assert_allclose(r["area"], (6 + 12 * math.sqrt(3)) * a * a / 8, rtol=1e-12)
    assert np.all(r["nv"] == 24) and np.all(r["ne"] == 36) and np.all(r["nf"] == 14)
    for i in range(s.n):
        _, _, order = faces_of(r, i)
        assert sorted(order.tolist()) == [4] * 6 + [6] * 8
    np.testing.assert_allclose(r["centroid"], 0.0, atol=1e-12)


def test_fcc_cells_are_rhombic_dodecahedra():
    a = 1.0
    s = W.fcc(3, a)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], a ** 3 / 4, rtol=1e-13)
    np.testing.assert_allclose(r["area"], 3 * math.sqrt(2) * a * a / 2, rtol=1e-12)
    # 14 vertices: 6 of degree 4 and 8 of degree 3 -> 24 edges, 12 rhombi
    assert np.all(r["nv"] == 14) and np.all(r["ne"] == 24) and np.all(r["nf"] == 12)
    assert np.all(r["face_order"] == 4)
    # the 12 neighbours are the nearest lattice points, at distance a/sqrt(2)
    for i in range(0, s.n, 7):
        for j, m in neighbour_set(r, i):
            q = s.pos[j] + np.array(m) * s.hi - s.pos[i]
            assert abs(np.linalg.norm(q) - a / math.sqrt(2)) < 1e-12


def test_perturbed_bcc_keeps_truncated_octahedra():
    s = W.bcc(4, 1.25, 0.02, seed=11)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(4, 4, 4))
    for i in range(s.n):
        _, _, order = faces_of(r, i)
        assert sorted(order.tolist()) == [4] * 6 + [6] * 8
    np.testing.assert_allclose(r["vol"].sum(), np.prod(s.hi), rtol=1e-12)


# -------------------------------------------------------- special cases

def test_two_particles_split_box_by_bisector():
    pos = np.array([[0.2, 0.3, 0.4], [0.7, 0.3, 0.4]])
    r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, method="brute")
    # bisector x = 0.45 ; cells are the slabs [0,0.45] and [0.45,1]
    np.testing.assert_allclose(r["vol"], [0.45, 0.55], rtol=1e-14)
    np.testing.assert_allclose(r["centroid"][0], [0.225 - 0.2, 0.5 - 0.3, 0.5 - 0.4], atol=1e-14)
    np.testing.assert_allclose(r["centroid"][1], [0.725 - 0.7, 0.2, 0.1], atol=1e-14)
    np.testing.assert_allclose(r["area"], [2 * 0.45 * 2 + 2, 2 * 0.55 * 2 + 2], rtol=1e-14)
    assert neighbour_set(r, 0) == {(-1, (0, 0, 0)), (-3, (0, 0, 0)), (-4, (0, 0, 0)),
                                   (-5, (0, 0, 0)), (-6, (0, 0, 0)), (1, (0, 0, 0))}


def test_two_particles_radical_plane_and_empty_cell():
    pos = np.array([[0.2, 0.5, 0.5], [0.7, 0.5, 0.5]])
    rad = np.array([0.3, 0.1])
    r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, radii=rad, method="brute")
    # power bisector: |x-0.2|^2 - 0.09 = |x-0.7|^2 - 0.01 -> x = (0.49-0.04+0.08)/1.0
    xs = (0.7 ** 2 - 0.2 ** 2 + 0.3 ** 2 - 0.1 ** 2) / (2 * (0.7 - 0.2))
    np.testing.assert_allclose(r["vol"], [xs, 1 - xs], rtol=1e-14)
    # a big radius swallows the other cell entirely: its cell does not exist
    rad2 = np.array([0.9, 0.05])
    r2 = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, radii=rad2, method="brute")
    xs2 = (0.7 ** 2 - 0.2 ** 2 + 0.9 ** 2 - 0.05 ** 2) / (2 * 0.5)
    assert xs2 > 1
    assert r2["status"][1] == oracle.ST_EMPTY and r2["vol"][1] == 0 and r2["nf"][1] == 0
    np.testing.assert_allclose(r2["vol"][0], 1.0, rtol=1e-14)


def test_single_particle_periodic_cell_is_the_box():
    pos = np.array([[0.3, 1.1, 0.2]])
    hi = np.array([1.0, 2.0, 0.5])
    r = oracle.compute(pos, [0, 0, 0], hi, (True,) * 3, method="brute")
    np.testing.assert_allclose(r["vol"], [1.0], rtol=1e-14)
    assert r["nf"][0] == 6
    assert neighbour_set(r, 0) == {(0, (-1, 0, 0)), (0, (1, 0, 0)), (0, (0, -1, 0)),
                                   (0, (0, 1, 0)), (0, (0, 0, -1)), (0, (0, 0, 1))}
    g = oracle.compute(pos, [0, 0, 0], hi, (True,) * 3, method="grid", nblocks=(1, 1, 1))
    np.testing.assert_allclose(g["vol"], [1.0], rtol=1e-14)


def test_single_particle_walled_cell_is_the_box():
    pos = np.array([[0.3, 0.6, 0.2]])
    r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, method="brute")
    np.testing.assert_allclose(r["vol"], [1.0], rtol=1e-14)
    np.testing.assert_allclose(r["centroid"][0], [0.2, -0.1, 0.3], atol=1e-14)
    assert r["nf"][0] == 6 and r["nv"][0] == 8


def test_equal_radii_radical_equals_voronoi():
    s = W.uniform(150, 3, 2.0, True, seed=21)
    a = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(3, 3, 3))
    b = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=np.full(s.n, 0.37),
                       method="grid", nblocks=(3, 3, 3))
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-12)
    assert np.array_equal(a["nbr_id"], b["nbr_id"]) and np.array_equal(a["nbr_img"], b["nbr_img"])


# ----------------------------------------------- independent construction

def _qhull_cells(pts_aug, n, dim):
    from scipy.spatial import ConvexHull, Voronoi
    vor = Voronoi(pts_aug)
    vols, nbrs = [], []
    for i in range(n):
        reg = vor.regions[vor.point_region[i]]
        assert -1 not in reg
        vols.append(ConvexHull(vor.vertices[reg]).volume)
    rp = vor.ridge_points
    for i in range(n):
        m = (rp[:, 0] == i) | (rp[:, 1] == i)
        other = np.where(rp[m, 0] == i, rp[m, 1], rp[m, 0])
        nbrs.append(other)
    return np.array(vols), nbrs


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_cells_match_qhull(dim):
    n = 120 if dim == 3 else 200
    s = W.uniform(n, dim, 3.0, True, seed=31 + dim)
    shifts = np.array(np.meshgrid(*([[0, -1, 1]] * dim), indexing="ij")).reshape(dim, -1).T
    aug = np.concatenate([s.pos + sh * s.hi for sh in shifts], axis=0)
    vols, nbrs = _qhull_cells(aug, n, dim)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], vols, rtol=1e-10)
    for i in range(n):
        want = {(int(k % n), tuple(int(x) for x in shifts[k // n])) for k in nbrs[i]}
        got = {(j, m[:dim]) for j, m in neighbour_set(r, i)}
        assert got == want, i


@pytest.mark.parametrize("dim", [2, 3])
def test_walled_cells_match_qhull_with_reflections(dim):
    # Reflecting every point in each wall adds the walls as bisectors and
    # leaves the cells inside the box unchanged.
    n = 150
    s = W.uniform(n, dim, 1.0, False, seed=41 + dim)
    aug = [s.pos]
    for a in range(dim):
        for side in (0, 1):
            ref = s.pos.copy()
            ref[:, a] = 2 * side * s.hi[a] - ref[:, a]
            aug.append(ref)
    aug = np.concatenate(aug, axis=0)
    vols, nbrs = _qhull_cells(aug, n, dim)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    np.testing.assert_allclose(r["vol"], vols, rtol=1e-10)
    for i in range(n):
        want = set()
        for k in nbrs[i]:
            if k < n:
                want.add((int(k), (0,) * dim))
            else:
                blk = k // n - 1           # reflection a*2+side
                assert k % n == i           # only a particle's own mirror touches it
                want.add((-(1 + blk), (0,) * dim))
        got = {(j, m[:dim]) for j, m in neighbour_set(r, i)}
        assert got == want, i


@pytest.mark.parametrize("radical", [False, True])
def test_monte_carlo_assignment(radical):
    # Each cell is the set of points whose nearest site (least power distance
    # for the radical variant) is its particle; sample and count.
    rng = np.random.default_rng(7)
    n = 40
    s = W.uniform(n, 3, 1.0, True, seed=51)
    rad = rng.uniform(0.02, 0.12, n) if radical else None
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=rad, method="brute")
    M = 400_000
    x = rng.random((M, 3))
    best = np.full(M, np.inf)
    owner = np.zeros(M, dtype=np.int64)
    w = np.zeros(n) if rad is None else rad ** 2
    for i in range(n):
        dx = x - s.pos[i]
        dx -= np.round(dx)
        pd = np.sum(dx * dx, axis=1) - w[i]
        better = pd < best
        best[better] = pd[better]
        owner[better] = i
    frac = np.bincount(owner, minlength=n) / M
    sd = np.sqrt(np.maximum(r["vol"] * (1 - r["vol"]), 1e-12) / M)
    assert np.all(np.abs(frac - r["vol"]) < 6 * sd + 1e-6)


# ----------------------------------------------------------- invariants

@pytest.mark.parametrize("periodic", [False, True])
def test_generic_3d_invariants(periodic):
    s = W.uniform(600, 3, 5.0, periodic, seed=61)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(5, 5, 5))
    assert np.all(r["status"] == 0)
    np.testing.assert_allclose(r["vol"].sum(), 125.0, rtol=1e-12)
    assert np.all(r["nv"] - r["ne"] + r["nf"] == 2)
    assert np.all(2 * r["ne"] == 3 * r["nv"])       # every vertex has degree 3
    for i in range(s.n):
        for j, m in neighbour_set(r, i):
            if j >= 0:
                assert (i, tuple(-x for x in m)) in neighbour_set(r, j)
    # face orders sum to twice the edges
    for i in range(s.n):
        _, _, order = faces_of(r, i)
        assert order.sum() == 2 * r["ne"][i]


def test_2d_torus_mean_edges_is_six():
    s = W.hexagonal(24, 28, (1.0, 1.0), 0.05, seed=3)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid")
    assert r["nv"].sum() == 6 * s.n
    np.testing.assert_allclose(r["vol"].sum(), 1.0, rtol=1e-12)


def test_radical_partition_with_empty_cells():
    s = W.radical_uniform(800, packing=0.4, sigma=0.6, seed=71)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, method="grid",
                       nblocks=(2, 2, 2))
    assert set(np.unique(r["status"])) <= {0, 1}
    np.testing.assert_allclose(r["vol"].sum(), np.prod(s.hi), rtol=1e-11)
    assert np.all(r["vol"][r["status"] == 1] == 0)


# ------------------------------------------------- grid walk = definition

@pytest.mark.parametrize("case", ["walled3", "periodic3", "mixed3", "walled2", "periodic2",
                                  "radical3", "tiny_periodic"])
def test_grid_walk_equals_brute_force(case):
    rad = None
    if case == "walled3":
        s, nb = W.uniform(300, 3, 1.0, False, 81), (4, 4, 4)
    elif case == "periodic3":
        s, nb = W.uniform(300, 3, 1.0, True, 82), (4, 4, 4)
    elif case == "mixed3":
        s, nb = W.uniform(300, 3, 1.0, False, 83), (3, 5, 4)
        s.periodic = (True, False, True)
    elif case == "walled2":
        s, nb = W.uniform(400, 2, 1.0, False, 84), (7, 5)
    elif case == "periodic2":
        s, nb = W.uniform(400, 2, 1.0, True, 85), (6, 6)
    elif case == "radical3":
        s, nb = W.radical_uniform(300, 0.4, 0.3, 86), (3, 3, 3)
        rad = s.radii
    else:
        s, nb = W.uniform(3, 3, 1.0, True, 87), (2, 2, 2)
    a = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=rad, method="brute")
    b = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=rad, method="grid", nblocks=nb)
    assert np.array_equal(a["status"], b["status"])
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-12, atol=1e-15)
    assert np.array_equal(a["face_off"], b["face_off"])
    assert np.array_equal(a["nbr_id"], b["nbr_id"])
    assert np.array_equal(a["nbr_img"], b["nbr_img"])
    assert np.array_equal(a["face_order"], b["face_order"])


# ------------------------------------------------------- paper's numbers

def test_table3_grid_sizes():
    for dim, n, nopt, want in _golden("table3_grid_sizes.txt"):
        dim = int(dim)
        got = oracle.grid_size(int(n), np.zeros(dim), np.ones(dim), nopt, "floor")
        assert got == (int(want),) * dim
        # the ceiling the text states is one more for all of these
        got_c = oracle.grid_size(int(n), np.zeros(dim), np.ones(dim), nopt, "ceil")
        assert got_c == (int(want) + 1,) * dim


@pytest.mark.slow
def test_worked_example_mean_perimeter():
    (n, nb, want, tol), = _golden("mean_perimeter_2d.txt")
    n, nb = int(n), int(nb)
    vals = []
    for seed in range(3):
        s = W.uniform(n, 2, 1.0, True, seed=100 + seed)
        r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(nb, nb))
        assert np.all(r["status"] == 0)
        vals.append(r["area"].mean())
    # the sampling spread of the mean over 10^5 cells is ~1e-6, below the
    # 5e-6 rounding of the printed digits
    for v in vals:
        assert abs(v - want) <= 0.5 * tol
    assert abs(np.mean(vals) - 4 / math.sqrt(n)) < 2e-5


def test_poisson_block_occupancy_fractions():
    # the paper's percentages follow from Pois(n_opt); reproduce them from
    # the oracle's block sort of uniform points
    from scipy.stats import poisson
    for dim, nopt, fb, fp in _golden("poisson_block_occupancy.txt"):
        dim = int(dim)
        assert abs(poisson.sf(8, nopt) - fb) < 5e-5
        over = sum((k - 8) * poisson.pmf(k, nopt) for k in range(9, 60)) / nopt
        # printed to two decimals of a percent (3D: 1.6665 % appears as 1.66 %)
        assert abs(over - fp) < 1e-4
        n = 2_000_000
        s = W.uniform(n, dim, 1.0, False, seed=90 + dim)
        nb = oracle.grid_size(n, s.lo, s.hi, nopt, "floor")
        order, start = oracle.block_sort(s.pos, s.lo, s.hi, nb)
        counts = np.diff(start)
        actual_nopt = n / counts.size
        assert abs((counts > 8).mean() - poisson.sf(8, actual_nopt)) < 0.002
        assert np.array_equal(np.sort(order), np.arange(n))


def test_3d_poisson_voronoi_mean_faces():
    # Literature constants for 3D Poisson-Voronoi cells (not from the paper):
    # mean faces 2 + 48 pi^2 / 35, mean vertices 96 pi^2 / 35.
    s = W.uniform(20000, 3, 20000 ** (1 / 3), True, seed=95)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid")
    assert abs(r["nf"].mean() - (2 + 48 * math.pi ** 2 / 35)) < 0.12
    assert abs(r["nv"].mean() - 96 * math.pi ** 2 / 35) < 0.25
