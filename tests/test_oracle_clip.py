"""Pins for clipped cells (Sec. 3.1.3): every cell starts from the box
intersected with a cube (2D: square) of side h centred on its particle, and
the cube's faces count as walls.  The expected values are closed forms of
elementary geometry, not computed by the oracle."""
import math

import numpy as np

import oracle
from paper_2209_11606_gb300 import workloads as W


def test_lone_particle_gives_the_cube():
    pos = np.array([[0.5, 0.4, 0.55]])
    for method in ("brute", "grid"):
        r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, method=method,
                           nblocks=(3, 3, 3), clip=0.3)
        np.testing.assert_allclose(r["vol"], [0.027], rtol=1e-14)
        np.testing.assert_allclose(r["area"], [6 * 0.09], rtol=1e-14)
        np.testing.assert_allclose(r["centroid"][0], 0.0, atol=1e-15)
        assert r["nv"][0] == 8 and r["ne"][0] == 12 and r["nf"][0] == 6
        assert r["nbr_id"].tolist() == [-6, -5, -4, -3, -2, -1]


def test_cube_is_cut_by_the_box_near_a_wall():
    # particle 0.1 from the x- wall, cube side 0.4: x spans [-0.1, 0.2]
    pos = np.array([[0.1, 0.5, 0.5]])
    r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (False,) * 3, method="brute", clip=0.4)
    np.testing.assert_allclose(r["vol"], [0.3 * 0.4 * 0.4], rtol=1e-14)
    np.testing.assert_allclose(r["centroid"][0], [0.05, 0.0, 0.0], atol=1e-15)


def test_periodic_axis_is_clipped_by_walls():
    # a lone particle on a unit torus: its cell is the whole period until the
    # cube is smaller than the period, then the cube, with wall faces
    pos = np.array([[0.2, 0.7, 0.9]])
    r = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (True,) * 3, method="brute", clip=0.5)
    np.testing.assert_allclose(r["vol"], [0.125], rtol=1e-14)
    assert (r["nbr_id"] < 0).all() and r["nf"][0] == 6
    big = oracle.compute(pos, [0, 0, 0], [1, 1, 1], (True,) * 3, method="brute", clip=3.0)
    np.testing.assert_allclose(big["vol"], [1.0], rtol=1e-14)
    assert (big["nbr_id"] == 0).all()


def test_clip_larger_than_the_cells_changes_nothing():
    s = W.uniform(300, 3, 1.0, False, seed=3)
    a = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute")
    b = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", clip=10.0)
    for k in ("vol", "area", "nv", "ne", "nf", "nbr_id", "face_order"):
        np.testing.assert_array_equal(a[k], b[k])


def test_simple_cubic_lattice_below_and_above_the_spacing():
    s = W.simple_cubic(4, 1.0)
    small = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", clip=0.6)
    np.testing.assert_allclose(small["vol"], 0.216, rtol=1e-13)
    assert (small["nbr_id"] < 0).all()
    large = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", clip=1.5)
    np.testing.assert_allclose(large["vol"], 1.0, rtol=1e-13)
    assert (large["nbr_id"] >= 0).all()


def test_bcc_cell_clipped_by_a_cube():
    # BCC, a = 1: hexagonal faces on the planes |x|+|y|+|z| = 3/4 (the eight
    # nearest neighbours), square faces at 1/2.  A cube of side 0.7 keeps
    # none of the squares, and each hexagon plane cuts a corner tetrahedron
    # with legs 3 (0.35) - 0.75 = 0.3 (the eight corners stay disjoint):
    # V = 0.7^3 - 8 (0.3^3 / 6); faces: 6 octagons (walls) and 8 equilateral
    # triangles of side 0.3 sqrt 2; 24 vertices and 36 edges.
    s = W.bcc(3, 1.0)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", clip=0.7)
    np.testing.assert_allclose(r["vol"], 0.7 ** 3 - 8 * 0.3 ** 3 / 6, rtol=1e-13)
    octagon = 0.7 ** 2 - 4 * 0.3 ** 2 / 2
    triangle = math.sqrt(3) / 4 * (0.3 * math.sqrt(2)) ** 2
    np.testing.assert_allclose(r["area"], 6 * octagon + 8 * triangle, rtol=1e-12)
    assert np.all(r["nv"] == 24) and np.all(r["ne"] == 36) and np.all(r["nf"] == 14)
    for i in range(s.n):
        a, b = r["face_off"][i], r["face_off"][i + 1]
        ids, order = r["nbr_id"][a:b], r["face_order"][a:b]
        assert sorted(order[ids < 0].tolist()) == [8] * 6
        assert sorted(order[ids >= 0].tolist()) == [3] * 8
    g = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(3, 3, 3), clip=0.7)
    np.testing.assert_allclose(g["vol"], r["vol"], rtol=1e-13)


def test_square_lattice_clipped_2d():
    s = W.square(5, 1.0)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", clip=0.8)
    np.testing.assert_allclose(r["vol"], 0.64, rtol=1e-13)    # 2D: area
    np.testing.assert_allclose(r["area"], 3.2, rtol=1e-13)    # 2D: perimeter
    assert (r["nbr_id"] < 0).all() and np.all(r["nf"] == 4)
