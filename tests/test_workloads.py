"""Synthetic inputs, and the oracle on the one built to stress FP32 inputs.

`corner_cluster` puts cells 1e-4 of a block beside a block corner.  The
FP64 bar of its GPU parity test (1e-7) rests on the oracle being exact there
up to its own rounding, so the oracle's cells of the cluster are checked
against exact rational arithmetic: each cell clipped (Eq. 3) by every point
within 2.5 R of its particle, R the oracle's largest vertex distance (a
point beyond 2R cannot cut, Sec. 2.1.3)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W


def test_corner_cluster_shape():
    for dim in (2, 3):
        s = W.corner_cluster(2000, 300, dim, nb=20, width=2e-3, seed=5)
        assert s.pos.shape == (2300, dim) and s.n == 2300
        assert np.all((s.pos >= 0) & (s.pos < 1))
        cl = s.pos[2000:]
        # the cluster: a cube 2e-3 block sides across around the corner (0.5, ...)
        assert np.all(np.abs(cl - 0.5) <= 0.5 * 2e-3 / 20)
        assert np.abs(cl - 0.5).max() > 0.4 * 2e-3 / 20
        assert not s.periodic[0] and s.radii is None


def _exact_cell_2d(pos, i, lo, hi, cand):
    """Exact polygon of cell i in the box, clipped by the bisectors of cand."""
    p = [Fraction(float(x)) for x in pos[i]]
    poly = [(Fraction(lo[0]) - p[0], Fraction(lo[1]) - p[1]), (Fraction(hi[0]) - p[0], Fraction(lo[1]) - p[1]),
            (Fraction(hi[0]) - p[0], Fraction(hi[1]) - p[1]), (Fraction(lo[0]) - p[0], Fraction(hi[1]) - p[1])]
    cutters = set()
    for j in cand:
        if j == i:
            continue
        q = [Fraction(float(x)) for x in pos[j]]
        nx, ny = q[0] - p[0], q[1] - p[1]
        c = (nx * nx + ny * ny) / 2
        out, cut = [], False
        for k in range(len(poly)):
            a, b = poly[k], poly[(k + 1) % len(poly)]
            da, db = nx * a[0] + ny * a[1] - c, nx * b[0] + ny * b[1] - c
            if da <= 0:
                out.append(a)
            else:
                cut = True
            if (da < 0 < db) or (db < 0 < da):
                t = da / (da - db)
                out.append((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
        poly = out
        if cut:
            cutters.add(int(j))
    area = sum(poly[k][0] * poly[(k + 1) % len(poly)][1] - poly[(k + 1) % len(poly)][0] * poly[k][1]
               for k in range(len(poly))) / 2
    # the neighbours: points whose bisector holds an edge of the final polygon
    nbrs = set()
    for j in cutters:
        q = [Fraction(float(x)) for x in pos[j]]
        nx, ny = q[0] - p[0], q[1] - p[1]
        c = (nx * nx + ny * ny) / 2
        on = [v for v in poly if nx * v[0] + ny * v[1] == c]
        if len(on) >= 2:
            nbrs.add(j)
    return float(area), nbrs


def test_oracle_exact_on_corner_cluster_cells_2d():
    s = W.corner_cluster(20_000, 2_000, 2, nb=20, seed=42)
    cells = np.arange(20_000, 22_000, 250)  # eight cells of the cluster
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(20, 20), cells=cells)
    for k, i in enumerate(cells):
        R = r["rmax"][k]
        d = np.linalg.norm(s.pos - s.pos[i], axis=1)
        cand = np.nonzero(d < 2.5 * R)[0]
        area, nbrs = _exact_cell_2d(s.pos, i, s.lo, s.hi, cand[np.argsort(d[cand])])
        got = set(r["nbr_id"][r["face_off"][k]:r["face_off"][k + 1]].tolist())
        assert got == nbrs, (i, got, nbrs)
        # the oracle places each new vertex where its two lines cross, so
        # its error is relative to the cell (interpolating along the edge,
        # at first as long as the box, was off by some 1e-10 here)
        assert abs(r["vol"][k] - area) <= 1e-14 * area, (i, r["vol"][k], area)
    # inside the cluster the cells are 1e-4 of a block (20 blocks per side);
    # one at its edge reaches out into the background
    assert np.median(r["rmax"]) < 1e-4 / 20 and r["rmax"].max() < 1e-2 / 20


def test_oracle_matches_qhull_on_corner_cluster_cells_3d():
    # an independent method for the 3D cells of the cluster: qhull's Voronoi
    # diagram (its vertices in box coordinates, good to about 1e-10 of these
    # cells) and the convex hull volume of each cell's vertices
    spatial = pytest.importorskip("scipy.spatial")
    s = W.corner_cluster(20_000, 2_000, 3, nb=20, seed=43)
    cells = np.arange(20_000, 22_000, 250)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(20, 20, 20), cells=cells)
    vor = spatial.Voronoi(s.pos)
    ridges = {}
    for (p, q) in vor.ridge_points:
        ridges.setdefault(int(p), set()).add(int(q))
        ridges.setdefault(int(q), set()).add(int(p))
    checked = 0
    for k, i in enumerate(cells):
        region = vor.regions[vor.point_region[i]]
        if -1 in region or r["rmax"][k] > 1e-3 / 20:
            continue  # only cells inside the cluster (1e-4 of a block), far from every wall
        vol = spatial.ConvexHull(vor.vertices[region]).volume
        got = set(r["nbr_id"][r["face_off"][k]:r["face_off"][k + 1]].tolist())
        assert got == ridges[int(i)], (i, got ^ ridges[int(i)])
        assert abs(r["vol"][k] - vol) <= 1e-7 * vol, (i, r["vol"][k], vol)
        checked += 1
    assert checked >= 5
