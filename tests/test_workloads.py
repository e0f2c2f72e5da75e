"""Synthetic inputs, and the oracle on the one built to stress FP32 inputs.

`corner_cluster` puts cells 1e-4 of a block beside a block corner.  The
FP64 bars of its GPU parity test rest on the oracle being exact there up to
its own rounding, so the oracle's cells of the cluster are checked against
exact rational arithmetic (Eq. 3, the bisector half-spaces, with every
point within 2.05-2.5 R of the particle, R the oracle's largest vertex
distance: a point beyond 2R cannot cut, Sec. 2.1.3): in 2D by clipping the
box polygon, in 3D by enumerating the points of plane triples that satisfy
every half-space."""
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


def _exact_cell_3d(pos, i, lo, hi, cand):
    """Exact volume and neighbours of cell i in the walled box, clipped by
    the bisectors of cand (Eq. 3): every vertex is the point of three planes
    that satisfies all of them (triples prefiltered in floating point, then
    solved and checked exactly); each plane holding three or more vertices
    is a face, whose vertices are put in angular order about its normal and
    summed as pyramids from the particle."""
    import itertools
    from functools import cmp_to_key
    p = [Fraction(float(x)) for x in pos[i]]
    planes = []  # (normal, constant, id): the cell is n.x <= c (x relative to p)
    for a in range(3):
        e = [Fraction(0)] * 3
        e[a] = Fraction(1)
        planes.append((tuple(e), Fraction(hi[a]) - p[a], -(1 + 2 * a + 1)))
        planes.append((tuple(-x for x in e), p[a] - Fraction(lo[a]), -(1 + 2 * a)))
    for j in cand:
        if j == i:
            continue
        r = tuple(Fraction(float(x)) - p[k] for k, x in enumerate(pos[j]))
        planes.append((r, sum(x * x for x in r) / 2, int(j)))
    nf = np.array([[float(x) for x in n] for n, _, _ in planes])
    cf = np.array([float(c) for _, c, _ in planes])
    tri = np.array(list(itertools.combinations(range(len(planes)), 3)))
    A = nf[tri]
    det = np.linalg.det(A)
    good = np.abs(det) > 1e-30 * np.abs(A).max(axis=(1, 2)) ** 3
    xs = np.full((len(tri), 3), np.nan)
    xs[good] = np.linalg.solve(A[good], cf[tri[good]][..., None])[..., 0]
    scale = np.abs(xs).max(axis=1, keepdims=True)
    near = good & np.all(nf @ np.nan_to_num(xs).T - cf[:, None] <= 1e-6 * scale.T * np.abs(nf).sum(axis=1)[:, None],
                         axis=0)

    def solve(t):
        (n1, c1, _), (n2, c2, _), (n3, c3, _) = (planes[k] for k in t)
        def cross(u, v):
            return (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        a23, a31, a12 = cross(n2, n3), cross(n3, n1), cross(n1, n2)
        d = sum(n1[k] * a23[k] for k in range(3))
        if d == 0:
            return None
        return tuple((c1 * a23[k] + c2 * a31[k] + c3 * a12[k]) / d for k in range(3))

    verts = set()
    for t in tri[near]:
        x = solve(t)
        if x is not None and all(sum(n[k] * x[k] for k in range(3)) <= c for n, c, _ in planes):
            verts.add(x)
    verts = list(verts)
    vol, nbrs = Fraction(0), set()
    for n, c, pid in planes:
        on = [v for v in verts if sum(n[k] * v[k] for k in range(3)) == c]
        if len(on) < 3:
            continue
        g = tuple(sum(v[k] for v in on) / len(on) for k in range(3))
        w = [tuple(v[k] - g[k] for k in range(3)) for v in on]

        def trip(u, v):
            cr = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
            return sum(n[k] * cr[k] for k in range(3))
        u0 = w[0]

        def half(v):  # 0: angle in [0, pi) from u0 about n, 1: [pi, 2 pi)
            s = trip(u0, v)
            if s > 0:
                return 0
            if s < 0:
                return 1
            return 0 if sum(u0[k] * v[k] for k in range(3)) > 0 else 1

        def cmp(a, b):
            ha, hb = half(w[a]), half(w[b])
            if ha != hb:
                return ha - hb
            s = trip(w[a], w[b])
            return -1 if s > 0 else (1 if s < 0 else 0)
        order = sorted(range(len(on)), key=cmp_to_key(cmp))
        poly = [on[k] for k in order]
        fv = Fraction(0)
        for k in range(1, len(poly) - 1):
            a, b, cc = poly[0], poly[k], poly[k + 1]
            fv += (a[0] * (b[1] * cc[2] - b[2] * cc[1]) - a[1] * (b[0] * cc[2] - b[2] * cc[0]) +
                   a[2] * (b[0] * cc[1] - b[1] * cc[0]))
        if fv != 0 and pid >= 0:
            nbrs.add(pid)
        vol += fv
    return float(vol / 6), nbrs


def test_oracle_exact_on_corner_cluster_cells_3d():
    # the oracle solves each vertex from its three planes, so its cells of
    # the cluster (1e-4 of a block, beside a block corner) carry no error
    # that grows with the box: exact arithmetic on four of them
    s = W.corner_cluster(20_000, 2_000, 3, nb=20, seed=43)
    # four cells from inside the cluster (their candidates within 2R stay few)
    centre = np.full(3, 0.5)
    inner = 20_000 + np.argsort(np.linalg.norm(s.pos[20_000:] - centre, axis=1))[:40:10]
    cells = np.sort(inner)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(20, 20, 20), cells=cells)
    for k, i in enumerate(cells):
        R = r["rmax"][k]
        d = np.linalg.norm(s.pos - s.pos[i], axis=1)
        cand = np.nonzero(d < 2.05 * R)[0]
        assert len(cand) < 80, len(cand)
        vol, nbrs = _exact_cell_3d(s.pos, i, s.lo, s.hi, cand)
        got = set(r["nbr_id"][r["face_off"][k]:r["face_off"][k + 1]].tolist())
        assert got == nbrs, (i, got, nbrs)
        assert abs(r["vol"][k] - vol) <= 1e-13 * vol, (i, r["vol"][k], vol)


def test_oracle_exact_on_uniform_cells_3d():
    # ordinary cells of a walled uniform set, one of them against walls
    s = W.uniform(3000, 3, 1.0, False, seed=44)
    corner = int(np.argmin(np.linalg.norm(s.pos, axis=1)))
    cells = np.sort(np.array([corner, 1000, 2000]))
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(8, 8, 8), cells=cells)
    for k, i in enumerate(cells):
        R = r["rmax"][k]
        d = np.linalg.norm(s.pos - s.pos[i], axis=1)
        cand = np.nonzero(d < 2.05 * R)[0]
        assert len(cand) < 80, len(cand)
        vol, nbrs = _exact_cell_3d(s.pos, i, s.lo, s.hi, cand)
        got = {x for x in r["nbr_id"][r["face_off"][k]:r["face_off"][k + 1]].tolist() if x >= 0}
        assert got == nbrs, (i, got, nbrs)
        assert abs(r["vol"][k] - vol) <= 1e-13 * vol, (i, r["vol"][k], vol)
