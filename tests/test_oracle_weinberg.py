"""Pins for the oracle's Weinberg codes (Sec. 4): closed forms for regular
cells, and for random cells an independent construction -- the cell's edge
graph from qhull (scipy.spatial.Voronoi) and networkx's isomorphism and
automorphism search.  A cell's edge graph is 3-connected and planar, so two
cells have the same minimal code iff their graphs are isomorphic, and the
number of (start dart, orientation) pairs reaching the minimal code equals
the number of graph automorphisms (Whitney: the embedding is unique up to
mirror image)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W


def test_box_cell_is_the_cube_code():
    r = oracle.compute(np.array([[0.5, 0.5, 0.5]]), [0, 0, 0], [1, 1, 1], (False,) * 3, method="brute",
                       weinberg=True)
    assert r["w_len"][0] == 24 and r["w_sym"][0] == 48  # 12 edges; |O_h| = 48


def test_lattice_cells_share_one_code_with_full_symmetry():
    for s, darts in ((W.bcc(3, 1.0), 72), (W.fcc(3, 1.0), 48), (W.simple_cubic(3, 1.0), 24)):
        r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", weinberg=True)
        assert np.all(r["w_len"] == darts)
        assert np.all(r["w_sym"] == 48)
        assert len(np.unique(r["w_hash"])) == 1
    # three different polyhedra, three different codes
    codes = [oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="brute", weinberg=True)["w_hash"][0]
             for s in (W.bcc(3, 1.0), W.fcc(3, 1.0), W.simple_cubic(3, 1.0))]
    assert len(set(codes)) == 3


def test_perturbed_bcc_keeps_the_truncated_octahedron_code():
    ref = oracle.compute(*_sys(W.bcc(3, 1.0)), method="brute", weinberg=True)["w_hash"][0]
    s = W.bcc(4, 1.0, 0.02, seed=5)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=(4, 4, 4), weinberg=True)
    assert np.all(r["w_hash"] == ref)


def _sys(s):
    return s.pos, s.lo, s.hi, s.periodic


def _qhull_graphs(pos, cells):
    spatial = pytest.importorskip("scipy.spatial")
    vor = spatial.Voronoi(pos)
    ridges = {}
    for (p, q), rv in zip(vor.ridge_points, vor.ridge_vertices):
        ridges.setdefault(p, []).append(rv)
        ridges.setdefault(q, []).append(rv)
    nx = pytest.importorskip("networkx")
    out = {}
    for i in cells:
        g = nx.Graph()
        for rv in ridges[i]:
            assert -1 not in rv
            for a, b in zip(rv, rv[1:] + rv[:1]):
                g.add_edge(a, b)
        out[i] = g
    return out


def test_codes_match_graph_isomorphism_and_automorphisms():
    nx = pytest.importorskip("networkx")
    s = W.uniform(3000, 3, 1.0, False, seed=17)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", weinberg=True)
    # cells with no wall face: their qhull cells are the same polyhedra
    inner = [i for i in range(s.n)
             if (r["nbr_id"][r["face_off"][i]:r["face_off"][i + 1]] >= 0).all()][:400]
    graphs = _qhull_graphs(s.pos, inner)
    for i in inner[:150]:
        g = graphs[i]
        assert 2 * g.number_of_edges() == r["w_len"][i]
        auts = sum(1 for _ in nx.algorithms.isomorphism.GraphMatcher(g, g).isomorphisms_iter())
        assert auts == r["w_sym"][i], (i, auts, r["w_sym"][i])
    # same code iff isomorphic, on pairs with equal vertex and edge counts
    groups = {}
    for i in inner:
        groups.setdefault((graphs[i].number_of_nodes(), graphs[i].number_of_edges()), []).append(i)
    checked = 0
    for members in groups.values():
        for i, j in itertools.islice(itertools.combinations(members, 2), 60):
            same = r["w_hash"][i] == r["w_hash"][j]
            assert same == nx.is_isomorphic(graphs[i], graphs[j]), (i, j)
            checked += 1
    assert checked > 100
