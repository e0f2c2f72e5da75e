"""The parity comparison itself (tests/compare.py), on oracle output: equal
results compare clean, and each planted difference is counted once."""
import copy

import numpy as np

import oracle
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare


def _ref():
    s = W.uniform(300, 3, 1.0, True, seed=3)
    return oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(4, 4, 4))


def test_identical_results_compare_clean():
    r = _ref()
    rep = compare(r, r, 1e-15)
    assert rep["topology_ok"] and rep["values_ok"]
    assert rep["vol_max_rel"] == 0.0 and rep["face_mismatch"] == 0


def test_planted_differences_are_counted():
    r = _ref()
    g = copy.deepcopy(r)
    a = g["face_off"][7]
    g["nbr_id"][a] += 1                      # one neighbour id in cell 7
    b = g["face_off"][20]
    g["nbr_img"][b + 1, 2] += 1              # one image shift in cell 20
    g["face_order"][g["face_off"][41]] += 1  # one face order in cell 41
    g["vol"][5] *= 1 + 3e-6
    rep = compare(g, r, 1e-5)
    assert rep["face_mismatch"] == 3 and not rep["topology_ok"]
    assert abs(rep["vol_max_rel"] - 3e-6) < 1e-9 and rep["values_ok"]
    g["nf"][9] += 1
    assert compare(g, r, 1e-5)["nf_mismatch"] == 1


def test_subset_of_cells():
    s = W.uniform(300, 3, 1.0, True, seed=3)
    full = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(4, 4, 4))
    cells = np.array([3, 50, 51, 299])
    part = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(4, 4, 4), cells=cells)
    rep = compare(full, part, 1e-15, cells=cells)
    assert rep["topology_ok"] and rep["values_ok"]
