"""Weinberg codes (Sec. 4) on the GPU against the oracle's: darts, hash of
the minimal code and symmetry count bit-exact for every cell whose edge
graph has only degree-3 vertices (the cells the GPU codes), and such cells
are exactly the ones the GPU codes."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()


def codes(s, nb, order="prefetch", precision="fp32"):
    from paper_2209_11606_gb300 import vorogpu
    got = vorogpu.compute_host(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, nblocks=nb, precision=precision,
                               order=order, weinberg=1)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii, method="grid", nblocks=got["grid"],
                         weinberg=True)
    return got, ref


def check(got, ref):
    ok = (ref["status"] == 0) & (got["status"] == 0)
    simple = ok & (ref["w_len"] == 3 * ref["nv"])  # every vertex of degree 3: 2E = 3V
    coded = got["w_len"] > 0
    assert np.array_equal(coded[ok], simple[ok])
    for k in ("w_len", "w_hash", "w_sym"):
        np.testing.assert_array_equal(got[k][simple], ref[k][simple])
    return simple


@pytest.mark.parametrize("order,precision", [("prefetch", "fp32"), ("walk", "fp32"), ("walk", "fp64")])
def test_uniform_periodic_codes(order, precision):
    s = W.uniform(3000, 3, 3000 ** (1 / 3), True, seed=41)
    got, ref = codes(s, (8, 8, 8), order, precision)
    simple = check(got, ref)
    assert simple.sum() > 2900
    assert len(np.unique(got["w_hash"][simple])) > 100  # many distinct topologies


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_walled_codes(precision):
    s = W.uniform(2000, 3, 1.0, False, seed=42)
    got, ref = codes(s, (7, 7, 7), "walk" if precision == "fp64" else "prefetch", precision)
    check(got, ref)


def test_perturbed_bcc_is_one_topology():
    s = W.bcc(6, 1.0, 0.02, seed=43)
    got, ref = codes(s, (6, 6, 6))
    simple = check(got, ref)
    assert simple.all()
    assert len(np.unique(got["w_hash"])) == 1 and np.all(got["w_sym"] == 48) and np.all(got["w_len"] == 72)


def test_lone_cell_is_the_cube():
    s = W.uniform(1, 3, 1.0, False, seed=44)
    got, ref = codes(s, (1, 1, 1))
    assert got["w_len"][0] == 24 and got["w_sym"][0] == 48 and got["w_hash"][0] == ref["w_hash"][0]


def test_weinberg_needs_3d():
    from paper_2209_11606_gb300 import vorogpu
    s = W.uniform(100, 2, 1.0, False, seed=45)
    with pytest.raises(vorogpu.VgError):
        vorogpu.compute_host(s.pos, s.lo, s.hi, s.periodic, nblocks=(2, 2), weinberg=1)
