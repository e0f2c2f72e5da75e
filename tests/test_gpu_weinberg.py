"""Weinberg codes (Sec. 4) on the GPU against the oracle's: darts, hash of
the minimal code and symmetry count bit-exact for every cell the GPU codes.
The GPU codes every complete cell of up to 64 triangles: cells whose edge
graph has only degree-3 vertices, and cells of exact lattices whose
coincident vertices merge into vertices of degree 4 or more (FCC, simple
cubic), in the FP32 and the FP64 form."""
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
    assert not np.any(coded & ~ok)
    assert np.all(coded[simple])  # every simple cell is coded
    for k in ("w_len", "w_hash", "w_sym"):
        np.testing.assert_array_equal(got[k][coded], ref[k][coded])
    return coded


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


@pytest.mark.parametrize("order,precision", [("prefetch", "fp32"), ("walk", "fp64")])
@pytest.mark.parametrize("lattice,darts", [("fcc", 48), ("simple_cubic", 24), ("bcc", 72)])
def test_exact_lattice_codes(lattice, darts, order, precision):
    # FCC: rhombic dodecahedra, six vertices where four faces meet; simple
    # cubic: cubes, each corner the meeting point of the planes of seven
    # neighbours; BCC: truncated octahedra.  One code, full symmetry (48)
    s = getattr(W, lattice)(4, 1.0)
    got, ref = codes(s, (4, 4, 4), order, precision)
    coded = check(got, ref)
    assert coded.all()
    assert np.all(got["w_len"] == darts) and np.all(got["w_sym"] == 48)
    assert len(np.unique(got["w_hash"])) == 1


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


def test_codes_in_graph_replays():
    # the code kernel captured with the cells: every replay's codes equal the
    # eager call's and the oracle's, and follow new input at the same address
    import torch
    from paper_2209_11606_gb300 import vorogpu as V
    s = W.uniform(3000, 3, 3000 ** (1 / 3), True, seed=46)
    s2 = W.uniform(3000, 3, 3000 ** (1 / 3), True, seed=47)
    nb = (8, 8, 8)
    eager = {}
    for k, sk in ((1, s), (2, s2)):
        eager[k] = V.compute_host(sk.pos, sk.lo, sk.hi, sk.periodic, nblocks=nb, weinberg=1)
    pos = torch.from_numpy(np.ascontiguousarray(s.pos)).cuda()
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, nb)
    try:
        cfg = V.vg_config_default()
        cfg.weinberg = 1
        V.vg_graph_capture(ctx, [s.n], pos, None, cfg)
        for k, sk in ((1, s), (2, s2), (1, s)):
            pos.copy_(torch.from_numpy(np.ascontiguousarray(sk.pos)))
            for _ in range(2):
                V.vg_graph_launch(ctx)
            V.vg_graph_sync(ctx)
            wl, wh, ws = np.zeros(s.n, np.int32), np.zeros(s.n, np.uint64), np.zeros(s.n, np.int32)
            V.vg_get_weinberg(ctx, wl, wh, ws)
            np.testing.assert_array_equal(wl, eager[k]["w_len"])
            np.testing.assert_array_equal(wh, eager[k]["w_hash"])
            np.testing.assert_array_equal(ws, eager[k]["w_sym"])
    finally:
        V.vg_destroy(ctx)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, method="grid", nblocks=nb, weinberg=True)
    check(eager[1], ref)
