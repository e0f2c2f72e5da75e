"""The library's block grid and counting sort against the oracle's.

Two steps of the hot path have plain definitions that the oracle writes
out (Sec. 2.1.1 and Sec. 2.1.4):

* the grid rule: lambda = (N / (n_opt V))^(1/d), n_a = max(1, floor(lambda
  L_a)) -- the floor is the reading that reproduces Table 3;
* the counting sort: block k = i + n_x (j + n_y l) with i = floor((x -
  a_x) / h_x) clamped to the grid, particles listed block by block, and by
  input index inside a block (a stable sort by block index).

Both are integer results and must match exactly: the library's grid (read
with vg_get_grid after an insert under the n_opt rule) against
oracle.grid_size, and the library's permutation (vg_get_sorted, and the
allocation-free vg_sort_blocks_noalloc) against oracle.block_sort, element
by element."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()
    return torch


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def library_grid(torch, n, lo, hi, periodic, n_opt):
    """Block counts the library picks for n particles under the n_opt rule
    (positions drawn on the device, uniform in the box)."""
    from paper_2209_11606_gb300 import vorogpu as V
    d = len(lo)
    g = torch.Generator(device="cuda")
    g.manual_seed(n % 1000003)
    lo_t = torch.tensor(lo, dtype=torch.float64, device="cuda")
    span = torch.tensor(np.asarray(hi) - np.asarray(lo), dtype=torch.float64, device="cuda")
    pos = (torch.rand((n, d), dtype=torch.float64, device="cuda", generator=g) * span + lo_t).contiguous()
    ctx = V.vg_create(d, lo, hi, periodic, None, n_opt)
    try:
        V.vg_insert(ctx, pos)
        return V.vg_get_grid(ctx, d)
    finally:
        V.vg_destroy(ctx)
        del pos
        torch.cuda.empty_cache()


def test_grid_rule_matches_table3(torch_dev):
    """Every row of Table 3 (N = 10^8 in the unit square / cube): the
    library's grid equals the oracle's and the printed value."""
    for dim, n, nopt, want in _golden("table3_grid_sizes.txt"):
        dim, n = int(dim), int(n)
        ref = oracle.grid_size(n, np.zeros(dim), np.ones(dim), nopt, "floor")
        assert ref == (int(want),) * dim
        got = library_grid(torch_dev, n, [0.0] * dim, [1.0] * dim, (False,) * dim, nopt)
        assert got == ref, (dim, n, nopt, got, ref)


@pytest.mark.parametrize("dim,n,lo,hi,nopt", [
    (3, 12_345, (0.0, 0.0, 0.0), (3.0, 1.7, 0.9), 4.6),
    (3, 1_000, (-2.0, 1.0, 0.5), (5.0, 1.3, 9.0), 1.0),
    (3, 77_777, (0.0, 0.0, 0.0), (1.0, 1.0, 50.0), 0.0),   # 0: the 3D default 4.6
    (2, 54_321, (0.0, -1.0), (10.0, 0.25), 3.4),
    (2, 999, (0.0, 0.0), (1.0, 1.0), 0.0),                 # 0: the 2D default 3.4
    (3, 5, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 4.6),         # lambda L < 1: one block per axis
])
def test_grid_rule_ragged_boxes(torch_dev, dim, n, lo, hi, nopt):
    want_nopt = nopt if nopt > 0 else (4.6 if dim == 3 else 3.4)
    ref = oracle.grid_size(n, np.asarray(lo), np.asarray(hi), want_nopt, "floor")
    got = library_grid(torch_dev, n, list(lo), list(hi), (False,) * dim, nopt)
    assert got == ref, (got, ref)


def library_sort(s, nb):
    from paper_2209_11606_gb300 import vorogpu as V
    ctx = V.vg_create(s.dim, s.lo, s.hi, s.periodic, nb)
    try:
        V.vg_insert(ctx, s.pos)
        nblk = int(np.prod(nb))
        bs = np.zeros(nblk + 1, np.int32)
        order = np.zeros(s.n, np.int32)
        assert V.vg_get_sorted(ctx, bs, order) == nblk
        return bs, order
    finally:
        V.vg_destroy(ctx)


def noalloc_sort(torch, s, nb):
    from paper_2209_11606_gb300 import vorogpu as V
    pos = torch.from_numpy(np.ascontiguousarray(s.pos)).cuda()
    bs = torch.full((int(np.prod(nb)) + 1,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((s.n,), -7, dtype=torch.int32, device="cuda")
    V.vg_sort_blocks_noalloc(s.dim, s.lo, s.hi, s.periodic, nb, pos, bs, order)
    torch.cuda.synchronize()
    return bs.cpu().numpy(), order.cpu().numpy()


def oracle_sort(s, nb):
    order, start = oracle.block_sort(s.pos, s.lo, s.hi, nb)
    return start.astype(np.int64), order.astype(np.int64)


def _cluster_big_block():
    """10^4 points in one block of a 10^3 grid, plus a uniform background:
    the in-block order of a heavily loaded block."""
    rng = np.random.default_rng(31)
    bg = rng.random((20_000, 3))
    cl = 0.5 + 0.05 * rng.random((12_000, 3)) + 1e-3   # inside block (5, 5, 5) of 10^3
    pos = np.concatenate([bg[:9000], cl, bg[9000:]])
    return W.System(pos=pos, lo=np.zeros(3), hi=np.ones(3), periodic=(False, False, False))


SORT_CASES = {
    "walled": (lambda: W.uniform(40_000, 3, 1.0, False, seed=21), (17, 23, 19)),
    "periodic": (lambda: W.uniform(60_000, 3, 60_000 ** (1 / 3), True, seed=22), (24, 24, 24)),
    "mixed": (lambda: _with_periodic(W.uniform(30_000, 3, 2.0, False, seed=23), (True, False, True)),
              (11, 13, 7)),
    "clustered": (lambda: W.extreme_clustering(50_000, 3, seed=24), (37, 37, 37)),
    "blobs": (lambda: W.blobs(40_000, 10.0, seed=25), (20, 20, 20)),
    "big_block": (_cluster_big_block, (10, 10, 10)),
    # blocks of every size class: a scan below 65 particles, a shared-memory
    # sort up to 4096, a radix sort beyond (5000 in the central blocks)
    "extreme_1m": (lambda: W.extreme_clustering(1_000_000, 3, seed=28), (50, 50, 50)),
    "2d_walled": (lambda: W.uniform(50_000, 2, 1.0, False, seed=26), (121, 97)),
    "2d_periodic": (lambda: W.uniform(50_000, 2, 3.0, True, seed=27), (130, 130)),
}


def _with_periodic(s, per):
    s.periodic = per
    return s


@pytest.mark.parametrize("name", sorted(SORT_CASES))
def test_sort_permutation_matches_oracle(torch_dev, name):
    make, nb = SORT_CASES[name]
    s = make()
    want_bs, want_order = oracle_sort(s, nb)
    if name == "big_block":
        assert np.diff(want_bs).max() >= 10_000
    bs, order = library_sort(s, nb)
    assert np.array_equal(bs.astype(np.int64), want_bs)
    assert np.array_equal(order.astype(np.int64), want_order)
    bs2, order2 = noalloc_sort(torch_dev, s, nb)
    assert np.array_equal(bs2.astype(np.int64), want_bs)
    assert np.array_equal(order2.astype(np.int64), want_order)


def test_periodic_wrap_matches_oracle(torch_dev):
    """Points outside a periodic box are wrapped into [lo, hi) before they
    are binned.  Coordinates on a dyadic grid with a dyadic period wrap
    exactly, so the oracle sorts the wrapped copy (np.mod) of the same
    points and the permutations must agree."""
    rng = np.random.default_rng(41)
    L = 4.0
    n = 20_000
    inside = rng.integers(0, 4096, size=(n, 3)) / 1024.0          # [0, 4) on a 2^-10 grid
    shift = rng.integers(-3, 4, size=(n, 3)).astype(np.float64) * L
    s = W.System(pos=inside + shift, lo=np.zeros(3), hi=np.full(3, L), periodic=(True, True, True))
    nb = (13, 16, 9)
    wrapped = W.System(pos=np.mod(s.pos, L), lo=s.lo, hi=s.hi, periodic=s.periodic)
    assert np.array_equal(wrapped.pos, inside)
    want_bs, want_order = oracle_sort(wrapped, nb)
    bs, order = library_sort(s, nb)
    assert np.array_equal(bs.astype(np.int64), want_bs)
    assert np.array_equal(order.astype(np.int64), want_order)
    bs2, order2 = noalloc_sort(torch_dev, s, nb)
    assert np.array_equal(bs2.astype(np.int64), want_bs)
    assert np.array_equal(order2.astype(np.int64), want_order)


def test_points_on_the_upper_face_go_to_the_last_block(torch_dev):
    """A walled coordinate equal to hi lies in the box; its block index is
    clamped to n - 1 (the reading of Sec. 2.1.1 for the closed box)."""
    pos = np.array([[1.0, 0.5, 0.0], [0.0, 1.0, 1.0], [1.0, 1.0, 1.0], [0.25, 0.25, 0.25]])
    s = W.System(pos=pos, lo=np.zeros(3), hi=np.ones(3), periodic=(False, False, False))
    nb = (4, 4, 4)
    want_bs, want_order = oracle_sort(s, nb)
    bs, order = library_sort(s, nb)
    assert np.array_equal(bs.astype(np.int64), want_bs)
    assert np.array_equal(order.astype(np.int64), want_order)
    bs2, order2 = noalloc_sort(torch_dev, s, nb)
    assert np.array_equal(bs2.astype(np.int64), want_bs)
    assert np.array_equal(order2.astype(np.int64), want_order)


@pytest.mark.parametrize("bad", ["nan", "inf", "outside"])
def test_invalid_points_are_reported(torch_dev, bad):
    """A non-finite coordinate gives VG_ERR_NONFINITE and a walled
    coordinate outside [lo, hi] VG_ERR_OUT_OF_BOX, from both sorts."""
    from paper_2209_11606_gb300 import vorogpu as V
    s = W.uniform(1000, 3, 1.0, False, seed=51)
    pos = s.pos.copy()
    if bad == "nan":
        pos[517, 1] = np.nan
    elif bad == "inf":
        pos[3, 2] = -np.inf
    else:
        pos[999, 0] = 1.0 + 1e-9
    want = V.STATUS_CODES["VG_ERR_OUT_OF_BOX" if bad == "outside" else "VG_ERR_NONFINITE"]
    ctx = V.vg_create(3, s.lo, s.hi, s.periodic, (4, 4, 4))
    try:
        with pytest.raises(V.VgError) as e:
            V.vg_insert(ctx, pos)
        assert e.value.code == want
    finally:
        V.vg_destroy(ctx)
    torch = torch_dev
    pos_d = torch.from_numpy(pos).cuda()
    bs = torch.zeros(65, dtype=torch.int32, device="cuda")
    order = torch.zeros(s.n, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VgError) as e:
        V.vg_sort_blocks_noalloc(3, s.lo, s.hi, s.periodic, (4, 4, 4), pos_d, bs, order)
    assert e.value.code == want
