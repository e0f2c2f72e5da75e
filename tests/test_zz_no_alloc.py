"""The allocation-free counting sort, checked against the regular one.

vg_sort_blocks_noalloc() exists for callers that must not allocate device
memory when they call the library (a framework that owns all device memory,
a loop that cannot take cudaMalloc's implicit synchronisation, a process
near its memory limit).  Its scratch is a fixed array inside the library
shared by every call, so this test runs it twice in a row, with different
inputs, and compares each result with what vg_insert() + vg_get_sorted()
produce for the same points: both are integer permutations and must match
exactly.  The file sorts last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()
    return torch


def reference_sort(torch, s, nb):
    from paper_2209_11606_gb300 import vorogpu as V
    ctx = V.vg_create(s.dim, s.lo, s.hi, s.periodic, nb)
    try:
        V.vg_insert(ctx, s.pos)
        nblk = int(np.prod(nb))
        bs = np.zeros(nblk + 1, np.int32)
        order = np.zeros(s.n, np.int32)
        V.vg_get_sorted(ctx, bs, order)
        return bs, order
    finally:
        V.vg_destroy(ctx)


def test_noalloc_sort_matches_regular_sort_twice(torch_dev):
    torch = torch_dev
    from paper_2209_11606_gb300 import vorogpu as V
    from paper_2209_11606_gb300 import workloads as W
    cases = [(W.uniform(300_000, 3, 300_000 ** (1 / 3), True, seed=5), (39, 39, 39)),
             (W.uniform(50_000, 3, 1.0, False, seed=6), (20, 17, 23))]
    for s, nb in cases:
        want_bs, want_order = reference_sort(torch, s, nb)
        pos = torch.from_numpy(s.pos).cuda()
        bs = torch.zeros(int(np.prod(nb)) + 1, dtype=torch.int32, device="cuda")
        order = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        V.vg_sort_blocks_noalloc(s.dim, s.lo, s.hi, s.periodic, nb, pos, bs, order)
        torch.cuda.synchronize()
        assert np.array_equal(bs.cpu().numpy(), want_bs)
        assert np.array_equal(order.cpu().numpy(), want_order)


def test_noalloc_sort_rejects_sizes_beyond_its_limit(torch_dev):
    torch = torch_dev
    from paper_2209_11606_gb300 import vorogpu as V
    n = (1 << 20) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    bs = torch.zeros(9, dtype=torch.int32, device="cuda")
    order = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(V.VgError, match="no-alloc limit"):
        V.vg_sort_blocks_noalloc(3, [0, 0, 0], [1, 1, 1], (True,) * 3, (2, 2, 2), pos, bs, order)
