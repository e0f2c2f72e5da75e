"""One whole step (sort -> cells -> faces) captured as a CUDA graph and
replayed: replays must give exactly what the eager calls give on the same
input, follow new input written to the same device buffers, and report
input errors after the replay."""
import numpy as np
import pytest

import oracle
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare

pytestmark = pytest.mark.gpu

KEYS = ("vol", "area", "centroid", "nv", "ne", "nf", "status", "face_off", "nbr_id", "nbr_img",
        "face_order")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_11606_gb300 import build
    build.build()


def V():
    from paper_2209_11606_gb300 import vorogpu
    return vorogpu


def fetch(ctx, n, d):
    return V()._fetch(ctx, n, d, False)


def test_graph_replay_equals_eager_and_follows_new_input():
    import torch
    v = V()
    a = W.uniform(4000, 3, 4000 ** (1 / 3), True, seed=61)
    b = W.uniform(4000, 3, 4000 ** (1 / 3), True, seed=62)
    nb = (9, 9, 9)
    ctx = v.vg_create(3, a.lo, a.hi, a.periodic, nb)
    try:
        pos = torch.from_numpy(a.pos).cuda()
        cfg = v.vg_config_default()
        v.vg_graph_capture(ctx, [a.n], pos, None, cfg)
        eager_a = fetch(ctx, a.n, 3)
        l0 = v.vg_get_launches(ctx)
        v.vg_graph_launch(ctx)
        v.vg_graph_sync(ctx)
        per_replay = v.vg_get_launches(ctx) - l0
        assert per_replay >= 6  # sort kernels, three cell tiers, compaction
        got_a = fetch(ctx, a.n, 3)
        for k in KEYS:
            assert np.array_equal(got_a[k], eager_a[k]), k
        # new input in the same buffer, replayed without re-capture
        pos.copy_(torch.from_numpy(b.pos))
        v.vg_graph_launch(ctx)
        got_b = fetch(ctx, b.n, 3)
        ref = oracle.compute(b.pos, b.lo, b.hi, b.periodic, nblocks=nb)
        rep = compare(got_b, ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], rep
        # and the eager path on that input agrees bit for bit
        eager_b = v.compute_host(b.pos, b.lo, b.hi, b.periodic, nblocks=nb)
        for k in KEYS:
            assert np.array_equal(got_b[k], eager_b[k]), k
    finally:
        v.vg_destroy(ctx)


def test_graph_batched_radical_and_kernel_timing():
    import torch
    v = V()
    systems = [W.radical_uniform(1200, packing=0.4, sigma=0.3, seed=71),
               W.radical_uniform(900, packing=0.4, sigma=0.6, seed=72)]
    systems[1].periodic = (False, False, True)
    descs = [v.vg_system(s.lo, s.hi, s.periodic) for s in systems]
    ctx = v.vg_batch_create(3, descs)
    try:
        pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).cuda()
        rad = torch.from_numpy(np.concatenate([s.radii for s in systems])).cuda()
        cfg = v.vg_config_default()
        cfg.time_kernels = 1
        v.vg_graph_capture(ctx, [s.n for s in systems], pos, rad, cfg)
        v.vg_get_kernel_ms(ctx)
        for _ in range(3):
            v.vg_graph_launch(ctx)
        ms, cnt = v.vg_get_kernel_ms(ctx)
        assert cnt == 3 and ms > 0
        got = fetch(ctx, pos.shape[0], 3)
        from tests.test_gpu_batch import slice_system
        base = 0
        for k, s in enumerate(systems):
            ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, radii=s.radii,
                                 nblocks=v.vg_get_system_grid(ctx, k, 3))
            rep = compare(slice_system(got, base, s.n), ref, 1e-5)
            assert rep["topology_ok"] and rep["values_ok"], (k, rep)
            base += s.n
    finally:
        v.vg_destroy(ctx)


def test_graph_reports_input_errors_after_replay():
    import torch
    v = V()
    s = W.uniform(1500, 3, 2.0, False, seed=81)
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, (5, 5, 5))
    try:
        pos = torch.from_numpy(s.pos).cuda()
        v.vg_graph_capture(ctx, [s.n], pos)
        bad = s.pos.copy()
        bad[17, 1] = np.nan
        pos.copy_(torch.from_numpy(bad))
        v.vg_graph_launch(ctx)
        with pytest.raises(v.VgError) as e:
            v.vg_graph_sync(ctx)
        assert e.value.code == 4  # VG_ERR_NONFINITE
        bad = s.pos.copy()
        bad[3, 0] = 2.5  # outside the walled box
        pos.copy_(torch.from_numpy(bad))
        v.vg_graph_launch(ctx)
        with pytest.raises(v.VgError) as e:
            v.vg_get_counts(ctx)
        assert e.value.code == 3  # VG_ERR_OUT_OF_BOX
        # valid input again: the same graph recovers
        pos.copy_(torch.from_numpy(s.pos))
        v.vg_graph_launch(ctx)
        got = fetch(ctx, s.n, 3)
        ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(5, 5, 5))
        rep = compare(got, ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], rep
    finally:
        v.vg_destroy(ctx)


def test_graph_dropped_by_eager_calls():
    import torch
    v = V()
    s = W.uniform(800, 3, 1.0, True, seed=91)
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, (5, 5, 5))
    try:
        pos = torch.from_numpy(s.pos).cuda()
        v.vg_graph_capture(ctx, [s.n], pos)
        v.vg_insert(ctx, pos)
        with pytest.raises(v.VgError) as e:
            v.vg_graph_launch(ctx)
        assert e.value.code == 7  # VG_ERR_STATE: no graph held
        with pytest.raises(ValueError):
            v.vg_graph_capture(ctx, [s.n], s.pos)  # host input cannot be replayed
    finally:
        v.vg_destroy(ctx)
