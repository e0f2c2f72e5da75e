"""The learned candidate count on the GPU against the FP64 oracle
(oracle/mlp.py): features, k* labels, training rows, forward pass, loss and
gradient, the Adam step, and the cells computed with predicted preloads."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as OM
from paper_2209_11606_gb300 import workloads as W
from tests.compare import compare

pytestmark = pytest.mark.gpu


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


def computed(s, nb, precision="fp64", order="walk"):
    v = V()
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, nb)
    v.vg_insert(ctx, s.pos)
    cfg = v.vg_config_default()
    cfg.precision = v.VG_FP64 if precision == "fp64" else v.VG_FP32_RETEST
    cfg.order = v.VG_WALK if order == "walk" else v.VG_PREFETCH
    v.vg_compute(ctx, cfg)
    return ctx


@pytest.mark.parametrize("periodic", [True, False])
def test_features_match_oracle(periodic):
    v = V()
    s = W.uniform(4000, 3, 1.0, periodic, seed=101)
    nb = (9, 7, 8)
    ctx = computed(s, nb)
    try:
        X = np.zeros((9 * 7 * 8, 27), np.float32)
        v.vg_mlp_features(ctx, X)
        ref = OM.block_features(s.pos, s.lo, s.hi, s.periodic, nb)
        # FP32 features c_j * (inside / sum) - 1: two roundings of values
        # below about 6, so within 1e-6 absolute of the FP64 ones
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-6)
    finally:
        v.vg_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_labels_match_oracle(precision):
    v = V()
    s = W.uniform(3000, 3, 3000 ** (1 / 3), True, seed=102)
    nb = (8, 8, 8)
    ctx = computed(s, nb, precision, "walk" if precision == "fp64" else "prefetch")
    try:
        R = np.zeros(s.n, np.float32)
        v.vg_get_radius(ctx, R)
        ks = np.zeros(s.n, np.int32)
        v.vg_mlp_labels(ctx, ks)
    finally:
        v.vg_destroy(ctx)
    ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=nb)
    # R: the largest vertex distance, to FP32 (plus the FP32 form's allowance)
    np.testing.assert_allclose(R, ref["rmax"], rtol=2e-5 if precision == "fp32" else 1e-6)
    # k* given the same R: the count itself is exact
    ks_same_r = OM.kstar(s.pos, s.lo, s.hi, s.periodic, R.astype(np.float64))
    assert np.array_equal(ks, ks_same_r)
    # k* from the oracle's own R: equal except where a candidate lies within
    # the R tolerance of the 2R sphere
    ks_o = OM.kstar(s.pos, s.lo, s.hi, s.periodic, ref["rmax"])
    diff = np.nonzero(ks != ks_o)[0]
    assert len(diff) <= 3
    for i in diff:
        lo_ = OM.kstar(s.pos, s.lo, s.hi, s.periodic, [ref["rmax"][i] * (1 - 3e-5)], cells=[i])[0]
        hi_ = OM.kstar(s.pos, s.lo, s.hi, s.periodic, [ref["rmax"][i] * (1 + 3e-5)], cells=[i])[0]
        assert lo_ <= ks[i] <= hi_


def test_dataset_matches_oracle():
    import torch
    v = V()
    s = W.uniform(1500, 3, 1.0, False, seed=103)
    nb = (9, 9, 9)  # some blocks are empty
    ctx = computed(s, nb)
    try:
        B = 9 * 9 * 9
        X = torch.zeros((B, 27), dtype=torch.float32, device="cuda")
        t = torch.zeros(B, dtype=torch.float32, device="cuda")
        m = v.vg_mlp_dataset(ctx, X, t)
        R = np.zeros(s.n, np.float32)
        v.vg_get_radius(ctx, R)
    finally:
        v.vg_destroy(ctx)
    ks = OM.kstar(s.pos, s.lo, s.hi, s.periodic, R.astype(np.float64))
    tt, has = OM.block_targets(s.pos, s.lo, s.hi, s.periodic, nb, ks)
    F = OM.block_features(s.pos, s.lo, s.hi, s.periodic, nb)
    assert m == int(has.sum()) and m < B
    np.testing.assert_allclose(X[:m].cpu().numpy(), F[has], rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(t[:m].cpu().numpy(), tt[has], rtol=1e-6, atol=1e-7)


def _rows(seed, M=3000):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.random((M, 27)).astype(np.float32)
    t = rng.normal(3.5, 0.6, M).astype(np.float32)
    return X, t, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()


def test_forward_matches_oracle():
    import torch
    v = V()
    p = (OM.init_params(5) + np.random.default_rng(6).normal(0, 0.1, OM.NPARAM)).astype(np.float32)
    X, _, Xd, _ = _rows(7)
    m = v.vg_mlp_create()
    try:
        v.vg_mlp_set_params(m, p)
        y = torch.zeros(len(X), dtype=torch.float32, device="cuda")
        v.vg_mlp_infer(m, Xd, len(X), y)
        torch.cuda.synchronize()
    finally:
        v.vg_mlp_destroy(m)
    ref, _ = OM.forward(OM.fp16_weights(p.astype(np.float64)), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("u", [1.0, 4.0])
def test_loss_and_gradient_match_oracle(u):
    v = V()
    p = (OM.init_params(8) + np.random.default_rng(9).normal(0, 0.05, OM.NPARAM)).astype(np.float32)
    X, t, Xd, td = _rows(10)
    m = v.vg_mlp_create()
    try:
        v.vg_mlp_set_params(m, p)
        L, g = v.vg_mlp_loss_grad(m, Xd, td, len(X), u)
    finally:
        v.vg_mlp_destroy(m)
    Lr, gr = OM.loss_grad(OM.fp16_weights(p.astype(np.float64)), X.astype(np.float64),
                          t.astype(np.float64), u)
    assert math.isclose(L, Lr, rel_tol=1e-5)
    # FP32 accumulation against FP64: relative to the gradient's size
    scale = np.max(np.abs(gr))
    assert np.max(np.abs(g - gr)) <= 1e-4 * scale
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr) * math.sqrt(OM.NPARAM)


def test_adam_step_matches_oracle():
    v = V()
    p = (OM.init_params(11)).astype(np.float32)
    X, t, Xd, td = _rows(12, 1000)
    m = v.vg_mlp_create()
    try:
        v.vg_mlp_set_params(m, p)
        _, g = v.vg_mlp_loss_grad(m, Xd, td, len(X), 4.0)
        v.vg_mlp_train(m, Xd, td, len(X), 4.0, 1e-3, 1)
        p1 = v.vg_mlp_get_params(m)
    finally:
        v.vg_mlp_destroy(m)
    ref, _, _ = OM.adam(p.astype(np.float64), np.zeros(OM.NPARAM), np.zeros(OM.NPARAM),
                        g.astype(np.float64), 1, lr=1e-3)
    np.testing.assert_allclose(p1, ref, rtol=0, atol=2e-6)


def test_training_lowers_the_loss():
    import torch
    v = V()
    s = W.uniform(20000, 3, 20000 ** (1 / 3), True, seed=104)
    ctx = computed(s, (15, 15, 15), "fp32", "prefetch")
    m = v.vg_mlp_create()
    try:
        B = 15 ** 3
        X = torch.zeros((B, 27), dtype=torch.float32, device="cuda")
        t = torch.zeros(B, dtype=torch.float32, device="cuda")
        M = v.vg_mlp_dataset(ctx, X, t)
        v.vg_mlp_set_params(m, OM.init_params(13).astype(np.float32))
        losses = v.vg_mlp_train(m, X, t, M, 4.0, 3e-3, 300)
        assert losses[-1] < 0.6 * losses[0]
        # better than the best constant prediction under the same loss: the
        # 27 block counts carry information about the cell sizes
        tt = t[:M].cpu().numpy().astype(np.float64)
        cs = np.linspace(tt.min(), tt.max(), 2001)
        e = cs[:, None] - tt[None, :]
        const_loss = np.min(np.mean(np.where(e < 0, 4.0, 1.0) * e * e, axis=1))
        y = torch.zeros(M, dtype=torch.float32, device="cuda")
        v.vg_mlp_infer(m, X, M, y)
        torch.cuda.synchronize()
        ey = y.cpu().numpy().astype(np.float64) - tt
        net_loss = np.mean(np.where(ey < 0, 4.0, 1.0) * ey * ey)
        assert net_loss < const_loss
    finally:
        v.vg_mlp_destroy(m)
        v.vg_destroy(ctx)


def test_predicted_preload_keeps_the_cells():
    """Cells computed with the learned per-block preload equal the oracle's,
    whatever the network predicts: the radius bound decides and shortfalls
    fall back to the walk."""
    v = V()
    s = W.bcc(14, 1.25, 0.02, seed=105)
    nb = (12, 12, 12)
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, nb)
    m = v.vg_mlp_create()
    try:
        v.vg_insert(ctx, s.pos)
        ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=nb)
        for params, alpha in ((OM.init_params(14), 1.0), (np.zeros(OM.NPARAM), 0.2)):
            v.vg_mlp_set_params(m, params.astype(np.float32))
            v.vg_mlp_predict(ctx, m, alpha, 8.0, 512.0)
            cfg = v.vg_config_default()
            cfg.use_mlp = 1
            cfg.collect_stats = 1
            v.vg_compute(ctx, cfg)
            got = v._fetch(ctx, s.n, 3, True)
            rep = compare(got, ref, 1e-5)
            assert rep["topology_ok"] and rep["values_ok"], rep
    finally:
        v.vg_mlp_destroy(m)
        v.vg_destroy(ctx)


def test_use_mlp_needs_a_prediction_after_insert():
    v = V()
    s = W.uniform(500, 3, 1.0, True, seed=106)
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, (4, 4, 4))
    m = v.vg_mlp_create()
    try:
        v.vg_insert(ctx, s.pos)
        cfg = v.vg_config_default()
        cfg.use_mlp = 1
        with pytest.raises(v.VgError) as e:
            v.vg_compute(ctx, cfg)
        assert e.value.code == 7
        v.vg_mlp_predict(ctx, m, 1.0, 8.0, 512.0)
        v.vg_compute(ctx, cfg)
        v.vg_insert(ctx, s.pos)  # a new insert invalidates the prediction
        with pytest.raises(v.VgError):
            v.vg_compute(ctx, cfg)
    finally:
        v.vg_mlp_destroy(m)
        v.vg_destroy(ctx)


def test_attached_predictor_runs_inside_the_graph():
    import torch
    v = V()
    s = W.uniform(20000, 3, 20000 ** (1 / 3), True, seed=107)
    nb = (15, 15, 15)
    ctx = v.vg_create(3, s.lo, s.hi, s.periodic, nb)
    m = v.vg_mlp_create()
    try:
        v.vg_mlp_set_params(m, OM.init_params(15).astype(np.float32))
        pos = torch.from_numpy(s.pos).cuda()
        # eager: explicit prediction after the insert
        v.vg_insert(ctx, pos)
        v.vg_mlp_predict(ctx, m, 1.3, 8.0, 512.0)
        cfg = v.vg_config_default()
        cfg.use_mlp = 1
        cfg.collect_stats = 1
        v.vg_compute(ctx, cfg)
        eager = v._fetch(ctx, s.n, 3, True)
        # attached: the graph runs sort -> predict -> cells -> faces
        v.vg_set_predictor(ctx, m, 1.3, 8.0, 512.0)
        v.vg_graph_capture(ctx, [s.n], pos, None, cfg)
        v.vg_graph_launch(ctx)
        got = v._fetch(ctx, s.n, 3, True)
        assert np.array_equal(got["work"]["n_prefetch"], eager["work"]["n_prefetch"])
        for k in ("vol", "area", "nf", "nbr_id", "face_off"):
            assert np.array_equal(got[k], eager[k]), k
        ref = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=nb)
        rep = compare(got, ref, 1e-5)
        assert rep["topology_ok"] and rep["values_ok"], rep
    finally:
        v.vg_destroy(ctx)
        v.vg_mlp_destroy(m)
