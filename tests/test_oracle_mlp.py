"""Pins for the FP64 oracle of the candidate-count predictor (oracle/mlp.py):
finite differences, closed forms and invariants, none computed by the
functions under test."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as M
from paper_2209_11606_gb300 import workloads as W


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.4, M.NPARAM)


def test_parameter_count():
    assert M.NPARAM == 32 * 27 + 32 + 32 * 32 + 32 + 32 + 1 == 1985


@pytest.mark.parametrize("u", [1.0, 4.0])
def test_gradient_matches_central_differences(u):
    rng = np.random.default_rng(1)
    p = _rand_params(2)
    X = rng.random((40, 27))
    t = rng.normal(3.0, 0.5, 40)
    L, g = M.loss_grad(p, X, t, u)
    assert math.isclose(L, M.loss(p, X, t, u), rel_tol=1e-14)
    h = 1e-6
    idx = rng.choice(M.NPARAM, 120, replace=False)
    # every block of the packed vector is probed: W1, b1, W2, b2, W3, b3
    idx = np.unique(np.concatenate([idx, [0, 864, 900, 1888, 1920, 1984]]))
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss(pp, X, t, u) - M.loss(pm, X, t, u)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_constant_network_loss_and_bias_gradient():
    # all weights zero: y = b3 everywhere, so L = mean(w (b3 - t)^2) and
    # dL/db3 = mean(2 w (b3 - t)), every other gradient zero (ReLUs at 0)
    p = np.zeros(M.NPARAM)
    p[-1] = 2.0
    t = np.array([1.0, 3.0, 2.5, 1.5])
    X = np.ones((4, 27))
    L, g = M.loss_grad(p, X, t, 4.0)
    w = np.array([1.0, 4.0, 4.0, 1.0])
    e = 2.0 - t
    assert math.isclose(L, np.mean(w * e * e), rel_tol=1e-15)
    assert math.isclose(g[-1], np.mean(2 * w * e), rel_tol=1e-15)
    assert np.all(g[:-1] == 0.0)


def test_first_adam_step_is_signed_learning_rate():
    # step 1: m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps)
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = M.adam(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-2)
    np.testing.assert_allclose(p - p1, 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-13)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-13)


def test_adam_minimises_a_quadratic():
    p = np.array([3.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for k in range(1, 3001):
        p, m, v = M.adam(p, m, v, 2 * p, k, lr=1e-2)
    assert np.all(np.abs(p) < 1e-3)


def test_fp16_rounding_touches_only_weights():
    p = _rand_params(4)
    q = M.fp16_weights(p)
    W1, b1, W2, b2, W3, b3 = M.unpack(q)
    P1, c1, P2, c2, P3, c3 = M.unpack(p)
    for a, b in ((W1, P1), (W2, P2), (W3, P3)):
        assert np.all(a == b.astype(np.float16).astype(np.float64))
        assert np.max(np.abs(a - b)) <= 2 ** -11 * np.max(np.abs(b))
    for a, b in ((b1, c1), (b2, c2), (b3, c3)):
        assert np.array_equal(a, b)


def test_features_count_invariants():
    s = W.uniform(3000, 3, 1.0, True, seed=5)
    nb = (7, 6, 5)
    c, v = M.block_counts27(s.pos, s.lo, s.hi, s.periodic, nb)
    assert np.all(v == 27)
    # the centre column is the block's own count; on a torus every particle
    # is seen by exactly 27 neighbourhoods
    assert c[:, 13].sum() == 3000
    assert c.sum() == 27 * 3000
    # the counts match a direct count of the shifted block
    k = oracle.block_index(s.pos, s.lo, s.hi, nb)
    own = np.bincount(k, minlength=7 * 6 * 5)
    assert np.array_equal(c[:, 13], own)
    b = 7 * (2 + 6 * 3) + 4        # block (4, 2, 3)
    nbk = (4 + 1) % 7 + 7 * (2 + 6 * ((3 - 1) % 5))  # (dx, dy, dz) = (+1, 0, -1)
    assert c[b, 2 + 3 * 1 + 9 * 0] == own[nbk]


def test_features_are_counts_over_their_mean():
    s = W.uniform(3000, 3, 1.0, False, seed=5)
    nb = (7, 6, 5)
    X = M.block_features(s.pos, s.lo, s.hi, s.periodic, nb)
    c, v = M.block_counts27(s.pos, s.lo, s.hi, s.periodic, nb)
    # inside the box the features average to 0 over a block's neighbourhood
    # (they are the counts over their mean, minus 1); past a wall they are -1
    ins = np.zeros_like(c, dtype=bool)
    for b in range(c.shape[0]):
        i, j, l = b % 7, (b // 7) % 6, b // 42
        for q in range(27):
            t = (i + q % 3 - 1, j + (q // 3) % 3 - 1, l + q // 9 - 1)
            ins[b, q] = 0 <= t[0] < 7 and 0 <= t[1] < 6 and 0 <= t[2] < 5
    assert np.array_equal(ins.sum(axis=1), v)
    np.testing.assert_allclose(np.where(ins, X, 0.0).sum(axis=1), 0.0, atol=1e-12)
    assert np.all(X[~ins] == -1.0)
    # x_j + 1 is proportional to c_j: ratios of counts are kept
    ok = (c[:, 13] > 0) & (c[:, 4] > 0)
    np.testing.assert_allclose((X[ok, 13] + 1.0) / (X[ok, 4] + 1.0), c[ok, 13] / c[ok, 4], rtol=1e-12)


def test_features_do_not_depend_on_density():
    # every particle doubled (a copy moved by a tenth of the spacing inside
    # its block): every count doubles and the features stay the same; the
    # same points in a box scaled by 3 (same block grid) give the same
    # features too
    s = W.uniform(2000, 3, 1.0, True, seed=8)
    nb = (6, 6, 6)
    X = M.block_features(s.pos, s.lo, s.hi, s.periodic, nb)
    h = 1.0 / 6
    cell = np.floor(s.pos / h)
    moved = np.clip(s.pos + 0.1 * h * 0.05, cell * h, (cell + 1) * h - 1e-12)
    X2 = M.block_features(np.concatenate([s.pos, moved]), s.lo, s.hi, s.periodic, nb)
    np.testing.assert_allclose(X2, X, atol=1e-12)
    X3 = M.block_features(3.0 * s.pos, 3.0 * s.lo, 3.0 * s.hi, s.periodic, nb)
    np.testing.assert_allclose(X3, X, atol=1e-12)


def test_features_walls_give_minus_one_outside():
    s = W.uniform(500, 3, 1.0, False, seed=6)
    X = M.block_features(s.pos, s.lo, s.hi, s.periodic, (1, 1, 1))
    # one block: it is its own neighbourhood's mean, every other block is
    # past a wall
    assert X[0, 13] == 0.0 and np.all(np.delete(X[0], 13) == -1.0)


def test_kstar_bcc_is_fourteen():
    # BCC: R = sqrt(5)/4 a, 2R = 1.118 a; 8 neighbours at 0.866 a and 6 at a
    # lie inside, the next 12 at 1.414 a outside
    s = W.bcc(3, 1.25)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(3, 3, 3))
    np.testing.assert_allclose(r["rmax"], math.sqrt(5) / 4 * 1.25, rtol=1e-12)
    ks = M.kstar(s.pos, s.lo, s.hi, s.periodic, r["rmax"])
    assert np.all(ks == 14)


def test_kstar_matches_kdtree_count():
    spatial = pytest.importorskip("scipy.spatial")
    s = W.uniform(800, 3, 800 ** (1 / 3), True, seed=7)
    r = oracle.compute(s.pos, s.lo, s.hi, s.periodic, nblocks=(5, 5, 5))
    ks = M.kstar(s.pos, s.lo, s.hi, s.periodic, r["rmax"])
    L = s.hi[0]
    tree = spatial.cKDTree(np.mod(s.pos, L), boxsize=L)
    for i in range(0, 800, 37):
        # strictly inside 2R: count within a radius just below it (no point
        # of this draw lies within 1e-9 of the sphere)
        n = len(tree.query_ball_point(np.mod(s.pos[i], L), 2 * r["rmax"][i] * (1 - 1e-12))) - 1
        assert ks[i] == n


def test_block_targets_take_the_block_maximum():
    s = W.uniform(400, 3, 1.0, True, seed=8)
    ks = np.arange(400)
    t, has = M.block_targets(s.pos, s.lo, s.hi, s.periodic, (3, 3, 3), ks)
    k = oracle.block_index(s.pos, s.lo, s.hi, (3, 3, 3))
    for b in range(27):
        sel = ks[k == b]
        assert has[b] == (len(sel) > 0)
        if len(sel):
            assert t[b] == math.log(max(1, sel.max()))
