"""Training driver of the learned candidate count (argument marshalling around
the vg_mlp_* entry points of include/vorogpu.h; every step runs in the
library's kernels).

A finished computation provides the labels: for each cell the number k* of
candidates within twice its final radius R (the radius bound of Sec. 2.1.3),
and per block the largest k* of its cells.  The network reads the 27 block
counts around a block and is trained with Adam on log k*, with
under-predictions weighted by `u` since they cost a fallback to the walk.
"""
from __future__ import annotations

import numpy as np

from . import vorogpu as V

NIN, H1, H2 = 27, 32, 32


def init_params(seed: int = 0) -> np.ndarray:
    """Initial parameters: weights normal with std sqrt(2 / fan_in) (sqrt(1 /
    fan_in) for the output row), biases 0, output bias log(40)."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, np.sqrt(2.0 / NIN), H1 * NIN)
    w2 = rng.normal(0.0, np.sqrt(2.0 / H1), H2 * H1)
    w3 = rng.normal(0.0, np.sqrt(1.0 / H2), H2)
    p = np.concatenate([w1, np.zeros(H1), w2, np.zeros(H2), w3, [np.log(40.0)]])
    assert p.size == V.MLP_NPARAM
    return p.astype(np.float32)


def rows_from(ctx, torch):
    """Training rows (features, targets) of a computed container, on the device."""
    nb = V.vg_get_sorted(ctx)
    X = torch.empty((nb, NIN), dtype=torch.float32, device="cuda")
    t = torch.empty(nb, dtype=torch.float32, device="cuda")
    m = V.vg_mlp_dataset(ctx, X, t)
    return X[:m], t[:m]


def rows_for_system(s, torch, nblocks=None):
    """Computes the cells of one system (FP32 form, default preload) and
    returns its training rows."""
    ctx = V.vg_create(s.dim, s.lo, s.hi, s.periodic, nblocks)
    try:
        V.vg_insert(ctx, torch.from_numpy(np.ascontiguousarray(s.pos)).cuda())
        V.vg_compute(ctx, V.vg_config_default())
        return rows_from(ctx, torch)
    finally:
        V.vg_destroy(ctx)


def train(X, t, torch, seed: int = 0, steps: int = 600, lr: float = 3e-3, u: float = 4.0):
    """Full-batch Adam from init_params(seed); returns (params, losses)."""
    m = V.vg_mlp_create()
    try:
        V.vg_mlp_set_params(m, init_params(seed))
        losses = V.vg_mlp_train(m, X.contiguous(), t.contiguous(), X.shape[0], u, lr, steps)
        return V.vg_mlp_get_params(m), losses
    finally:
        V.vg_mlp_destroy(m)


def predictor(params):
    """A vg_mlp handle holding `params` (destroy with vorogpu.vg_mlp_destroy)."""
    m = V.vg_mlp_create()
    V.vg_mlp_set_params(m, params)
    return m
