"""FP64 CPU oracle of the learned candidate-count predictor.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may use it; the
library never does.  Plain numpy in float64, written from the definitions
below; it shares nothing with the CUDA kernels.

The paper itself has no learned part: a cell's candidates come from the block
walk with the radius bound of Sec. 2.1.3 (stop once no remaining block can
hold a particle within 2R of the particle, R the cell's largest vertex
distance).  The predictor estimates, per block, how many nearest candidates
a cell of that block needs so that a single distance-sorted preload already
contains every candidate within 2R.  Definitions:

* Features of block b: the particle counts c_j of the 27 blocks b + (dx, dy,
  dz), dx, dy, dz in {-1, 0, 1}, j = (dx+1) + 3 (dy+1) + 9 (dz+1), wrapped on
  periodic axes and 0 outside a walled box, relative to their mean:
  x_j = c_j / m - 1 with m = (sum_j c_j) / v, v the number of those blocks
  inside the box (x = 0 where m = 0).  The features do not change with the
  density or the block size, only with how the particles are spread over
  the 27 blocks; the cell kernel turns a count into a radius with the same
  local density m / h^d.
* Label of cell i: k*_i = the number of candidates (particle j and periodic
  image m, excluding i itself with m = 0) at distance < 2 R_i.  Cutting those
  in distance order leaves the final cell, and the radius bound then stops.
* Target of block b: t_b = log(max(1, max over the block's cells of k*_i)),
  defined for blocks that hold at least one particle.
* Network: y = W3 . relu(W2 relu(W1 x + b1) + b2) + b3 with hidden widths 32
  and 32; parameters are packed as W1 (32 x 27, row = hidden unit), b1 (32),
  W2 (32 x 32), b2 (32), W3 (32), b3 (1) -- 1985 numbers.  The predicted
  count is exp(y).
* Loss over M blocks: L = (1/M) sum_b w_b (y_b - t_b)^2 with w_b = u when
  y_b < t_b (an under-prediction, which costs a fallback to the walk) and 1
  otherwise.
* Update: Adam (Kingma and Ba, 2015) with bias correction.

Every function is pinned by tests/test_oracle_mlp.py: central finite
differences of the loss, the closed-form first Adam step, the BCC neighbour
count 14, count invariants and density invariance of the features, and a
k-d tree count.
"""
from __future__ import annotations

import numpy as np

from . import block_index

H1 = 32
H2 = 32
NIN = 27
NPARAM = H1 * NIN + H1 + H2 * H1 + H2 + H2 + 1  # 1985


def unpack(p):
    """Views of the packed parameter vector: W1, b1, W2, b2, W3, b3."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H1 * NIN].reshape(H1, NIN); o += H1 * NIN
    b1 = p[o:o + H1]; o += H1
    W2 = p[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = p[o:o + H2]; o += H2
    W3 = p[o:o + H2]; o += H2
    b3 = p[o:o + 1]; o += 1
    assert o == NPARAM
    return W1, b1, W2, b2, W3, b3


def fp16_weights(p):
    """The parameters as inference sees them: W1, W2, W3 rounded to FP16
    (round to nearest even), biases kept."""
    q = np.array(p, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(q)
    for w in (W1, W2, W3):
        w[...] = w.astype(np.float16).astype(np.float64)
    return q


def block_counts(pos, lo, hi, periodic, nblocks):
    """Particle count of every block, as an (nz, ny, nx) array (2D: nz = 1)."""
    pos = np.asarray(pos, dtype=np.float64)
    d = pos.shape[1]
    nb = [int(v) for v in nblocks] + [1] * (3 - d)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    wrapped = pos.copy()
    for a in range(d):
        if periodic[a]:
            L = hi[a] - lo[a]
            wrapped[:, a] = lo[a] + np.mod(pos[:, a] - lo[a], L)
    k = block_index(wrapped, lo, hi, nblocks)
    c = np.bincount(k, minlength=nb[0] * nb[1] * nb[2])
    return c.reshape(nb[2], nb[1], nb[0])


def _neighbour(c, d, axis, periodic):
    """out[..., i, ...] = c[..., i + d, ...] along `axis`: wrapped when
    periodic, 0 past a wall."""
    if d == 0:
        return c
    if periodic:
        return np.roll(c, -d, axis=axis)
    out = np.zeros_like(c)
    n = c.shape[axis]
    if abs(d) >= n:
        return out
    src = [slice(None)] * c.ndim
    dst = [slice(None)] * c.ndim
    if d > 0:
        src[axis], dst[axis] = slice(d, n), slice(0, n - d)
    else:
        src[axis], dst[axis] = slice(0, n + d), slice(-d, n)
    out[tuple(dst)] = c[tuple(src)]
    return out


def block_counts27(pos, lo, hi, periodic, nblocks):
    """(B, 27) counts c_j of the blocks b + (dx, dy, dz) of every block b =
    i + n_x (j + n_y l) (0 past a wall), and (B,) the number of those 27
    blocks that lie inside the box."""
    c = block_counts(pos, lo, hi, periodic, nblocks).astype(np.float64)
    one = np.ones_like(c)
    per = list(periodic) + [False] * (3 - len(periodic))
    out = np.zeros((c.size, NIN))
    inside = np.zeros(c.size)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                j = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                # array axes are (z, y, x)
                sh, e = c, one
                for d, ax, p in ((dz, 0, per[2]), (dy, 1, per[1]), (dx, 2, per[0])):
                    sh = _neighbour(sh, d, ax, p)
                    e = _neighbour(e, d, ax, p)
                out[:, j] = sh.reshape(-1)
                inside += e.reshape(-1)
    return out, inside


def block_features(pos, lo, hi, periodic, nblocks):
    """(B, 27) features of every block: counts over their mean."""
    c, v = block_counts27(pos, lo, hi, periodic, nblocks)
    m = c.sum(axis=1) / np.maximum(v, 1.0)
    x = np.zeros_like(c)
    ok = m > 0
    x[ok] = c[ok] / m[ok, None] - 1.0
    return x


def kstar(pos, lo, hi, periodic, rmax, cells=None):
    """Candidates within 2R of each cell: the number of (j, image) pairs with
    |x_j + m L - x_i| < 2 R_i, excluding j = i with m = 0.  Positions on
    periodic axes are wrapped into the box first."""
    pos = np.asarray(pos, dtype=np.float64)
    n, d = pos.shape
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    x = pos.copy()
    for a in range(d):
        if periodic[a]:
            x[:, a] = lo[a] + np.mod(pos[:, a] - lo[a], L[a])
    idx = np.arange(n) if cells is None else np.asarray(cells)
    out = np.zeros(len(idx), dtype=np.int64)
    for o, i in enumerate(idx):
        R2 = 4.0 * rmax[o] ** 2
        reach = [int(np.ceil(2.0 * rmax[o] / L[a])) + 1 if periodic[a] else 0 for a in range(d)]
        grids = np.meshgrid(*[np.arange(-r, r + 1) for r in reach], indexing="ij")
        shifts = np.stack([g.reshape(-1) for g in grids], axis=1)
        cnt = 0
        for m in shifts:
            q = x + m * L - x[i]
            inside = np.einsum("ij,ij->i", q, q) < R2
            if not m.any():
                inside[i] = False
            cnt += int(inside.sum())
        out[o] = cnt
    return out


def block_targets(pos, lo, hi, periodic, nblocks, ks):
    """t_b = log(max(1, max k* over the block's cells)) and the mask of
    blocks that hold a particle; ks holds k* of every particle."""
    pos = np.asarray(pos, dtype=np.float64)
    d = pos.shape[1]
    wrapped = pos.copy()
    for a in range(d):
        if periodic[a]:
            wrapped[:, a] = lo[a] + np.mod(pos[:, a] - lo[a], hi[a] - lo[a])
    k = block_index(wrapped, lo, hi, nblocks)
    B = int(np.prod([int(v) for v in nblocks]))
    mx = np.full(B, -1, dtype=np.int64)
    np.maximum.at(mx, k, np.asarray(ks, dtype=np.int64))
    has = mx >= 0
    t = np.zeros(B)
    t[has] = np.log(np.maximum(1, mx[has]))
    return t, has


def forward(p, X):
    """Network output y for each row of X, with every intermediate."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3[0]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, t, u):
    y, _ = forward(p, X)
    e = y - np.asarray(t, dtype=np.float64)
    w = np.where(e < 0.0, u, 1.0)
    return float(np.mean(w * e * e))


def loss_grad(p, X, t, u):
    """L and dL/dp by the chain rule (ReLU derivative 0 at 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    M = X.shape[0]
    e = y - np.asarray(t, dtype=np.float64)
    w = np.where(e < 0.0, u, 1.0)
    L = float(np.mean(w * e * e))
    gy = 2.0 * w * e / M                   # dL/dy_b
    gW3 = h2.T @ gy
    gb3 = np.array([gy.sum()])
    gz2 = np.outer(gy, W3) * (z2 > 0.0)    # dL/dz2
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(axis=0)
    gz1 = (gz2 @ W2) * (z1 > 0.0)
    gW1 = gz1.T @ X
    gb1 = gz1.sum(axis=0)
    g = np.concatenate([gW1.reshape(-1), gb1, gW2.reshape(-1), gb2, gW3, gb3])
    return L, g


def adam(p, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * np.asarray(m) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(p) - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int = 0):
    """He-style initial weights (normal, std sqrt(2/fan_in)), zero biases and
    b3 = log(40), drawn from a seeded generator."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM)
    W1, b1, W2, b2, W3, b3 = unpack(p)
    W1[...] = rng.normal(0.0, np.sqrt(2.0 / NIN), W1.shape)
    W2[...] = rng.normal(0.0, np.sqrt(2.0 / H1), W2.shape)
    W3[...] = rng.normal(0.0, np.sqrt(1.0 / H2), W3.shape)
    b3[...] = np.log(40.0)
    return p
