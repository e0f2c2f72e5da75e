"""Seeded synthetic inputs for the cell-based Voronoi method.

This module only draws particle sets; it holds none of the method's
arithmetic (no block indices, no cuts, no statistics), so that both the CUDA
path and the FP64 oracle can take their inputs from here without sharing any
computation.  Every generator uses numpy's PCG64 (`numpy.random.default_rng`)
with an explicit seed.

Workloads (the paper's own are described in Sec. 3.1; the sizes below are the
ones this library is measured and tested on):

* ``uniform``      -- i.i.d. uniform points in a box (Sec. 3.1, "homogeneous").
* ``bcc`` / ``fcc`` / ``simple_cubic`` -- lattices in a periodic cube, with
  optional Gaussian position noise (Sec. 1 discusses BCC/FCC topology).
* ``square`` / ``hexagonal`` -- 2D lattices in a periodic box.
* ``radii_lognormal`` -- radical-tessellation radii, log-normal, rescaled to a
  target packing fraction.
* ``batched_systems`` -- many independent 3D systems of uneven size.
* ``fcc_uniform_slabs`` -- periodic cube split into z-slabs alternating
  perturbed FCC and uniform points.
* ``localized`` / ``extreme_clustering`` -- the paper's other two test
  arrangements (Sec. 3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    """One particle system: positions, box, periodicity and optional radii."""

    pos: np.ndarray                 # (n, d) float64
    lo: np.ndarray                  # (d,) float64
    hi: np.ndarray                  # (d,) float64
    periodic: tuple                 # d booleans
    radii: np.ndarray | None = None  # (n,) float64 or None
    tag: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.pos.shape[1]

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def uniform(n: int, dim: int = 3, side: float = 1.0, periodic: bool = False,
            seed: int = 0) -> System:
    """n points i.i.d. uniform in [0, side)^dim."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, dim)) * side
    return System(pos, np.zeros(dim), np.full(dim, float(side)),
                  (periodic,) * dim, tag="uniform")


def _lattice(basis: np.ndarray, m: int, a: float, sigma_frac: float,
             seed: int, tag: str) -> System:
    dim = basis.shape[1]
    grid = np.stack(np.meshgrid(*([np.arange(m)] * dim), indexing="ij"),
                    axis=-1).reshape(-1, dim).astype(np.float64)
    pos = (grid[:, None, :] + basis[None, :, :]).reshape(-1, dim) * a
    side = np.full(dim, m * a)
    if sigma_frac > 0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, sigma_frac * a, pos.shape)
        pos = np.mod(pos, side)
        pos = np.where(pos >= side, pos - side, pos)
    return System(pos, np.zeros(dim), side, (True,) * dim, tag=tag,
                  meta={"a": a, "m": m, "sigma": sigma_frac * a})


def simple_cubic(m: int, a: float = 1.0, sigma_frac: float = 0.0, seed: int = 0) -> System:
    return _lattice(np.zeros((1, 3)), m, a, sigma_frac, seed, "sc")


def bcc(m: int, a: float = 1.0, sigma_frac: float = 0.0, seed: int = 0) -> System:
    """Body-centred cubic, cube side a, m^3 unit cells (2 m^3 points)."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    return _lattice(basis, m, a, sigma_frac, seed, "bcc")


def fcc(m: int, a: float = 1.0, sigma_frac: float = 0.0, seed: int = 0) -> System:
    """Face-centred cubic, cube side a, m^3 unit cells (4 m^3 points)."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                      [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    return _lattice(basis, m, a, sigma_frac, seed, "fcc")


def square(m: int, a: float = 1.0, sigma_frac: float = 0.0, seed: int = 0) -> System:
    return _lattice(np.zeros((1, 2)), m, a, sigma_frac, seed, "square")


def hexagonal(nx: int, ny: int, side: tuple = (1.0, 1.0), sigma_frac: float = 0.0,
              seed: int = 0) -> System:
    """Hexagonal (triangular) lattice of nx columns x ny rows (ny even) in a
    periodic box; odd rows are shifted by half a column.  The row spacing is
    side_y/ny and the column spacing side_x/nx; the lattice is exactly regular
    when side_y/ny = (sqrt(3)/2) side_x/nx, otherwise slightly anisotropic.
    Noise sigma is `sigma_frac` times the column spacing."""
    if ny % 2:
        raise ValueError("ny must be even for a periodic hexagonal lattice")
    dx, dy = side[0] / nx, side[1] / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (i + 0.5 * (j % 2)) * dx
    y = j * dy
    pos = np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float64)
    sidev = np.array(side, dtype=np.float64)
    if sigma_frac > 0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, sigma_frac * dx, pos.shape)
        pos = np.mod(pos, sidev)
        pos = np.where(pos >= sidev, pos - sidev, pos)
    return System(pos, np.zeros(2), sidev, (True, True), tag="hex",
                  meta={"dx": dx, "dy": dy, "sigma": sigma_frac * dx})


def radii_lognormal(n: int, box_volume: float, packing: float, dim: int = 3,
                    sigma: float = 0.3, seed: int = 0) -> np.ndarray:
    """Log-normal radii exp(N(0, sigma^2)), rescaled so that the summed ball
    volume is `packing` times the box volume (overlaps allowed)."""
    rng = np.random.default_rng(seed)
    r = np.exp(rng.normal(0.0, sigma, n))
    unit = (4.0 / 3.0) * math.pi if dim == 3 else math.pi
    cur = unit * np.sum(r ** dim)
    return r * (packing * box_volume / cur) ** (1.0 / dim)


def radical_uniform(n: int, packing: float = 0.4, sigma: float = 0.3,
                    seed: int = 4) -> System:
    """n uniform points at unit density in a periodic cube with log-normal radii."""
    side = n ** (1.0 / 3.0)
    s = uniform(n, 3, side, True, seed)
    s.radii = radii_lognormal(n, side ** 3, packing, 3, sigma, seed + 1000)
    s.tag = "radical"
    return s


def localized(n_candidates: int, dim: int = 3, frac: float = 0.1, seed: int = 0) -> System:
    """Sec. 3.1 'localized': keep the points of a uniform set that fall in a
    centred square/cube of area/volume `frac`; walled unit box."""
    s = uniform(n_candidates, dim, 1.0, False, seed)
    half = 0.5 * frac ** (1.0 / dim)
    keep = np.all(np.abs(s.pos - 0.5) < half, axis=1)
    s.pos = s.pos[keep]
    s.tag = "localized"
    return s


def extreme_clustering(n: int, dim: int = 3, seed: int = 0) -> System:
    """Sec. 3.1 'extreme clustering': each coordinate 1/2 + 4 (X - 1/2)^3."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, dim))
    pos = 0.5 + 4.0 * (X - 0.5) ** 3
    return System(pos, np.zeros(dim), np.ones(dim), (False,) * dim, tag="clustered")


def corner_cluster(n_bg: int, n_cl: int, dim: int = 3, nb: int = 20, width: float = 2e-3,
                   seed: int = 0) -> System:
    """A uniform background of n_bg points in the walled unit box plus n_cl
    points uniform in a cube (square) `width` block sides across, centred
    on the block corner at the middle of an nb^dim grid: cells 1e-4 of a
    block and smaller next to the block boundary, as at the centre of the
    extreme-clustering set at 10^7-10^8 points, where block-relative FP32
    positions are coarse against the cells."""
    rng = np.random.default_rng(seed)
    h = 1.0 / nb
    corner = np.full(dim, (nb // 2) * h)
    bg = rng.random((n_bg, dim))
    cl = corner + (rng.random((n_cl, dim)) - 0.5) * (width * h)
    return System(np.concatenate([bg, cl]), np.zeros(dim), np.ones(dim), (False,) * dim, tag="corner_cluster")


def blobs(n: int, side: float, nblobs: int = 50, sigma_frac: float = 0.02,
          periodic: bool = True, seed: int = 0) -> System:
    """n points drawn from `nblobs` isotropic Gaussian blobs of std
    sigma_frac*side with uniform centres; wrapped if periodic, redrawn if
    they fall outside a walled box."""
    rng = np.random.default_rng(seed)
    centres = rng.random((nblobs, 3)) * side
    which = rng.integers(0, nblobs, n)
    pos = centres[which] + rng.normal(0.0, sigma_frac * side, (n, 3))
    sidev = np.full(3, side)
    if periodic:
        pos = np.mod(pos, sidev)
        pos = np.where(pos >= sidev, pos - sidev, pos)
    else:
        bad = np.any((pos < 0) | (pos >= side), axis=1)
        while bad.any():
            k = int(bad.sum())
            pos[bad] = centres[which[bad]] + rng.normal(0.0, sigma_frac * side, (k, 3))
            bad = np.any((pos < 0) | (pos >= side), axis=1)
    return System(pos, np.zeros(3), sidev, (periodic,) * 3, tag="blobs")


def batched_systems(nsys: int = 256, nmin: int = 1000, nmax: int = 200000,
                    seed: int = 5, scale: float = 1.0) -> list:
    """`nsys` independent 3D systems, sizes log-uniform in [nmin, nmax]
    (optionally scaled down by `scale`), each a uniform, perturbed-FCC
    (sigma 0.05 a) or 50-blob set at unit density, with each axis periodic
    with probability 1/2 (blob sets are all-periodic or all-walled)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nsys):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) * scale))
        n = max(n, 8)
        kind = int(rng.integers(0, 3))
        per = tuple(bool(b) for b in rng.integers(0, 2, 3))
        sub_seed = int(rng.integers(0, 2 ** 31))
        if kind == 0:
            side = n ** (1.0 / 3.0)
            s = uniform(n, 3, side, False, sub_seed)
            s.periodic = per
        elif kind == 1:
            m = max(1, int(round((n / 4) ** (1.0 / 3.0))))
            s = fcc(m, 1.0, 0.05, sub_seed)
            s.pos = np.mod(s.pos, s.hi)
            s.periodic = per
            # a walled axis must hold its points inside [lo, hi)
            s.pos = np.where(s.pos >= s.hi, s.pos - s.hi, s.pos)
            s.tag = "fcc"
        else:
            side = n ** (1.0 / 3.0)
            allper = bool(rng.integers(0, 2))
            s = blobs(n, side, 50, 0.02, allper, sub_seed)
            per = (allper,) * 3
            s.periodic = per
        out.append(s)
    return out


def fcc_uniform_slabs(cells_per_side: int = 296, slabs: int = 8, a: float = 51.0 / 32.0,
                      n_total: int = 102_400_000, sigma_frac: float = 0.05,
                      seed: int = 6) -> System:
    """Periodic cube of side cells_per_side*a split into `slabs` z-slabs that
    alternate perturbed FCC (even slabs) and uniform points (odd slabs); the
    uniform slabs share n_total minus the FCC count."""
    m = cells_per_side
    if m % slabs:
        raise ValueError("cells_per_side must divide into slabs")
    per_slab = m // slabs
    side = m * a
    rng = np.random.default_rng(seed)
    parts = []
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                      [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    n_fcc = 4 * m * m * per_slab * (slabs // 2)
    n_uni = n_total - n_fcc
    uni_each = [n_uni // (slabs // 2) + (1 if k < n_uni % (slabs // 2) else 0)
                for k in range(slabs // 2)]
    ix, iy = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    ixy = np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float64)
    for s in range(slabs):
        z0 = s * per_slab
        if s % 2 == 0:
            for kz in range(per_slab):
                cell = np.concatenate([ixy, np.full((ixy.shape[0], 1), z0 + kz)], axis=1)
                p = (cell[:, None, :] + basis[None]).reshape(-1, 3) * a
                parts.append(p + rng.normal(0.0, sigma_frac * a, p.shape))
        else:
            k = uni_each[s // 2]
            p = rng.random((k, 3)) * np.array([side, side, per_slab * a])
            p[:, 2] += z0 * a
            parts.append(p)
    pos = np.concatenate(parts, axis=0)
    sidev = np.full(3, side)
    pos = np.mod(pos, sidev)
    pos = np.where(pos >= sidev, pos - sidev, pos)
    return System(pos, np.zeros(3), sidev, (True,) * 3, tag="fcc_uniform_slabs",
                  meta={"a": a, "n_fcc": n_fcc})


# --- the named workloads -------------------------------------------------------

def workload(name: str) -> System:
    """Named workloads with fixed seeds and sizes (see module docstring)."""
    if name == "unit1000":          # 1,000 uniform points, walled unit cube, 6^3 grid
        s = uniform(1000, 3, 1.0, False, 0)
        s.meta["grid"] = (6, 6, 6)
        return s
    if name == "uniform1m":         # 1M uniform, periodic side-100 cube, 58^3 grid
        s = uniform(1_000_000, 3, 100.0, True, 1)
        s.meta["grid"] = (58, 58, 58)
        return s
    if name == "bcc1m":             # BCC a=1.25, 80^3 cells, sigma = 0.02 a
        s = bcc(80, 1.25, 0.02, 2)
        s.meta["grid"] = (64, 64, 64)
        return s
    if name == "hex10m":            # 2D perturbed hexagonal, 2943 x 3398
        s = hexagonal(2943, 3398, (1.0, 1.0), 0.05, 3)
        return s
    if name == "radical2m":         # 3D radical, 2M points, packing 0.4
        return radical_uniform(2_000_000, 0.4, 0.3, 4)
    raise KeyError(name)
