"""FP64 CPU oracle for the cell-based Voronoi method (arXiv 2209.11606).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library itself
never does.  The arithmetic lives in ``voro_oracle.c`` (plain C, FP64,
OpenMP over cells); this module compiles it with gcc on first use and wraps
it with ctypes.  It shares no code with the CUDA library.

Functions follow the paper:

* :func:`compute` -- Voronoi (or radical) cells: the box of Eqs. (1)-(2)
  clipped by the half-spaces of Eq. (3); ``method="brute"`` clips by every
  particle and periodic image (the definition, Sec. 2.1.2), ``method="grid"``
  walks the block grid outward and stops at the radius bound (Sec. 2.1.3);
  ``clip`` starts every cell from a cube centred on its particle (clipped
  cells, Sec. 3.1.3).
* :func:`grid_size` -- the block-count rule of Sec. 2.1.4.
* :func:`block_sort` -- the counting sort of particles into blocks
  (Sec. 2.1.1 and Sec. 2.2.5), written as a stable sort by block index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voro_oracle.c")
_LIB = os.path.join(_HERE, "libvoro_oracle.so")
_lock = threading.Lock()
_lib = None

# Band for "on the plane" (relative to mean spacing times |q|) and distance
# below which two points are one vertex (relative to mean spacing).
TAU_REL = 1e-11
MERGE_REL = 1e-9

ST_OK, ST_EMPTY, ST_CAP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile voro_oracle.c into a shared library next to it."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                   _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.vo_compute.restype = ctypes.c_int
        lib.vo_compute.argtypes = [ctypes.c_int, ctypes.c_longlong, P, P, P, P, P,
                                   ctypes.c_int, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_longlong, P, ctypes.c_int,
                                   P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int, P, P, P]
        lib.vo_grid_size.restype = None
        lib.vo_grid_size.argtypes = [ctypes.c_int, ctypes.c_longlong, P, P, ctypes.c_double,
                                     ctypes.c_int, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def grid_size(n: int, lo, hi, n_opt: float, rounding: str = "floor") -> tuple:
    """Block counts of Sec. 2.1.4: lambda = (N / (n_opt V))^(1/d),
    n_a = round(lambda L_a) >= 1, with rounding "ceil" (the text) or "floor"
    (what Table 3's numbers follow)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = np.zeros(len(lo), dtype=np.int32)
    lib.vo_grid_size(len(lo), n, _ptr(lo), _ptr(hi), float(n_opt),
                     1 if rounding == "floor" else 0, _ptr(out))
    return tuple(int(v) for v in out)


def block_index(pos, lo, hi, nblocks) -> np.ndarray:
    """Block k = i + n_x (j + n_y l) of each particle (Sec. 2.1.1, Fig. 3),
    with i = floor((x - a_x) / h_x) clamped to [0, n_x - 1]."""
    pos = np.asarray(pos, dtype=np.float64)
    d = pos.shape[1]
    k = np.zeros(pos.shape[0], dtype=np.int64)
    mul = 1
    for a in range(d):
        h = (hi[a] - lo[a]) / nblocks[a]
        b = np.floor((pos[:, a] - lo[a]) / h).astype(np.int64)
        b = np.clip(b, 0, nblocks[a] - 1)
        k += mul * b
        mul *= nblocks[a]
    return k


def block_sort(pos, lo, hi, nblocks):
    """Counting sort into blocks: returns (order, start) where `order` lists
    particle ids block by block (ascending id inside a block) and
    start[k]..start[k+1] is block k's range."""
    k = block_index(pos, lo, hi, nblocks)
    nblk = int(np.prod(nblocks))
    counts = np.bincount(k, minlength=nblk)
    start = np.zeros(nblk + 1, dtype=np.int64)
    np.cumsum(counts, out=start[1:])
    order = np.argsort(k, kind="stable")
    return order, start


def compute(pos, lo, hi, periodic, radii=None, method: str = "grid", nblocks=None,
            cells=None, maxf: int | None = None, threads: int = 0,
            tau_rel: float = TAU_REL, merge_rel: float = MERGE_REL, clip: float = 0.0,
            weinberg: bool = False) -> dict:
    """Cells of the particles `cells` (default: all).  Returns a dict of
    per-cell arrays (vol, area, centroid relative to the particle, nv, ne,
    nf, status, rmax, ntested, ncut) and a CSR of faces (face_off, nbr_id,
    nbr_img (n_faces x 3), face_order) in canonical order: ascending
    (neighbour id, image shift), walls (negative ids) first.  In 2D, `vol`
    is the area and `area` the perimeter.  `clip` > 0: clipped cells
    (Sec. 3.1.3), each starting from the box intersected with the cube (2D:
    square) of side `clip` centred on its particle, whose faces count as
    walls.  `weinberg`: also the Weinberg code of each 3D cell's edge graph
    (Sec. 4) as `w_len` (darts, 2E), `w_hash` (FNV-1a 64 over the 2E+1 vertex
    labels of the minimal code, two little-endian bytes each) and `w_sym` (the
    number of start darts and orientations that give it)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n, d = pos.shape
    if maxf is None:
        # face slots per cell: radical cells of large particles can have many
        maxf = (320 if radii is not None else 96) if d == 3 else (256 if radii is not None else 64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    per = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    rad = None if radii is None else np.ascontiguousarray(radii, dtype=np.float64)
    if method == "grid":
        if nblocks is None:
            nblocks = grid_size(n, lo, hi, 4.6 if d == 3 else 3.4, "floor")
        nb = np.ascontiguousarray(nblocks, dtype=np.int32)
        m = 1
    elif method == "brute":
        nb = np.ones(d, dtype=np.int32)
        m = 0
    else:
        raise ValueError(method)
    if cells is None:
        cl = None
        nc = n
    else:
        cl = np.ascontiguousarray(cells, dtype=np.int64)
        nc = len(cl)
    vol = np.zeros(nc)
    area = np.zeros(nc)
    cen = np.zeros((nc, d))
    nv = np.zeros(nc, dtype=np.int32)
    ne = np.zeros(nc, dtype=np.int32)
    nf = np.zeros(nc, dtype=np.int32)
    st = np.zeros(nc, dtype=np.int32)
    rmax = np.zeros(nc)
    ntest = np.zeros(nc, dtype=np.int64)
    ncut = np.zeros(nc, dtype=np.int64)
    sid = np.zeros((nc, maxf), dtype=np.int64)
    simg = np.zeros((nc, maxf, 3), dtype=np.int32)
    sord = np.zeros((nc, maxf), dtype=np.int32)
    wl = np.zeros(nc, dtype=np.int32) if weinberg else None
    wh = np.zeros(nc, dtype=np.uint64) if weinberg else None
    ws = np.zeros(nc, dtype=np.int32) if weinberg else None
    rc = lib.vo_compute(d, n, _ptr(pos), _ptr(rad), _ptr(lo), _ptr(hi), _ptr(per), m, _ptr(nb),
                        tau_rel, merge_rel, float(clip), nc, _ptr(cl), maxf,
                        _ptr(vol), _ptr(area), _ptr(cen), _ptr(nv), _ptr(ne), _ptr(nf), _ptr(st),
                        _ptr(sid), _ptr(simg), _ptr(sord), _ptr(rmax), _ptr(ntest), _ptr(ncut),
                        int(threads), _ptr(wl), _ptr(wh), _ptr(ws))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    nfc = np.where(st == ST_OK, nf, 0).astype(np.int64)
    off = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(nfc, out=off[1:])
    mask = np.arange(maxf)[None, :] < nfc[:, None]
    out = {
        "vol": vol, "area": area, "centroid": cen, "nv": nv, "ne": ne, "nf": nf,
        "status": st, "rmax": rmax, "ntested": ntest, "ncut": ncut,
        "face_off": off, "nbr_id": sid[mask], "nbr_img": simg[mask][:, :d] if d < 3 else simg[mask],
        "face_order": sord[mask],
    }
    if weinberg:
        out.update({"w_len": wl, "w_hash": wh, "w_sym": ws})
    return out
