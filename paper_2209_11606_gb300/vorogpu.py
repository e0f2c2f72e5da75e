"""Python binding of libvorogpu (include/vorogpu.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain pointers through ctypes; all computation runs in the library's CUDA
kernels.  PyTorch is used for device memory and streams: tensors are passed
by ``data_ptr()``.  If the shared library has not been built the import-time
loader raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvorogpu.so")

VG_OK = 0
STATUS_NAMES = {0: "VG_OK", 1: "VG_ERR_ARG", 2: "VG_ERR_OOM", 3: "VG_ERR_OUT_OF_BOX",
                4: "VG_ERR_NONFINITE", 5: "VG_ERR_CAP", 6: "VG_ERR_CUDA", 7: "VG_ERR_STATE",
                8: "VG_ERR_DUP_POINT"}
STATUS_CODES = {v: k for k, v in STATUS_NAMES.items()}
VG_F64, VG_F32 = 0, 1
VG_FP64, VG_FP32_RETEST = 0, 1
VG_WALK, VG_PREFETCH = 0, 1
VG_CELL_OK, VG_CELL_EMPTY, VG_CELL_CAP, VG_CELL_DUP, VG_CELL_LIMIT = 0, 1, 2, 3, 4

EXPORTS = ["vg_config_default", "vg_create", "vg_batch_create", "vg_insert", "vg_batch_insert",
           "vg_compute", "vg_compute_subset", "vg_get_counts", "vg_get_cells", "vg_get_faces", "vg_get_work",
           "vg_get_radius", "vg_get_weinberg", "vg_get_sorted", "vg_get_grid", "vg_get_system_grid", "vg_get_launches",
           "vg_get_kernel_ms", "vg_get_sort_ms", "vg_get_deferred", "vg_set_system_split", "vg_graph_capture", "vg_graph_launch", "vg_graph_sync",
           "vg_sort_blocks_noalloc", "vg_last_error", "vg_destroy",
           "vg_mlp_create", "vg_mlp_destroy", "vg_mlp_last_error", "vg_mlp_set_params",
           "vg_mlp_get_params", "vg_mlp_features", "vg_mlp_labels", "vg_mlp_dataset",
           "vg_mlp_loss_grad", "vg_mlp_train", "vg_mlp_infer", "vg_mlp_predict", "vg_set_predictor"]
MLP_NPARAM = 1985


class VgConfig(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("order", ctypes.c_int), ("tol32", ctypes.c_double),
                ("tau_rel", ctypes.c_double), ("merge_rel", ctypes.c_double),
                ("prefetch_k", ctypes.c_int), ("use_mlp", ctypes.c_int), ("chunk", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("collect_stats", ctypes.c_int),
                ("time_kernels", ctypes.c_int), ("clip", ctypes.c_double), ("weinberg", ctypes.c_int),
                ("split", ctypes.c_int)]


class VgSystem(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("nblocks", ctypes.c_int * 3),
                ("n_opt", ctypes.c_double)]


class VgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Loads the shared library (build it with paper_2209_11606_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libvorogpu.so not built at {path}; run paper_2209_11606_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "vg_config_default": (None, [ctypes.POINTER(VgConfig)]),
        "vg_create": (I, [ctypes.POINTER(P), I, P, P, P, P, D, P]),
        "vg_batch_create": (I, [ctypes.POINTER(P), I, I, ctypes.POINTER(VgSystem), P]),
        "vg_insert": (I, [P, L, P, P, I, I]),
        "vg_batch_insert": (I, [P, P, P, P, I, I]),
        "vg_compute": (I, [P, ctypes.POINTER(VgConfig)]),
        "vg_compute_subset": (I, [P, ctypes.POINTER(VgConfig), P, L, I]),
        "vg_graph_capture": (I, [P, P, P, P, I, ctypes.POINTER(VgConfig)]),
        "vg_graph_launch": (I, [P]),
        "vg_graph_sync": (I, [P]),
        "vg_get_counts": (I, [P, ctypes.POINTER(L), ctypes.POINTER(L)]),
        "vg_get_cells": (I, [P, P, P, P, P, P, P, P, I]),
        "vg_get_faces": (I, [P, P, P, P, P, I]),
        "vg_get_work": (I, [P, P, P, P, P, P, P, P, I]),
        "vg_get_radius": (I, [P, P, I]),
        "vg_get_weinberg": (I, [P, P, P, P, I]),
        "vg_get_kernel_ms": (I, [P, ctypes.POINTER(D), ctypes.POINTER(L)]),
        "vg_get_sort_ms": (I, [P, ctypes.POINTER(D), ctypes.POINTER(L)]),
        "vg_get_deferred": (I, [P, ctypes.POINTER(L)]),
        "vg_set_system_split": (I, [P, I, I]),
        "vg_get_sorted": (I, [P, ctypes.POINTER(L), P, P, I]),
        "vg_get_grid": (I, [P, P]),
        "vg_get_system_grid": (I, [P, I, P]),
        "vg_get_launches": (I, [P, ctypes.POINTER(L)]),
        "vg_sort_blocks_noalloc": (I, [I, P, P, P, P, L, P, P, P, P, ctypes.c_char_p, I]),
        "vg_last_error": (ctypes.c_char_p, [P]),
        "vg_mlp_create": (I, [ctypes.POINTER(P), P]),
        "vg_mlp_destroy": (None, [P]),
        "vg_mlp_last_error": (ctypes.c_char_p, [P]),
        "vg_mlp_set_params": (I, [P, P]),
        "vg_mlp_get_params": (I, [P, P]),
        "vg_mlp_features": (I, [P, P, I]),
        "vg_mlp_labels": (I, [P, P, I]),
        "vg_mlp_dataset": (I, [P, P, P, ctypes.POINTER(L)]),
        "vg_mlp_loss_grad": (I, [P, P, P, L, ctypes.c_float, ctypes.POINTER(D), P]),
        "vg_mlp_train": (I, [P, P, P, L, ctypes.c_float, ctypes.c_float, I, P]),
        "vg_mlp_infer": (I, [P, P, L, P]),
        "vg_mlp_predict": (I, [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "vg_set_predictor": (I, [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "vg_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx, code):
    if code != VG_OK:
        msg = _lib.vg_last_error(ctx).decode() if ctx else ""
        raise VgError(code, msg)


def _ptr(x):
    """Address of a numpy array or torch tensor, and whether it is on a GPU."""
    if x is None:
        return None, 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    # torch tensor
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if x.is_cuda:
        import torch
        if x.device.index != torch.cuda.current_device():
            raise ValueError(f"tensor is on {x.device}, but the current device is "
                             f"cuda:{torch.cuda.current_device()}")
    return x.data_ptr(), 1 if x.is_cuda else 0


def _dtype_name(x) -> str:
    """'float64', 'float32', 'int32', ... of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.dtype.name
    return str(x.dtype).replace("torch.", "")


def _numel(x) -> int:
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _input_dtype(pos, radii, n, dim):
    """VG_F64 or VG_F32 for positions of shape (n, dim) and radii of shape
    (n,) of one floating type; anything else raises before the library can
    read past a buffer."""
    dt = _dtype_name(pos)
    if dt not in ("float64", "float32"):
        raise ValueError(f"positions must be float64 or float32, not {dt}")
    if tuple(pos.shape) != (n, dim):
        raise ValueError(f"positions must have shape ({n}, {dim}), not {tuple(pos.shape)}")
    if radii is not None:
        if _dtype_name(radii) != dt:
            raise ValueError("radii must have the positions' dtype")
        if tuple(radii.shape) != (n,):
            raise ValueError(f"radii must have shape ({n},), not {tuple(radii.shape)}")
    return VG_F32 if dt == "float32" else VG_F64


# dimension of every live container, by handle value (inputs are checked
# against it before they reach the library)
_ctx_dim: dict = {}


def _dim_of(ctx) -> int:
    key = ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx
    if key not in _ctx_dim:
        raise ValueError("not a live container")
    return _ctx_dim[key]


def vg_config_default() -> VgConfig:
    cfg = VgConfig()
    load().vg_config_default(ctypes.byref(cfg))
    return cfg


def vg_create(dim, lo, hi, periodic, nblocks=None, n_opt=0.0, stream=None):
    lib = load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    per = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    nb = None if nblocks is None else np.ascontiguousarray(nblocks, dtype=np.int32)
    h = ctypes.c_void_p()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    code = lib.vg_create(ctypes.byref(h), int(dim), lo.ctypes.data, hi.ctypes.data, per.ctypes.data,
                         None if nb is None else nb.ctypes.data, float(n_opt), st)
    if code != VG_OK:
        raise VgError(code, "vg_create failed")
    _ctx_dim[h.value] = int(dim)
    return h


def vg_system(lo, hi, periodic, nblocks=None, n_opt=0.0) -> VgSystem:
    """One system of a batched container (the arguments of vg_create)."""
    s = VgSystem()
    for a in range(len(lo)):
        s.lo[a] = float(lo[a])
        s.hi[a] = float(hi[a])
        s.periodic[a] = 1 if periodic[a] else 0
        s.nblocks[a] = 0 if nblocks is None else int(nblocks[a])
    s.n_opt = float(n_opt)
    return s


def vg_batch_create(dim, systems, stream=None):
    lib = load()
    arr = (VgSystem * len(systems))(*systems)
    h = ctypes.c_void_p()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    code = lib.vg_batch_create(ctypes.byref(h), int(dim), len(systems), arr, st)
    if code != VG_OK:
        raise VgError(code, "vg_batch_create failed")
    _ctx_dim[h.value] = int(dim)
    return h


def vg_batch_insert(ctx, counts, pos, radii=None):
    """`counts[k]` rows of `pos` (and `radii`) belong to system k, systems
    one after another."""
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    p, dev = _ptr(pos)
    r, rdev = _ptr(radii)
    if radii is not None and rdev != dev:
        raise ValueError("pos and radii must both be host or both device")
    if int(cnt.sum()) != pos.shape[0]:
        raise ValueError("counts do not add up to the rows of pos")
    dt = _input_dtype(pos, radii, int(cnt.sum()), _dim_of(ctx))
    _check(ctx, load().vg_batch_insert(ctx, cnt.ctypes.data, p, r, dt, dev))


def vg_insert(ctx, pos, radii=None):
    """Positions (n, dim) and optional radii (n,), float64 or float32 (one
    type for both), numpy arrays or CUDA tensors on the current device."""
    p, dev = _ptr(pos)
    r, rdev = _ptr(radii)
    if radii is not None and rdev != dev:
        raise ValueError("pos and radii must both be host or both device")
    n = pos.shape[0]
    dt = _input_dtype(pos, radii, n, _dim_of(ctx))
    _check(ctx, load().vg_insert(ctx, n, p, r, dt, dev))


def vg_compute(ctx, cfg: VgConfig | None = None):
    _check(ctx, load().vg_compute(ctx, None if cfg is None else ctypes.byref(cfg)))


def vg_compute_subset(ctx, cells, cfg: VgConfig | None = None):
    """Computes the cells whose input indices are listed (int32 numpy array
    or CUDA tensor)."""
    if isinstance(cells, np.ndarray):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
    p, dev = _ptr(cells)
    _check(ctx, load().vg_compute_subset(ctx, None if cfg is None else ctypes.byref(cfg), p,
                                         int(cells.shape[0]), dev))


def vg_graph_capture(ctx, counts, pos, radii=None, cfg: VgConfig | None = None):
    """Captures sort -> cells -> faces of device tensors `pos` (and `radii`)
    into a CUDA graph owned by `ctx`; `counts` per system."""
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    p, dev = _ptr(pos)
    r, rdev = _ptr(radii)
    if not dev or (radii is not None and not rdev):
        raise ValueError("graph inputs must be CUDA tensors")
    if int(cnt.sum()) != pos.shape[0]:
        raise ValueError("counts do not add up to the rows of pos")
    dt = _input_dtype(pos, radii, int(cnt.sum()), _dim_of(ctx))
    _check(ctx, load().vg_graph_capture(ctx, cnt.ctypes.data, p, r, dt,
                                        None if cfg is None else ctypes.byref(cfg)))


def vg_graph_launch(ctx):
    _check(ctx, load().vg_graph_launch(ctx))


def vg_graph_sync(ctx):
    _check(ctx, load().vg_graph_sync(ctx))


def vg_get_counts(ctx):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().vg_get_counts(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def vg_get_cells(ctx, vol=None, area=None, centroid=None, nv=None, ne=None, nf=None, status=None):
    arrs = [vol, area, centroid, nv, ne, nf, status]
    dev = {(_ptr(a)[1]) for a in arrs if a is not None}
    if len(dev) > 1:
        raise ValueError("outputs must all be host or all device")
    on_dev = dev.pop() if dev else 0
    _check(ctx, load().vg_get_cells(ctx, *[_ptr(a)[0] for a in arrs], on_dev))


def vg_get_faces(ctx, face_off=None, nbr_id=None, nbr_img=None, face_order=None):
    arrs = [face_off, nbr_id, nbr_img, face_order]
    dev = {(_ptr(a)[1]) for a in arrs if a is not None}
    on_dev = dev.pop() if dev else 0
    _check(ctx, load().vg_get_faces(ctx, *[_ptr(a)[0] for a in arrs], on_dev))


def vg_get_work(ctx, n_tested=None, n_vtests=None, n_cuts=None, n_newv=None, n_retest=None,
                fallback=None, n_prefetch=None):
    arrs = [n_tested, n_vtests, n_cuts, n_newv, n_retest, fallback, n_prefetch]
    dev = {(_ptr(a)[1]) for a in arrs if a is not None}
    on_dev = dev.pop() if dev else 0
    _check(ctx, load().vg_get_work(ctx, *[_ptr(a)[0] for a in arrs], on_dev))


def vg_get_radius(ctx, rmax):
    p, dev = _ptr(rmax)
    _check(ctx, load().vg_get_radius(ctx, p, dev))


def vg_get_weinberg(ctx, length, hash_, sym):
    """Weinberg codes of the last compute with cfg.weinberg = 1: darts (2E,
    0 = none), FNV-1a 64 hash of the minimal code, symmetry count."""
    ptrs = [_ptr(a) for a in (length, hash_, sym)]
    if len({d for _, d in ptrs}) > 1:
        raise ValueError("outputs must all be host or all device")
    _check(ctx, load().vg_get_weinberg(ctx, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[0][1]))


def vg_get_sorted(ctx, block_start=None, order=None):
    nb = ctypes.c_int64()
    arrs = [block_start, order]
    dev = {(_ptr(a)[1]) for a in arrs if a is not None}
    on_dev = dev.pop() if dev else 0
    _check(ctx, load().vg_get_sorted(ctx, ctypes.byref(nb), *[_ptr(a)[0] for a in arrs], on_dev))
    return nb.value


def vg_get_grid(ctx, dim):
    out = np.zeros(dim, dtype=np.int32)
    _check(ctx, load().vg_get_grid(ctx, out.ctypes.data))
    return tuple(int(v) for v in out)


def vg_get_system_grid(ctx, k, dim):
    out = np.zeros(dim, dtype=np.int32)
    _check(ctx, load().vg_get_system_grid(ctx, int(k), out.ctypes.data))
    return tuple(int(v) for v in out)


def vg_get_kernel_ms(ctx):
    t, c = ctypes.c_double(), ctypes.c_int64()
    _check(ctx, load().vg_get_kernel_ms(ctx, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def vg_get_sort_ms(ctx):
    t, c = ctypes.c_double(), ctypes.c_int64()
    _check(ctx, load().vg_get_sort_ms(ctx, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def vg_get_deferred(ctx):
    v = ctypes.c_int64()
    _check(ctx, load().vg_get_deferred(ctx, ctypes.byref(v)))
    return v.value


def vg_set_system_split(ctx, k, split):
    _check(ctx, load().vg_set_system_split(ctx, int(k), int(split)))


def vg_get_launches(ctx):
    v = ctypes.c_int64()
    _check(ctx, load().vg_get_launches(ctx, ctypes.byref(v)))
    return v.value


def vg_sort_blocks_noalloc(dim, lo, hi, periodic, nblocks, pos, block_start, order, stream=None):
    """Counting sort into blocks with no device allocation (see vorogpu.h):
    `pos` (n, dim) float64, `block_start` (>= B + 1) and `order` (>= n)
    int32, all CUDA tensors on the current device; raises ValueError before
    the call on any other shape, type or device (the library cannot check
    the sizes of caller buffers), and VgError with the library's reason on
    failure."""
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    per = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    nb = np.ascontiguousarray(nblocks, dtype=np.int32)
    dim = int(dim)
    if dim not in (2, 3) or lo.shape != (dim,) or hi.shape != (dim,) or per.shape != (dim,) or nb.shape != (dim,):
        raise ValueError("lo, hi, periodic and nblocks must each hold dim (2 or 3) entries")
    n = int(pos.shape[0])
    if _dtype_name(pos) != "float64" or tuple(pos.shape) != (n, dim):
        raise ValueError(f"pos must be float64 of shape (n, {dim})")
    nblk = int(np.prod(nb.astype(np.int64)))
    if _dtype_name(block_start) != "int32" or _numel(block_start) < nblk + 1:
        raise ValueError(f"block_start must be int32 with at least {nblk + 1} entries")
    if _dtype_name(order) != "int32" or _numel(order) < n:
        raise ValueError(f"order must be int32 with at least {n} entries")
    for t in (pos, block_start, order):
        if _ptr(t)[1] != 1:
            raise ValueError("pos, block_start and order must be CUDA tensors")
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    buf = ctypes.create_string_buffer(256)
    code = load().vg_sort_blocks_noalloc(dim, lo.ctypes.data, hi.ctypes.data, per.ctypes.data,
                                         nb.ctypes.data, n, pos.data_ptr(),
                                         block_start.data_ptr(), order.data_ptr(), st, buf, 256)
    if code != VG_OK:
        raise VgError(code, buf.value.decode())


def vg_last_error(ctx) -> str:
    return load().vg_last_error(ctx).decode()


def vg_mlp_last_error(m) -> str:
    return load().vg_mlp_last_error(m).decode()


def vg_destroy(ctx):
    if ctx:
        _ctx_dim.pop(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx, None)
        load().vg_destroy(ctx)


# ---- learned candidate count ------------------------------------------------------

def _mcheck(m, code):
    if code != VG_OK:
        msg = _lib.vg_mlp_last_error(m).decode() if m else ""
        raise VgError(code, msg)


def _dev_ptr(x, what):
    p, dev = _ptr(x)
    if not dev:
        raise ValueError(f"{what} must be a CUDA tensor")
    return p


def vg_mlp_create(stream=None):
    h = ctypes.c_void_p()
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    code = load().vg_mlp_create(ctypes.byref(h), st)
    if code != VG_OK:
        raise VgError(code, "vg_mlp_create failed")
    return h


def vg_mlp_destroy(m):
    if m:
        load().vg_mlp_destroy(m)


def vg_mlp_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (MLP_NPARAM,):
        raise ValueError(f"params must hold {MLP_NPARAM} floats")
    _mcheck(m, load().vg_mlp_set_params(m, p.ctypes.data))


def vg_mlp_get_params(m):
    p = np.zeros(MLP_NPARAM, np.float32)
    _mcheck(m, load().vg_mlp_get_params(m, p.ctypes.data))
    return p


def vg_mlp_features(ctx, X):
    p, dev = _ptr(X)
    _check(ctx, load().vg_mlp_features(ctx, p, dev))


def vg_mlp_labels(ctx, kstar):
    p, dev = _ptr(kstar)
    _check(ctx, load().vg_mlp_labels(ctx, p, dev))


def vg_mlp_dataset(ctx, X, t):
    """Training rows into device tensors X (>= blocks x 27) and t (>= blocks);
    returns the number of rows."""
    m = ctypes.c_int64()
    _check(ctx, load().vg_mlp_dataset(ctx, _dev_ptr(X, "X"), _dev_ptr(t, "t"), ctypes.byref(m)))
    return m.value


def vg_mlp_loss_grad(m, X, t, M, u):
    loss = ctypes.c_double()
    g = np.zeros(MLP_NPARAM, np.float32)
    _mcheck(m, load().vg_mlp_loss_grad(m, _dev_ptr(X, "X"), _dev_ptr(t, "t"), int(M), float(u),
                                       ctypes.byref(loss), g.ctypes.data))
    return loss.value, g


def vg_mlp_train(m, X, t, M, u, lr, steps):
    losses = np.zeros(max(int(steps), 1), np.float32)
    _mcheck(m, load().vg_mlp_train(m, _dev_ptr(X, "X"), _dev_ptr(t, "t"), int(M), float(u), float(lr),
                                   int(steps), losses.ctypes.data))
    return losses[:int(steps)]


def vg_mlp_infer(m, X, M, y):
    _mcheck(m, load().vg_mlp_infer(m, _dev_ptr(X, "X"), int(M), _dev_ptr(y, "y")))


def vg_mlp_predict(ctx, m, alpha=1.0, kmin=8.0, kmax=1024.0):
    _check(ctx, load().vg_mlp_predict(ctx, m, float(alpha), float(kmin), float(kmax)))


def vg_set_predictor(ctx, m, alpha=1.0, kmin=8.0, kmax=1024.0):
    _check(ctx, load().vg_set_predictor(ctx, m, float(alpha), float(kmin), float(kmax)))


# ---- convenience: one call from host arrays to host results -------------------

def _make_cfg(precision, order, work, cfg_kw) -> VgConfig:
    cfg = vg_config_default()
    cfg.precision = VG_FP64 if precision == "fp64" else VG_FP32_RETEST
    cfg.order = VG_WALK if order == "walk" else VG_PREFETCH
    cfg.collect_stats = 1 if work else 0
    for k, v in cfg_kw.items():
        setattr(cfg, k, v)
    return cfg


def _fetch(ctx, n, d, work) -> dict:
    ncell, nface = vg_get_counts(ctx)
    out = {
        "vol": np.zeros(n), "area": np.zeros(n), "centroid": np.zeros((n, d)),
        "nv": np.zeros(n, np.int32), "ne": np.zeros(n, np.int32), "nf": np.zeros(n, np.int32),
        "status": np.zeros(n, np.uint8),
    }
    vg_get_cells(ctx, out["vol"], out["area"], out["centroid"], out["nv"], out["ne"], out["nf"],
                 out["status"])
    fo = np.zeros(n + 1, np.int64)
    ids = np.zeros(max(nface, 1), np.int32)
    img = np.zeros((max(nface, 1), 3), np.int8)
    order_ = np.zeros(max(nface, 1), np.uint8)
    vg_get_faces(ctx, fo, ids, img, order_)
    out.update({"face_off": fo, "nbr_id": ids[:nface], "nbr_img": img[:nface, :d],
                "face_order": order_[:nface]})
    rfin = np.zeros(n, np.float32)
    vg_get_radius(ctx, rfin)
    out["rmax"] = rfin
    if work:
        w = {k: np.zeros(n, np.int32)
             for k in ("n_tested", "n_vtests", "n_cuts", "n_newv", "n_retest", "n_prefetch")}
        fb = np.zeros(n, np.uint8)
        vg_get_work(ctx, w["n_tested"], w["n_vtests"], w["n_cuts"], w["n_newv"], w["n_retest"], fb,
                    w["n_prefetch"])
        w["fallback"] = fb
        out["work"] = w
    return out


def compute_host(pos, lo, hi, periodic, radii=None, nblocks=None, n_opt=0.0, precision="fp32",
                 order="prefetch", work=False, **cfg_kw) -> dict:
    """Runs insert + compute on the current CUDA device from host numpy arrays
    and returns host numpy results in the oracle's layout."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n, d = pos.shape
    ctx = vg_create(d, lo, hi, periodic, nblocks, n_opt)
    try:
        vg_insert(ctx, pos, None if radii is None else np.ascontiguousarray(radii, dtype=np.float64))
        vg_compute(ctx, _make_cfg(precision, order, work, cfg_kw))
        out = _fetch(ctx, n, d, work)
        out["grid"] = vg_get_grid(ctx, d)
        if cfg_kw.get("weinberg"):
            wl, wh, ws = np.zeros(n, np.int32), np.zeros(n, np.uint64), np.zeros(n, np.int32)
            vg_get_weinberg(ctx, wl, wh, ws)
            out.update({"w_len": wl, "w_hash": wh, "w_sym": ws})
        return out
    finally:
        vg_destroy(ctx)


def compute_batch_host(systems, pos_list, radii_list=None, precision="fp32", order="prefetch",
                       work=False, **cfg_kw) -> dict:
    """Batched form of :func:`compute_host`: `systems` is a list of VgSystem,
    `pos_list[k]` the host positions of system k.  Results are concatenated
    in system order (neighbour ids in the concatenated numbering)."""
    d = pos_list[0].shape[1]
    counts = [p.shape[0] for p in pos_list]
    pos = np.ascontiguousarray(np.concatenate(pos_list), dtype=np.float64)
    rad = None if radii_list is None else np.ascontiguousarray(np.concatenate(radii_list), dtype=np.float64)
    ctx = vg_batch_create(d, systems)
    try:
        vg_batch_insert(ctx, counts, pos, rad)
        vg_compute(ctx, _make_cfg(precision, order, work, cfg_kw))
        out = _fetch(ctx, pos.shape[0], d, work)
        out["grids"] = [vg_get_system_grid(ctx, k, d) for k in range(len(systems))]
        return out
    finally:
        vg_destroy(ctx)
