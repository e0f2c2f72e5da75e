"""Argument checks of the Python binding, which run before any call reaches
the library (no GPU needed).  The library reads caller buffers through plain
pointers and cannot know their sizes, so a wrong shape, element type or
length must be refused here, before a kernel could read or write past the
end of a buffer."""
import numpy as np
import pytest
import torch

from paper_2209_11606_gb300 import vorogpu as V


def test_input_dtype_accepts_f64_and_f32():
    pos = np.zeros((5, 3))
    assert V._input_dtype(pos, None, 5, 3) == V.VG_F64
    assert V._input_dtype(pos.astype(np.float32), None, 5, 3) == V.VG_F32
    assert V._input_dtype(torch.zeros((4, 2), dtype=torch.float32), torch.ones(4, dtype=torch.float32),
                          4, 2) == V.VG_F32


@pytest.mark.parametrize("pos,radii,n,dim", [
    (np.zeros((5, 3), np.int64), None, 5, 3),            # not floating point
    (np.zeros((5, 2)), None, 5, 3),                      # wrong dimension
    (np.zeros(15), None, 5, 3),                          # flat
    (np.zeros((5, 3)), np.zeros(5, np.float32), 5, 3),   # mixed types
    (np.zeros((5, 3)), np.zeros(4), 5, 3),               # short radii
    (torch.zeros((5, 3), dtype=torch.float16), None, 5, 3),
])
def test_input_dtype_rejects(pos, radii, n, dim):
    with pytest.raises(ValueError):
        V._input_dtype(pos, radii, n, dim)


def _noalloc(pos, bs, order, nb=(2, 2, 2)):
    V.vg_sort_blocks_noalloc(3, [0, 0, 0], [1, 1, 1], (False,) * 3, nb, pos, bs, order)


@pytest.mark.parametrize("case", ["pos_f32", "pos_2d", "bs_short", "bs_i64", "order_short", "order_f32",
                                  "host_tensors"])
def test_noalloc_rejects_bad_buffers_before_the_call(case):
    n = 10
    pos = torch.zeros((n, 3), dtype=torch.float64)
    bs = torch.zeros(9, dtype=torch.int32)
    order = torch.zeros(n, dtype=torch.int32)
    if case == "pos_f32":
        pos = pos.float()
    elif case == "pos_2d":
        pos = torch.zeros((n, 2), dtype=torch.float64)
    elif case == "bs_short":
        bs = torch.zeros(8, dtype=torch.int32)
    elif case == "bs_i64":
        bs = torch.zeros(9, dtype=torch.int64)
    elif case == "order_short":
        order = torch.zeros(n - 1, dtype=torch.int32)
    elif case == "order_f32":
        order = torch.zeros(n, dtype=torch.float32)
    # "host_tensors": everything right except that the tensors live on the host
    with pytest.raises(ValueError):
        _noalloc(pos, bs, order)


def test_noalloc_rejects_a_grid_of_the_wrong_dimension():
    pos = torch.zeros((3, 3), dtype=torch.float64)
    with pytest.raises(ValueError):
        V.vg_sort_blocks_noalloc(3, [0, 0, 0], [1, 1, 1], (False,) * 3, (2, 2), pos,
                                 torch.zeros(9, dtype=torch.int32), torch.zeros(3, dtype=torch.int32))
