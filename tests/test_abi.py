"""The C ABI library loads and exports every entry point include/*.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(vg_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2209_11606_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("vg_create", "vg_insert", "vg_compute", "vg_get_cells", "vg_get_faces",
              "vg_get_counts", "vg_destroy", "vg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2209_11606_gb300 import vorogpu
    assert set(vorogpu.EXPORTS) <= declared_functions()
    for n in vorogpu.EXPORTS:
        assert hasattr(vorogpu, n), n


def test_config_defaults_without_gpu(lib):
    from paper_2209_11606_gb300 import vorogpu
    cfg = vorogpu.vg_config_default()
    assert cfg.precision == vorogpu.VG_FP32_RETEST and cfg.order == vorogpu.VG_PREFETCH
    assert abs(cfg.tol32 - 1e-5) < 1e-20 and abs(cfg.tau_rel - 1e-11) < 1e-25
