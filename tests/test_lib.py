"""CPU-side checks of the C-ABI library: it builds, loads without a GPU and exports every
entry point declared in include/fgb.h; host logic that needs no device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "fgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_1906_06317_gb300 as fgb
    return fgb.lib()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("fgb_nq_create", "fgb_nq_query", "fgb_nlist_arrays", "fgb_rdf_compute", "fgb_rdf_result",
                 "fgb_steinhardt_compute", "fgb_steinhardt_backward", "fgb_batch_run", "fgb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_symbol(lib):
    import paper_1906_06317_gb300 as fgb
    assert set(declared()) <= set(fgb._SIGS)


def test_host_side_argument_checks(lib):
    import ctypes
    import paper_1906_06317_gb300 as fgb
    assert lib.fgb_version() >= 10000
    h = ctypes.c_void_p()
    assert lib.fgb_rdf_create(0, 1.0, 0.0, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert b"bins" in lib.fgb_last_error()
    assert lib.fgb_rdf_create(10, 1.0, 2.0, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_steinhardt_create(13, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_nq_create(None, None, 0, 1.0, None, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    b = fgb.fgb_box(10.0, -1.0, 10.0, 0, 0, 0)
    assert lib.fgb_nq_create(ctypes.byref(b), None, 0, 1.0, None, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    # a 2D box (Lz = 0) must have xz = yz = 0
    b = fgb.fgb_box(10.0, 10.0, 0.0, 0.1, 0.2, 0.0)
    assert lib.fgb_nq_create(ctypes.byref(b), None, 0, 1.0, None, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert b"2D" in lib.fgb_last_error()
    # PMFT(x, y): extents and bin counts are checked on the host; a fresh accumulator
    # reports zero counts, pcf 0 and an infinite PMFT without touching the device
    assert lib.fgb_pmftxy_create(0.0, 1.0, 10, 10, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_pmftxy_create(1.0, float("inf"), 10, 10, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_pmftxy_create(1.0, 1.0, 0, 10, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_pmftxy_create(1.0, 1.0, 1 << 14, 1 << 13, ctypes.byref(h)) == fgb.ERR_INVALID_ARG
    assert lib.fgb_pmftxy_create(1.5, 1.0, 3, 2, ctypes.byref(h)) == 0
    import numpy as np
    c = np.full(6, 7, np.uint64)
    g = np.full(6, 7.0)
    f = np.zeros(6)
    assert lib.fgb_pmftxy_result(h, c.ctypes.data, g.ctypes.data, f.ctypes.data, None) == 0
    assert not c.any() and not g.any() and np.all(np.isinf(f))
    lib.fgb_pmftxy_destroy(h)
    # batched frames: tuning parameters are checked before any device work
    off = np.array([0, 10], np.int64)
    boxes = (fgb.fgb_box * 1)(fgb.fgb_box(10.0, 10.0, 10.0, 0, 0, 0))
    for bad in (dict(tile_cells=-2), dict(tile_cells=5000), dict(cell_div=3), dict(block=48),
                dict(hist_copies=5), dict(cells_per_warp=3), dict(cells_per_warp=16)):
        prm = fgb.fgb_batch_params(1.5, 6, 200, 3.0, 0.0, bad.get("cell_div", 0), bad.get("block", 0),
                                   bad.get("hist_copies", 0), bad.get("tile_cells", 0),
                                   bad.get("cells_per_warp", 0))
        assert lib.fgb_batch_create(1, off.ctypes.data, boxes, ctypes.byref(prm), None,
                                    ctypes.byref(h)) == fgb.ERR_INVALID_ARG, bad
        assert b"tuning" in lib.fgb_last_error()
    assert lib.fgb_batch_routes(None, None, None) == fgb.ERR_INVALID_ARG


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1906_06317_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
