"""The C-ABI library builds, loads and exports every entry point that include/tomo.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tomo.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tomo_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_12282_gb300 import _build, tomo
    if not os.path.exists(tomo.LIB_PATH):
        _build.build()
    return tomo.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["tomo_create_grid", "tomo_destroy_grid", "tomo_solve", "tomo_sensitivity",
              "tomo_filter", "tomo_oc_step", "tomo_gradient", "tomo_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_exports_every_declared_symbol(libpath):
    """The bounds-checked variant (-DTOMO_CHECKED) has the same boundary and says so."""
    from paper_2104_12282_gb300 import _build
    if not os.path.exists(_build.LIB_CHECKED):
        _build.build(checked=True)
    lib = ctypes.CDLL(_build.LIB_CHECKED)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    plain = ctypes.CDLL(libpath)
    for L, want in ((plain, 0),):
        c, w = ctypes.c_int32(-1), ctypes.c_uint64(7)
        assert L.tomo_check_report(ctypes.byref(c), ctypes.byref(w)) == 0
        assert c.value == want and w.value == 0


def test_binding_signatures_cover_header(libpath):
    from paper_2104_12282_gb300 import tomo
    assert set(tomo.exported_symbols()) == set(_declared())
    tomo.lib()


def test_create_rejects_bad_descriptor_without_gpu(libpath):
    """Argument validation happens before any device call."""
    from paper_2104_12282_gb300 import tomo
    L = tomo.lib()
    d = tomo.GridDesc()
    L.tomo_default_desc(ctypes.byref(d))
    d.nx = 0
    h = ctypes.c_void_p()
    st = L.tomo_create_grid(ctypes.byref(d), ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"dimensions" in L.tomo_last_error(None)


def test_device_footprint_estimate_without_gpu(libpath):
    """The footprint estimate used for admission is host arithmetic: it covers at least the
    nodal vectors CG needs, grows linearly with the grid beyond a fixed reserve, costs more
    in FP64, and rejects empty grids."""
    from paper_2104_12282_gb300 import problems as P
    from paper_2104_12282_gb300 import tomo
    p = P.mbb_192x96x76(0)
    ndof = 3 * p.dims.n_nodes
    e32 = tomo.estimate_device_bytes(p, precision=tomo.FP32)
    e64 = tomo.estimate_device_bytes(p, precision=tomo.FP64)
    # x (hi, lo), r, p, q and the level-0 smoother vectors: at least six FP32 nodal vectors
    assert 6 * 4 * ndof <= e32 <= 200 * ndof
    assert e64 > e32
    # beyond a fixed reserve, each added DOF costs at least the six FP32 vectors' 24 bytes
    small = P.cantilever(96, 48, 48)
    big = P.cantilever(192, 96, 96)
    grow = tomo.estimate_device_bytes(big) - tomo.estimate_device_bytes(small)
    per_dof = grow / (3 * (big.dims.n_nodes - small.dims.n_nodes))
    assert 24.0 <= per_dof <= 200.0
    L = tomo.lib()
    d = tomo.GridDesc()
    L.tomo_default_desc(ctypes.byref(d))
    d.nx = 0
    out = ctypes.c_size_t()
    assert L.tomo_estimate_device_bytes(ctypes.byref(d), ctypes.byref(out)) == 1
