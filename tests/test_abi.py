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


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, b"dimensions"),
    ("nz", -3, b"dimensions"),
    ("nx", 1290, b"32-bit"),          # 3 (nx+1)^3 >= 2^31 - 1 with ny = nz = 1290
    ("nu", 0.5, b"material"),
    ("nu", -1.0, b"material"),
    ("h", 0.0, b"material"),
    ("Emin", -1e-9, b"material"),
    ("E0", 0.0, b"material"),         # E0 <= Emin
    ("penal", 0.5, b"material"),
    ("rmin", 0.0, b"material"),
    ("rmin", 16.5, b"material"),
    ("precision", 7, b"precision"),
    ("precond", 9, b"preconditioner"),
])
def test_create_rejects_each_bad_field_without_gpu(libpath, field, value, msg):
    """Every descriptor check runs before any device call and names the problem."""
    from paper_2104_12282_gb300 import tomo
    L = tomo.lib()
    d = tomo.GridDesc()
    L.tomo_default_desc(ctypes.byref(d))
    d.nx, d.ny, d.nz = 4, 2, 2
    if field == "nx" and value == 1290:
        d.ny = d.nz = 1290
    fixed = (ctypes.c_uint8 * 3)()
    f = (ctypes.c_double * 3)()
    d.fixed_dof = ctypes.cast(fixed, ctypes.POINTER(ctypes.c_uint8))
    d.f = ctypes.cast(f, ctypes.POINTER(ctypes.c_double))
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert L.tomo_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value
    assert msg in L.tomo_last_error(None)


def test_create_needs_descriptor_and_arrays_without_gpu(libpath):
    from paper_2104_12282_gb300 import tomo
    L = tomo.lib()
    h = ctypes.c_void_p()
    assert L.tomo_create_grid(None, ctypes.byref(h)) == 1
    d = tomo.GridDesc()
    L.tomo_default_desc(ctypes.byref(d))
    d.nx, d.ny, d.nz = 4, 2, 2
    assert L.tomo_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1   # no fixed_dof / f
    assert b"required" in L.tomo_last_error(None)


@pytest.mark.parametrize("n_el", [0, -5, (1 << 22) + 1])
def test_no_alloc_oc_step_rejects_sizes_outside_its_scratch_without_gpu(libpath, n_el):
    """The allocation-free OC step checks the size against its static scratch first."""
    from paper_2104_12282_gb300 import tomo
    L = tomo.lib()
    one = (ctypes.c_float * 1)()
    st = L.tomo_oc_step_noalloc(ctypes.c_int64(n_el), ctypes.c_double(1.0), one, one, one,
                                ctypes.c_double(0.5), ctypes.c_double(0.2), one, None, None)
    assert st == 1
    assert b"4194304" in L.tomo_last_error(None)
