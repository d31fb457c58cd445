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
