"""The C ABI library builds, loads without a GPU, and exports every function
that include/*.h declares; the Python binding covers the same names."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(swe_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libswe():
    from paper_1107_2157_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("swe_create", "swe_create_ex", "swe_set_state", "swe_step", "swe_get_state",
              "swe_mass", "swe_cfl_dt", "swe_destroy", "swe_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(libswe):
    missing = [n for n in _declared() if not hasattr(libswe, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1107_2157_gb300 import swe
    assert set(_declared()) <= set(swe.declared_symbols())


def test_strerror_without_gpu(libswe):
    libswe.swe_strerror.restype = ctypes.c_char_p
    assert libswe.swe_strerror(0) == b"ok"
    assert libswe.swe_strerror(4) == b"device wait timed out"


def test_invalid_arguments_rejected_before_any_device_work(libswe):
    h = ctypes.c_void_p()
    f = libswe.swe_create
    f.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.POINTER(ctypes.c_void_p)]
    assert f(0, 10, 1.0, 1.0, 0.1, 9.8, ctypes.byref(h)) == 1
    assert f(10, 10, -1.0, 1.0, 0.1, 9.8, ctypes.byref(h)) == 1
    assert f(10, 10, 1.0, 1.0, float("nan"), 9.8, ctypes.byref(h)) == 1
    assert f(70000, 10, 1.0, 1.0, 0.1, 9.8, ctypes.byref(h)) == 1
    assert h.value is None
