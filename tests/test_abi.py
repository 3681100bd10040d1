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


def test_more_entry_points_reject_bad_arguments_before_device_work(libswe):
    """Each call below fails its argument checks, which the header states run
    before any device work, so it returns SWE_EINVAL (1) on a machine without a GPU."""
    c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
    EINVAL = 1
    out = c_void_p()
    fake = c_void_p(64)  # never dereferenced: the checks reject the call first

    bc = libswe.swe_batch_create
    bc.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)] + [ctypes.POINTER(c_double)] * 3 + \
        [c_double, ctypes.POINTER(c_void_p)]

    def batch(nx, ny, dx=1.0, dy=1.0, dt=0.1, g=9.8):
        n = len(nx)
        ia = lambda v: (c_int * n)(*v)  # noqa: E731
        da = lambda v: (c_double * n)(*([v] * n))  # noqa: E731
        return bc(n, ia(nx), ia(ny), da(dx), da(dy), da(dt), g, ctypes.byref(out))

    assert bc(0, None, None, None, None, None, 9.8, ctypes.byref(out)) == EINVAL
    assert batch([64, 0], [64, 64]) == EINVAL
    assert batch([64, 70000], [64, 64]) == EINVAL
    assert batch([64], [64], dt=-0.1) == EINVAL
    assert batch([64], [64], dx=float("inf")) == EINVAL
    assert batch([64], [64], g=float("nan")) == EINVAL
    assert out.value is None

    nc = libswe.swe_net_create
    nc.argtypes = [c_int, c_int, c_int, ctypes.POINTER(c_void_p)]
    assert nc(0, 256, 256, ctypes.byref(out)) == EINVAL
    assert nc(4, 8193, 256, ctypes.byref(out)) == EINVAL
    assert nc(4, 256, 0, ctypes.byref(out)) == EINVAL

    pc = libswe.swe_part_create
    pc.argtypes = [c_int] * 4 + [c_double] * 4 + [ctypes.POINTER(c_void_p)]
    assert pc(64, 64, 65, 1, 1.0, 1.0, 0.1, 9.8, ctypes.byref(out)) == EINVAL  # more partitions than columns
    assert pc(4096, 4096, 64, 65, 1.0, 1.0, 0.1, 9.8, ctypes.byref(out)) == EINVAL  # > 4096 partitions
    assert pc(64, 64, 2, 2, 1.0, 1.0, 0.0, 9.8, ctypes.byref(out)) == EINVAL
    assert out.value is None

    sd = libswe.swe_selftest_div
    sd.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]
    assert sd(fake, fake, fake, 16, 5, None) == EINVAL      # no such mode
    assert sd(fake, fake, fake, 15, 2, None) == EINVAL      # pairs need an even count
    assert sd(fake, fake, fake, -1, 0, None) == EINVAL
    assert sd(None, fake, fake, 16, 0, None) == EINVAL
    assert sd(fake, fake, fake, 0, 3, None) == 0            # nothing to do

    pr = libswe.swe_probe_rate
    pr.argtypes = [c_int, ctypes.POINTER(c_double)]
    rate = c_double(0.0)
    assert pr(3, ctypes.byref(rate)) == EINVAL              # no such kind
    assert pr(0, None) == EINVAL

    rk = libswe.swe_part_create_rank
    rk.argtypes = [c_int, c_int, c_int] + [c_double] * 4 + [ctypes.POINTER(c_void_p)]
    assert rk(64, 64, 16, 1.0, 1.0, 0.1, 9.8, ctypes.byref(out)) == EINVAL  # walls outside 0..15
    assert rk(64, 64, -1, 1.0, 1.0, 0.1, 9.8, ctypes.byref(out)) == EINVAL
    assert rk(64, 64, 15, 1.0, 1.0, 0.1, 9.8, None) == EINVAL
    assert out.value is None
    pe = libswe.swe_part_edges
    pe.argtypes = [c_void_p, c_void_p, c_void_p]
    assert pe(None, fake, None) == EINVAL
    pg = libswe.swe_part_set_ghosts
    pg.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    assert pg(None, fake, 15, None) == EINVAL

    sw = libswe.swe_selftest_wait
    sw.argtypes = [c_int, c_double, c_void_p]
    assert sw(2, 1.0, None) == EINVAL
    assert sw(0, 0.0, None) == EINVAL
    assert sw(1, 6000.0, None) == EINVAL

    ds = libswe.swe_downsample
    ds.argtypes = [c_int, c_void_p, c_ll, c_ll, c_ll, c_void_p, c_ll, c_ll, c_ll, c_int, c_int, c_int, c_void_p]
    assert ds(5, fake, 0, 0, 1024, fake, 0, 0, 256, 256, 256, 1, None) == EINVAL   # factor above 4
    assert ds(4, fake, 0, 0, 1000, fake, 0, 0, 256, 256, 256, 1, None) == EINVAL   # fine rows too short
    rs = libswe.swe_resample
    rs.argtypes = [c_void_p, c_ll, c_ll, c_ll, c_int, c_int, c_void_p, c_ll, c_ll, c_ll, c_int, c_int, c_int, c_void_p]
    assert rs(fake, 0, 0, 256, 256, 256, fake, 0, 0, 512, 512, 512, 1, None) == EINVAL  # upsampling

    run = libswe.swe_run
    run.argtypes = [c_void_p, c_int, c_double, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                    ctypes.POINTER(c_void_p), c_void_p]
    d = c_double()
    assert run(None, 2, 0.2, ctypes.byref(d), None, None, None) == EINVAL   # no context
    assert run(fake, -1, 0.2, ctypes.byref(d), None, None, None) == EINVAL  # negative step count
    assert run(fake, 2, 0.0, ctypes.byref(d), None, None, None) == EINVAL   # CFL number not positive
