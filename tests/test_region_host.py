"""Host side of the region front end (no GPU): the index sets the step's and
the wall fill's region statements take (Sec. 2.3 halo semantics; Sec. 3.1's
face arrays, one face more than cells in their direction), checked against
the sizes the oracle allocates for the same face arrays, and argument
checks that return before any device work."""
import ctypes

import pytest

import oracle


def _lib():
    from paper_1107_2157_gb300 import swe
    return swe


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (10, 7), (64, 8), (129, 33), (4096, 3), (65536, 65536)])
def test_statement_extents(nx, ny):
    ext = _lib().swe_region_shapes(nx, ny)
    assert ext == [(nx + 2, ny + 2),                          # cell fluxes
                   (nx + 1, ny), (nx, ny + 1), (nx, ny),       # x-faces, y-faces, update
                   (1, ny), (1, ny), (nx, 1), (nx, 1)]        # left, right, bottom, top ghosts


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 3), (200, 97)])
def test_face_arrays_match_the_oracle_workspace(nx, ny):
    """The oracle sizes its six face arrays independently (plain C); the
    region statements' face groups, three arrays each, must fill exactly
    that workspace."""
    ext = _lib().swe_region_shapes(nx, ny)
    faces = 3 * ext[1][0] * ext[1][1] + 3 * ext[2][0] * ext[2][1]
    assert faces == oracle.lib().oracle_face_workspace(nx, ny)


def test_shapes_rejects_bad_sizes():
    swe = _lib()
    ext = (ctypes.c_int * 32)()
    n = ctypes.c_int()
    for nx, ny in [(0, 5), (5, 0), (70000, 5), (-1, -1)]:
        assert swe.lib().swe_region_shapes(nx, ny, ext, 16, ctypes.byref(n)) == swe.SWE_EINVAL


def test_create_rejects_bad_arguments_before_device_work():
    swe = _lib()
    h = ctypes.c_void_p()
    f = swe.lib().swe_region_create
    assert f(2, 10, 10, 32, 0, ctypes.byref(h)) == swe.SWE_EINVAL            # dtype
    assert f(swe.SWE_F32, 0, 10, 32, 0, ctypes.byref(h)) == swe.SWE_EINVAL   # nx
    assert f(swe.SWE_F32, 10, 10, 11, 0, ctypes.byref(h)) == swe.SWE_EINVAL  # pitch < nx + 2
    assert f(swe.SWE_F32, 10, 10, 14, 0, ctypes.byref(h)) == swe.SWE_EINVAL  # 56-byte rows
    assert f(swe.SWE_F64, 10, 10, 13, 0, ctypes.byref(h)) == swe.SWE_EINVAL  # 104-byte rows
    assert f(swe.SWE_F32, 10, 10, 32, 6, ctypes.byref(h)) == swe.SWE_EINVAL  # no such variant
    assert f(swe.SWE_F64, 10, 10, 32, 4, ctypes.byref(h)) == swe.SWE_EINVAL
    assert f(swe.SWE_F32, 10, 10, 32, 0, None) == swe.SWE_EINVAL
    null = (ctypes.c_void_p * 3)()
    assert swe.lib().swe_region_step(None, null, null, 1.0, 1.0, 0.1, 9.8, None) == swe.SWE_EINVAL
    assert swe.lib().swe_region_walls(None, null, 15, None) == swe.SWE_EINVAL
