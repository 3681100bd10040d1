"""CPU oracle for the shallow-water Lax-Wendroff path (TEST INFRASTRUCTURE).

Plain, slow, FP64 code that states what the GPU path must compute:
  * the reflective halo fill, the x- and y-face half steps and the full-step
    update of the two-step Lax-Wendroff scheme (Sec. 3, step equations;
    Sec. 3.1, Fortran statements) -- in ``swe_oracle.c``;
  * the FP64 mass and CFL time step (Sec. 3) -- in ``swe_oracle.c``;
  * the same step and wall fill in binary32, the paper's precision -- in
    ``swe_oracle_f32.c``;
  * open (transmissive) sides and the step with a bed-slope source over a
    bottom topography, two variants the paper leaves open -- in
    ``swe_oracle_bathy.c``;
  * the block-average restriction and the corrector network -- in
    ``nn.py`` (numpy, FP64); the learned coarse step built from them and
    the Lax-Wendroff step -- in ``learned.py``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library; the two meet only in the seeded input generators of ``swe_inputs``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Callable, Tuple

import numpy as np

from . import build as _build

WALL_LEFT, WALL_RIGHT, WALL_BOTTOM, WALL_TOP = 1, 2, 4, 8
WALL_ALL = 15

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def lib():
    """Load (building if needed) the oracle's C library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_fill_halo.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.oracle_face_workspace.restype = ctypes.c_size_t
        L.oracle_face_workspace.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [_dp] * 7
        L.oracle_run.restype = ctypes.c_int
        L.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 \
            + [ctypes.c_int, _dp, _dp, _dp]
        L.oracle_mass.restype = ctypes.c_double
        L.oracle_mass.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.oracle_cfl_dt.restype = ctypes.c_double
        L.oracle_cfl_dt.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [_dp] * 3
        L.oracle_fill_halo_f32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, _fp]
        L.oracle_step_f32.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [_fp] * 7
        L.oracle_run_f32.restype = ctypes.c_int
        L.oracle_run_f32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 \
            + [ctypes.c_int, _fp, _fp, _fp]
        L.oracle_fill_open.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.oracle_step_bathy.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [_dp] * 8
        L.oracle_run_bc.restype = ctypes.c_int
        L.oracle_run_bc.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 4 + [ctypes.c_int, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def pad(a: np.ndarray) -> np.ndarray:
    """Interior (ny, nx) -> (ny+2, nx+2) with a zero ghost ring."""
    out = np.zeros((a.shape[0] + 2, a.shape[1] + 2), dtype=np.float64)
    out[1:-1, 1:-1] = a
    return out


def fill_halo(H: np.ndarray, U: np.ndarray, V: np.ndarray, walls: int = WALL_ALL) -> None:
    """Reflective ghost fill in place on padded arrays (see swe_oracle.c)."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    lib().oracle_fill_halo(nx, ny, walls, _ptr(H), _ptr(U), _ptr(V))


def step_padded(H, U, V, dx, dy, dt, g):
    """One step on padded arrays whose ghost ring is already filled.

    Returns the padded outputs (ghost ring zero) and the six face arrays
    (Hx, Ux, Vx of shape (ny, nx+1); Hy, Uy, Vy of shape (ny+1, nx))."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    L = lib()
    oH, oU, oV = (np.zeros_like(H) for _ in range(3))
    faces = np.zeros(L.oracle_face_workspace(nx, ny), dtype=np.float64)
    L.oracle_step(nx, ny, dx, dy, dt, g, _ptr(H), _ptr(U), _ptr(V),
                  _ptr(oH), _ptr(oU), _ptr(oV), _ptr(faces))
    nfx, nfy = (nx + 1) * ny, nx * (ny + 1)
    fx = [faces[k * nfx:(k + 1) * nfx].reshape(ny, nx + 1) for k in range(3)]
    fy = [faces[3 * nfx + k * nfy:3 * nfx + (k + 1) * nfy].reshape(ny + 1, nx) for k in range(3)]
    return (oH, oU, oV), fx, fy


def run_padded(H, U, V, dx, dy, dt, g, n_steps, walls=WALL_ALL):
    """n_steps in place on padded float64 arrays."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    rc = lib().oracle_run(nx, ny, walls, dx, dy, dt, g, int(n_steps), _ptr(H), _ptr(U), _ptr(V))
    if rc != 0:
        raise MemoryError("oracle_run could not allocate its buffers")


def _ptr32(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_fp)


def fill_halo_f32(H: np.ndarray, U: np.ndarray, V: np.ndarray, walls: int = WALL_ALL) -> None:
    """The reflective ghost fill on padded float32 arrays."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    lib().oracle_fill_halo_f32(nx, ny, walls, _ptr32(H), _ptr32(U), _ptr32(V))


def step_padded_f32(H, U, V, dx, dy, dt, g):
    """One binary32 step (the paper's precision) on padded float32 arrays
    whose ghost ring is filled; returns the padded outputs (ghosts zero)."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    L = lib()
    out = [np.zeros_like(H) for _ in range(3)]
    faces = np.zeros(L.oracle_face_workspace(nx, ny), dtype=np.float32)
    L.oracle_step_f32(nx, ny, dx, dy, dt, g, _ptr32(H), _ptr32(U), _ptr32(V),
                      _ptr32(out[0]), _ptr32(out[1]), _ptr32(out[2]), _ptr32(faces))
    return out


def run_f32(h, hu, hv, dx, dy, dt, g, n_steps, walls=WALL_ALL):
    """n_steps in binary32 with reflective walls on interior arrays (values
    rounded to float32 first); returns float32 interiors."""
    P = []
    for a in (h, hu, hv):
        p = np.zeros((a.shape[0] + 2, a.shape[1] + 2), np.float32)
        p[1:-1, 1:-1] = np.asarray(a, np.float32)
        P.append(p)
    ny, nx = P[0].shape[0] - 2, P[0].shape[1] - 2
    if lib().oracle_run_f32(nx, ny, walls, dx, dy, dt, g, int(n_steps), *(_ptr32(p) for p in P)) != 0:
        raise MemoryError("oracle_run_f32 could not allocate its buffers")
    return tuple(p[1:-1, 1:-1].copy() for p in P)


def fill_open(H: np.ndarray, U: np.ndarray, V: np.ndarray, sides: int) -> None:
    """Open (zero-gradient) ghost fill of the given sides on padded arrays."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    lib().oracle_fill_open(nx, ny, sides, _ptr(H), _ptr(U), _ptr(V))


def pad_bed(b: np.ndarray) -> np.ndarray:
    """Interior bed elevation (ny, nx) -> padded, ghosts copying the edge
    cells (the rule for walls and open sides alike), corners NaN (unread)."""
    B = np.pad(np.asarray(b, np.float64), 1, mode="edge")
    B[[0, 0, -1, -1], [0, -1, 0, -1]] = np.nan
    return B


def step_padded_bathy(H, U, V, B, dx, dy, dt, g):
    """One step with the bed-slope source on padded arrays (ghosts filled)."""
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    L = lib()
    out = [np.zeros_like(H) for _ in range(3)]
    faces = np.zeros(L.oracle_face_workspace(nx, ny), dtype=np.float64)
    L.oracle_step_bathy(nx, ny, dx, dy, dt, g, _ptr(H), _ptr(U), _ptr(V), _ptr(B),
                        _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(faces))
    return out


def run_bc(h, hu, hv, dx, dy, dt, g, n_steps, walls=WALL_ALL, open_sides=0, bed=None):
    """n_steps on interior arrays with reflective ``walls`` sides, open
    ``open_sides`` (bitmasks left 1, right 2, bottom 4, top 8) and, if
    ``bed`` (ny, nx) is given, the bed-slope source; returns interiors."""
    H, U, V = pad(np.asarray(h, np.float64)), pad(np.asarray(hu, np.float64)), pad(np.asarray(hv, np.float64))
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    B = pad_bed(bed) if bed is not None else None
    rc = lib().oracle_run_bc(nx, ny, walls, open_sides, dx, dy, dt, g, int(n_steps), _ptr(H), _ptr(U), _ptr(V),
                             _ptr(B) if B is not None else None)
    if rc != 0:
        raise MemoryError("oracle_run_bc could not allocate its buffers")
    return H[1:-1, 1:-1].copy(), U[1:-1, 1:-1].copy(), V[1:-1, 1:-1].copy()


def run(h, hu, hv, dx, dy, dt, g, n_steps):
    """n_steps with reflective walls on interior arrays; returns interiors."""
    H, U, V = pad(np.asarray(h, np.float64)), pad(np.asarray(hu, np.float64)), pad(np.asarray(hv, np.float64))
    run_padded(H, U, V, dx, dy, dt, g, n_steps)
    return H[1:-1, 1:-1].copy(), U[1:-1, 1:-1].copy(), V[1:-1, 1:-1].copy()


def mass(h, dx, dy) -> float:
    """FP64 mass sum(h) dx dy over an interior array."""
    H = pad(np.asarray(h, np.float64))
    return float(lib().oracle_mass(H.shape[1] - 2, H.shape[0] - 2, dx, dy, _ptr(H)))


def cfl_dt(h, hu, hv, dx, dy, g, cfl) -> float:
    """FP64 CFL time step over interior arrays."""
    H, U, V = (pad(np.asarray(a, np.float64)) for a in (h, hu, hv))
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    return float(lib().oracle_cfl_dt(nx, ny, dx, dy, g, cfl, _ptr(H), _ptr(U), _ptr(V)))


def run_window(ic: Callable[[Tuple[int, int, int, int]], Tuple[np.ndarray, np.ndarray, np.ndarray]],
               nx: int, ny: int, window: Tuple[int, int, int, int],
               dx, dy, dt, g, n_steps, binary32: bool = False, open_sides: int = 0,
               bed: Callable[[Tuple[int, int, int, int]], np.ndarray] | None = None):
    """Exact values on a window of a large grid after n_steps.

    The scheme reads only the four edge neighbours of a cell, so after n
    steps a cell depends only on cells at most n away (domain of dependence).
    ``ic(w)`` evaluates the initial interior state on the 1-based inclusive
    index rectangle w = (i0, i1, j0, j1).  The window is grown by n cells per
    side (clipped at the walls), its outer ring holds the true neighbour
    values on sides that are not walls, and the ordinary step runs on it with
    reflective fill on the wall sides only.  Cells inside ``window`` are then
    exactly those of the full-grid run (checked bitwise in the tests).
    ``binary32`` runs the binary32 step instead of the FP64 one.  Sides of
    the grid named in ``open_sides`` are open instead of walls, and ``bed``
    (evaluated like ``ic``) runs the step over that bed (FP64 only; its
    ghosts on the grid boundary copy the edge cells).
    Returns (h, hu, hv) on the window, shape (j1-j0+1, i1-i0+1).
    """
    i0, i1, j0, j1 = window
    n = int(n_steps)
    a, b = max(1, i0 - n + 1), min(nx, i1 + n - 1)
    c, d = max(1, j0 - n + 1), min(ny, j1 + n - 1)
    edges = 0
    edges |= WALL_LEFT if a == 1 else 0
    edges |= WALL_RIGHT if b == nx else 0
    edges |= WALL_BOTTOM if c == 1 else 0
    edges |= WALL_TOP if d == ny else 0
    walls, opens = edges & ~open_sides, edges & open_sides
    fields = ic((a - 1, b + 1, c - 1, d + 1))
    if bed is not None or opens:
        assert not binary32
        H, U, V = (np.ascontiguousarray(f, dtype=np.float64) for f in fields)
        B = None
        if bed is not None:
            B = np.ascontiguousarray(bed((a - 1, b + 1, c - 1, d + 1)), dtype=np.float64)
            if edges & WALL_LEFT:
                B[:, 0] = B[:, 1]
            if edges & WALL_RIGHT:
                B[:, -1] = B[:, -2]
            if edges & WALL_BOTTOM:
                B[0, :] = B[1, :]
            if edges & WALL_TOP:
                B[-1, :] = B[-2, :]
        if lib().oracle_run_bc(b - a + 1, d - c + 1, walls, opens, dx, dy, dt, g, n, _ptr(H), _ptr(U), _ptr(V),
                               _ptr(B) if B is not None else None):
            raise MemoryError("oracle_run_bc could not allocate its buffers")
    elif binary32:
        H, U, V = (np.ascontiguousarray(f, dtype=np.float32) for f in fields)
        if lib().oracle_run_f32(b - a + 1, d - c + 1, walls, dx, dy, dt, g, n, _ptr32(H), _ptr32(U), _ptr32(V)):
            raise MemoryError("oracle_run_f32 could not allocate its buffers")
    else:
        H, U, V = (np.ascontiguousarray(f, dtype=np.float64) for f in fields)
        run_padded(H, U, V, dx, dy, dt, g, n, walls)
    sl = (slice(j0 - c + 1, j1 - c + 2), slice(i0 - a + 1, i1 - a + 2))
    return H[sl].copy(), U[sl].copy(), V[sl].copy()
