"""Helpers shared by the parity tests: run the GPU library and the oracle on
the same seeded inputs and compare them field by field.

Relative error of a field (the reading stated in the design doc): max|gpu - ref|
divided by max|ref|; for the momenta hu, hv the denominator is floored at
1e-3 * max(h) * sqrt(g * max(h)), since momenta can be identically zero.

On grids one or a few cells wide the wall-normal momentum stays at the size
of rounding while the pressure flux g h^2 / 2 it is computed from is O(1);
there an FP32 evaluation of the oracle's own formula (numpy, float32) is
already 3.3e-5 off with that floor, so those tests use a floor of 1e-2.
"""
from __future__ import annotations

import math

import numpy as np

G = 9.80
TOL_F64 = 1e-12
TOL_F32 = 2e-5


def rel_errors(gpu, ref, g=G, floor_frac=1e-3):
    hmax = float(np.max(np.abs(ref[0])))
    floor = floor_frac * hmax * math.sqrt(g * hmax)
    out = []
    for k in range(3):
        den = float(np.max(np.abs(ref[k])))
        if k > 0:
            den = max(den, floor)
        out.append(float(np.max(np.abs(np.asarray(gpu[k], np.float64) - ref[k]))) / den)
    return out


def run_gpu(state, dx, dy, dt, g, n_steps, dtype="f32", kernel=0):
    """Upload ``state`` (swe_inputs.State), take n_steps, download."""
    from paper_1107_2157_gb300 import Grid
    npd = np.float32 if dtype == "f32" else np.float64
    with Grid(state.nx, state.ny, dx, dy, dt, g, dtype=dtype, kernel=kernel) as grid:
        grid.set_state(*(np.ascontiguousarray(a, dtype=npd) for a in (state.h, state.hu, state.hv)))
        grid.step(n_steps)
        out = grid.get_state()
        assert grid.check() == 0
        return out
