"""Helpers shared by the parity tests: run the GPU library and the oracle on
the same seeded inputs and compare them field by field.

Relative error of a field (the reading this suite takes of "relative"): max|gpu - ref|
divided by the field's scale -- max|ref| for h; for the momenta hu, hv the
larger of max|ref| and the wave momentum h_max * sqrt(g * h_max).  Momenta
can be identically zero (a state at rest) and, in FP32, their rounding
error is set by the rounding of the stored depth through the pressure
gradient, i.e. it scales with h_max * sqrt(g h_max), not with the (possibly
tiny) momentum of the moment.  ``strict_errors`` also reports the ratio to
max|ref| alone.
"""
from __future__ import annotations

import math

import numpy as np

G = 9.80
TOL_F64 = 1e-12
TOL_F32 = 2e-5


def rel_errors(gpu, ref, g=G, floor_frac=1.0):
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


def strict_errors(gpu, ref):
    """max|gpu - ref| / max|ref| per field (no floor)."""
    return [float(np.max(np.abs(np.asarray(gpu[k], np.float64) - ref[k]))) / max(float(np.max(np.abs(ref[k]))), 1e-300)
            for k in range(3)]
