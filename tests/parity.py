"""Helpers shared by the parity tests: run the GPU library and the oracle on
the same seeded inputs and compare them field by field.

Relative error of a field: max|gpu - ref| / max|ref|.  For the momenta hu,
hv the denominator is floored at 1e-3 of the wave momentum h_max sqrt(g
h_max); the floor only binds when a momentum field is (nearly) identically
zero, e.g. a state at rest, where max|ref| alone would divide by zero.

FP32 bar.  A field passes when its relative error is at most TOL_F32 = 2e-5.
Binary32 evaluation of the scheme itself -- every operation one IEEE binary32
operation in the oracle's order (``oracle.run_f32``, the paper's precision)
-- misses that bar on some workloads: its depth is stored with a relative
rounding of 2^-24 each step, and the pressure gradient g h dh turns that
into momentum errors that grow with the number of steps.  Where the GPU
misses 2e-5, ``f32_bar`` therefore runs the binary32 oracle on the same
inputs and accepts the field only if the GPU's error is within
B32_RATIO = 2 times the binary32 oracle's own error against the FP64 oracle:
the miss is then a property of binary32 arithmetic, not of the kernels.
``f32_bar`` returns both errors so that the tests state which fields pass
the bar outright.
"""
from __future__ import annotations

import math

import numpy as np

G = 9.80
TOL_F64 = 1e-12
TOL_F32 = 2e-5
MOMENTUM_FLOOR = 1e-3
B32_RATIO = 2.0


def scales_from_max(maxabs, g=G):
    """Per-field denominators from the fields' max|.|: the momenta floored at
    MOMENTUM_FLOOR of the wave momentum h_max sqrt(g h_max)."""
    hmax = float(maxabs[0])
    floor = MOMENTUM_FLOOR * hmax * math.sqrt(g * hmax)
    return [max(hmax, 1e-300), max(float(maxabs[1]), floor), max(float(maxabs[2]), floor)]


def scales(ref, g=G):
    """Per-field denominators of ``ref``: max|ref|, momenta floored as above."""
    return scales_from_max([float(np.max(np.abs(np.asarray(a)))) for a in ref], g)


def rel_errors(gpu, ref, g=G):
    """max|gpu - ref| / scale per field (see ``scales``)."""
    den = scales(ref, g)
    return [float(np.max(np.abs(np.asarray(gpu[k], np.float64) - ref[k]))) / den[k] for k in range(3)]


def strict_errors(gpu, ref):
    """max|gpu - ref| / max|ref| per field (no floor)."""
    return [float(np.max(np.abs(np.asarray(gpu[k], np.float64) - ref[k]))) / max(float(np.max(np.abs(ref[k]))), 1e-300)
            for k in range(3)]


def f32_bar(got, ref, b32=None, g=G):
    """The FP32 acceptance rule described above.

    ``got`` and ``ref`` are the GPU's and the FP64 oracle's fields; ``b32`` is
    the binary32 oracle's result on the same inputs, or a callable returning
    it (called only if some field misses TOL_F32).  Returns (ok, e_gpu,
    e_b32): per-field errors of the GPU and of the binary32 oracle against
    the FP64 oracle (e_b32 is None when every field passes outright)."""
    e = rel_errors(got, ref, g)
    if max(e) <= TOL_F32:
        return True, e, None
    if b32 is None:
        return False, e, None
    b = b32() if callable(b32) else b32
    eb = rel_errors(b, ref, g)
    ok = all(e[k] <= max(TOL_F32, B32_RATIO * eb[k]) for k in range(3))
    return ok, e, eb


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


def b32_run(state, dx, dy, dt, g, n_steps):
    """A callable for ``f32_bar``: the binary32 oracle on ``state``."""
    import oracle
    return lambda: oracle.run_f32(state.h, state.hu, state.hv, dx, dy, dt, g, n_steps)
