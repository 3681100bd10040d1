"""FP32 and FP64 errors against the FP64 oracle on each workload, stated.

Asserts the same bars as the other parity tests and, when SWE_PARITY_REPORT
names a file, writes the measured maximum relative errors there as JSON
(field order h, hu, hv; the relative error is defined in tests/parity.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import G, TOL_F32, TOL_F64, rel_errors, run_gpu, strict_errors

pytestmark = pytest.mark.gpu

REPORT = {}


def _record(key, value):
    REPORT[key] = value
    path = os.environ.get("SWE_PARITY_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_report_128_grid_all_seeds(dtype):
    npd = np.float64 if dtype == "f64" else np.float32
    worst = [0.0, 0.0, 0.0]
    strict = [0.0, 0.0, 0.0]
    for seed in range(10):
        s = si.single_bump_state(seed).rounded_to(npd)
        dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
        ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 100)
        got = run_gpu(s, 1.0, 1.0, dt, G, 100, dtype)
        worst = [max(a, b) for a, b in zip(worst, rel_errors(got, ref))]
        strict = [max(a, b) for a, b in zip(strict, strict_errors(got, ref))]
    _record("128x128_100steps_%s_max_rel_err" % dtype, worst)
    _record("128x128_100steps_%s_max_err_over_max_abs_ref" % dtype, strict)
    assert max(worst) <= (TOL_F64 if dtype == "f64" else TOL_F32)


def test_report_ensemble_instances_500_steps():
    """Eight instances of the 512-grid ensemble (sizes and states of the
    ensemble recipe), 500 FP32 steps in one persistent launch."""
    from paper_1107_2157_gb300 import Batch
    sizes_all = si.ensemble_sizes(seed=2, count=512)
    pick = [0, 37, 101, 202, 303, 404, 480, 511]
    sizes = [sizes_all[i] for i in pick]
    states = [si.ensemble_state(2, i, *sizes_all[i]).rounded_to(np.float32) for i in pick]
    dts = [oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2) for s in states]
    oracle.set_threads(os.cpu_count() or 1)
    worst = [0.0, 0.0, 0.0]
    strict = [0.0, 0.0, 0.0]
    with Batch(sizes, 1.0, 1.0, dts, G) as b:
        for i, s in enumerate(states):
            b.set_state(i, *(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
        b.step(500)
        for i, s in enumerate(states):
            ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dts[i], G, 500)
            got = b.get_state(i)
            worst = [max(a, c) for a, c in zip(worst, rel_errors(got, ref))]
            strict = [max(a, c) for a, c in zip(strict, strict_errors(got, ref))]
    oracle.set_threads(1)
    _record("ensemble_8_instances_500steps_f32_max_rel_err", worst)
    _record("ensemble_8_instances_500steps_f32_max_err_over_max_abs_ref", strict)
    assert max(worst) <= TOL_F32


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_report_8192_grid_windows(dtype):
    """8192x8192 after 100 steps, on the 13 sampled windows of the full-size
    parity test (corners, edges, interior, a tile seam)."""
    import math
    from paper_1107_2157_gb300 import Grid
    from test_gpu_step import _full_windows
    n, steps = 8192, 100
    npd = np.float32 if dtype == "f32" else np.float64
    h0 = si.large_grid_state(seed=1, n=n).h.astype(npd)
    z = np.zeros_like(h0)
    with Grid(n, n, 1.0, 1.0, 0.01, G, dtype=dtype) as grid:
        grid.set_state(h0, z, z)
        dt = grid.cfl_dt(0.2)
        grid.set_dt(dt)
        grid.step(steps)
        got = grid.get_state()

    def ic(w):
        h = si.large_grid_state(seed=1, n=n, window=w).h.astype(npd).astype(np.float64)
        return h, np.zeros_like(h), np.zeros_like(h)

    scale_h = float(h0.max())
    floor = scale_h * math.sqrt(G * scale_h)
    worst = [0.0, 0.0, 0.0]
    for w in _full_windows(n):
        ref = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps)
        i0, i1, j0, j1 = w
        for k in range(3):
            sub = np.asarray(got[k][j0 - 1:j1, i0 - 1:i1], np.float64)
            worst[k] = max(worst[k], float(np.abs(sub - ref[k]).max() / (scale_h if k == 0 else floor)))
    _record("8192x8192_100steps_%s_windows_max_rel_err" % dtype, worst)
    assert max(worst) <= (TOL_F64 if dtype == "f64" else TOL_F32)
