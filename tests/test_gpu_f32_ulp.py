"""The FP32 hand kernels against the binary32 oracle, with a bound in units
of FP32 rounding per step.

The binary32 oracle (``oracle.run_f32``) evaluates the scheme with one IEEE
binary32 operation per operation of the FP64 oracle, in its order.  The GPU
kernels compute the same formulas in FP32 but contract products into FMAs and
form quotients as a product with the approximate reciprocal (rcp.approx, at
most one ulp), so each of their operations may differ from the oracle's by
about one ulp of its result.  Per step and cell, those differences enter:

  * the depth through the update h - (dt/dx)(F.a difference) - ...: at most a
    few ulps of h plus (dt/dx) times a few ulps of the momentum;
  * a momentum through the flux differences, whose terms have the size of
    f = g h^2 / 2 + m^2 / h: a few ulps of m plus (dt/dx) times a few ulps
    of f per face.

So the per-step unit of field k is eps_h = ulp(h_max) + lam ulp(m_max) and
eps_m = ulp(m_max) + lam ulp(f_max), lam = max(dt/dx, dt/dy), ulp(x) the
spacing of binary32 numbers at x; the test allows PER_STEP = 16 units per
step, summed over the steps (the scheme is stable, so a difference made at
one step is not amplified by the later ones beyond that sum).  A plausible
kernel mistake (a dropped term, a wrong sign or index) changes a cell by
order dt/dx times a flux difference, many thousands of these units.
"""
import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import G, run_gpu

pytestmark = pytest.mark.gpu

PER_STEP = 16.0
KERNELS = {"naive": 1, "tiled": 2, "two_step": 3, "packed": 4}


def _ulp(x):
    return float(np.spacing(np.float32(abs(x))))


def _units(s, dx, dy, dt):
    h_max = float(np.abs(s.h).max())
    h_min = float(np.abs(s.h).min())
    m_max = float(max(np.abs(s.hu).max(), np.abs(s.hv).max()))
    f_max = 0.5 * G * h_max * h_max + m_max * m_max / h_min
    lam = max(dt / dx, dt / dy)
    eps_h = _ulp(h_max) + lam * _ulp(m_max)
    eps_m = _ulp(m_max) + lam * _ulp(f_max)
    return [eps_h, eps_m, eps_m]


def _check(got, b32, units, steps):
    ratios = [float(np.abs(got[k].astype(np.float64) - b32[k].astype(np.float64)).max()) / (units[k] * steps)
              for k in range(3)]
    assert max(ratios) <= PER_STEP, ratios
    return ratios


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("nx,ny", [(300, 77), (1025, 40), (129, 33)])
@pytest.mark.parametrize("steps", [1, 10])
def test_hand_kernels_within_ulp_bound_of_binary32_oracle(kernel, nx, ny, steps):
    s = si.smooth_flow_state(nx * 31 + ny, nx, ny).rounded_to(np.float32)
    dx, dy = 0.8, 1.1
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3)
    got = run_gpu(s, dx, dy, dt, G, steps, "f32", KERNELS[kernel])
    b32 = oracle.run_f32(s.h, s.hu, s.hv, dx, dy, dt, G, steps)
    _check(got, b32, _units(s, dx, dy, dt), steps)


def test_batch_variants_within_ulp_bound_of_binary32_oracle():
    """Every persistent-batch variant (tile shape, staging depth, one or two
    steps per pass) on uneven grids, 9 steps (odd: the two-step variants end
    with a one-step pass)."""
    from paper_1107_2157_gb300 import Batch, swe
    sizes = [(300, 77), (65, 190), (129, 33), (1, 1), (517, 9)]
    states = [si.smooth_flow_state(900 + i, nx, ny).rounded_to(np.float32) for i, (nx, ny) in enumerate(sizes)]
    dts = [oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3) for s in states]
    steps = 9
    b32 = [oracle.run_f32(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, steps) for s, dt in zip(states, dts)]
    with Batch(sizes, 1.0, 1.0, dts, G) as b:
        for v in range(b.query(swe.SWE_BQ_VARIANT_COUNT)):
            b.configure(v, 1)
            for i, s in enumerate(states):
                b.set_state(i, *(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
            b.step(steps)
            rc, flags = b.status()
            assert rc == 0 and not flags.any()
            for i, s in enumerate(states):
                _check(b.get_state(i), b32[i], _units(s, 1.0, 1.0, dts[i]), steps)


def test_packed_kernel_against_the_fp64_oracle():
    """The packed-state kernel against the FP64 oracle directly (not only
    against the plane kernel), at a size with interior and wall tiles."""
    from parity import b32_run, f32_bar
    s = si.smooth_flow_state(77, 517, 263).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.8, 1.1, G, 0.3)
    ref = oracle.run(s.h, s.hu, s.hv, 0.8, 1.1, dt, G, 40)
    got = run_gpu(s, 0.8, 1.1, dt, G, 40, "f32", KERNELS["packed"])
    ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s, 0.8, 1.1, dt, G, 40))
    assert ok, (errs, errs_b32)
