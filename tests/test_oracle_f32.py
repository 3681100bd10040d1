"""Pins of the oracle's binary32 step (the paper's precision, Sec. 3.1 `real`
and Sec. 4.2 `float`): within binary32 rounding of the FP64 oracle (itself
pinned in test_oracle_pins.py), and bitwise on the invariants that hold in
any IEEE precision (lake at rest, mirror symmetry, the ghost rule)."""
import math

import numpy as np
import pytest

import oracle
import swe_inputs as si

G = 9.80
ULP = 2.0 ** -24  # binary32 unit roundoff


def _rel(a, b):
    hmax = float(np.abs(b[0]).max())
    floor = hmax * math.sqrt(G * hmax)
    return [float(np.abs(np.asarray(a[k], np.float64) - b[k]).max()) /
            (hmax if k == 0 else max(floor, float(np.abs(b[k]).max()))) for k in range(3)]


@pytest.mark.parametrize("seed,nx,ny", [(1, 40, 30), (2, 64, 17), (5, 9, 50), (8, 1, 12)])
def test_binary32_step_is_the_fp64_step_to_rounding(seed, nx, ny):
    """Each output is a short chain of roundings of O(1) terms: one step
    stays within a few units of binary32 roundoff of the FP64 step on the
    same (binary32) inputs, and 30 steps within 30 times that.  A dropped or
    mis-signed term, a swapped index or a wrong coefficient would differ by
    thousands of units."""
    s = si.smooth_flow_state(seed, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.8, 1.1, G, 0.3)
    for n, bound in ((1, 4 * ULP), (30, 30 * ULP)):
        a = oracle.run_f32(s.h, s.hu, s.hv, 0.8, 1.1, dt, G, n)
        b = oracle.run(s.h, s.hu, s.hv, 0.8, 1.1, dt, G, n)
        assert max(_rel(a, b)) <= bound, (n, _rel(a, b))


def test_binary32_step_alone_matches_run():
    s = si.smooth_flow_state(4, 23, 19).rounded_to(np.float32)
    P = [np.zeros((21, 25), np.float32) for _ in range(3)]
    for p, a in zip(P, (s.h, s.hu, s.hv)):
        p[1:-1, 1:-1] = a
    oracle.fill_halo_f32(*P)
    out = oracle.step_padded_f32(*P, 0.8, 1.1, 0.02, G)
    ref = oracle.run_f32(s.h, s.hu, s.hv, 0.8, 1.1, 0.02, G, 1)
    for k in range(3):
        assert np.array_equal(out[k][1:-1, 1:-1], ref[k])


def test_binary32_ghost_rule_equals_fp64_ghost_rule():
    rng = np.random.default_rng(0)
    for walls in (1, 2, 4, 8, 15):
        A = [rng.standard_normal((9, 12)).astype(np.float32) for _ in range(3)]
        B = [a.astype(np.float64) for a in A]
        oracle.fill_halo_f32(*A, walls=walls)
        oracle.fill_halo(*B, walls=walls)
        for a, b in zip(A, B):
            assert np.array_equal(a.astype(np.float64), b, equal_nan=True)


def test_binary32_lake_at_rest_is_bitwise_steady():
    h = np.full((23, 37), 1.7, np.float32)
    z = np.zeros_like(h)
    out = oracle.run_f32(h, z, z, 0.7, 1.1, 0.03, G, 500)
    assert np.array_equal(out[0], h) and not out[1].any() and not out[2].any()


def test_binary32_mirror_symmetry_is_bitwise():
    s = si.single_bump_state(0, centred=True).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
    h, hu, hv = oracle.run_f32(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 60)
    assert np.abs(hu).max() > 1e-3
    assert np.array_equal(h, h[:, ::-1]) and np.array_equal(hu, -hu[:, ::-1]) and np.array_equal(hv, hv[:, ::-1])
    assert np.array_equal(h, h[::-1, :]) and np.array_equal(hu, hu[::-1, :]) and np.array_equal(hv, -hv[::-1, :])


def _numpy_binary32_step(h, hu, hv, dx, dy, dt, g):
    """One step restated with numpy float32 arrays (each elementwise numpy
    operation is one IEEE binary32 operation; Python scalars are rounded to
    binary32 where they meet an array): the statements of Sec. 3.1 with the
    reflective ghost rule, written independently of the C oracle."""
    f = np.float32
    P = []
    for a in (h, hu, hv):
        p = np.zeros((a.shape[0] + 2, a.shape[1] + 2), f)
        p[1:-1, 1:-1] = a
        P.append(p)
    H, U, V = P
    for F, sx, sy in ((H, 1, 1), (U, -1, 1), (V, 1, -1)):
        F[1:-1, 0], F[1:-1, -1] = sx * F[1:-1, 1], sx * F[1:-1, -2]
        F[0, 1:-1], F[-1, 1:-1] = sy * F[1, 1:-1], sy * F[-2, 1:-1]
    hx, hy, lx, ly = f(0.5 * dt / dx), f(0.5 * dt / dy), f(dt / dx), f(dt / dy)
    g = f(g)
    fxu = lambda H, U: U * U / H + f(0.5) * g * H * H  # noqa: E731
    fuv = lambda H, U, V: U * V / H  # noqa: E731
    fyv = lambda H, V: V * V / H + f(0.5) * g * H * H  # noqa: E731
    Hl, Hr, Ul, Ur, Vl, Vr = H[1:-1, :-1], H[1:-1, 1:], U[1:-1, :-1], U[1:-1, 1:], V[1:-1, :-1], V[1:-1, 1:]
    Hx = f(0.5) * (Hl + Hr) + hx * (Ul - Ur)
    Ux = f(0.5) * (Ul + Ur) + hx * (fxu(Hl, Ul) - fxu(Hr, Ur))
    Vx = f(0.5) * (Vl + Vr) + hx * (fuv(Hl, Ul, Vl) - fuv(Hr, Ur, Vr))
    Hd, Hu, Ud, Uu, Vd, Vu = H[:-1, 1:-1], H[1:, 1:-1], U[:-1, 1:-1], U[1:, 1:-1], V[:-1, 1:-1], V[1:, 1:-1]
    Hy = f(0.5) * (Hd + Hu) + hy * (Vd - Vu)
    Uy = f(0.5) * (Ud + Uu) + hy * (fuv(Hd, Ud, Vd) - fuv(Hu, Uu, Vu))
    Vy = f(0.5) * (Vd + Vu) + hy * (fyv(Hd, Vd) - fyv(Hu, Vu))
    a, b = fxu(Hx, Ux), fuv(Hx, Ux, Vx)
    c, d = fuv(Hy, Uy, Vy), fyv(Hy, Vy)
    nh = H[1:-1, 1:-1] + lx * (Ux[:, :-1] - Ux[:, 1:]) + ly * (Vy[:-1] - Vy[1:])
    nu = U[1:-1, 1:-1] + lx * (a[:, :-1] - a[:, 1:]) + ly * (c[:-1] - c[1:])
    nv = V[1:-1, 1:-1] + lx * (b[:, :-1] - b[:, 1:]) + ly * (d[:-1] - d[1:])
    return nh, nu, nv


@pytest.mark.parametrize("seed,nx,ny", [(1, 40, 30), (3, 7, 5), (6, 1, 9)])
def test_binary32_step_is_a_numpy_restatement_bit_for_bit(seed, nx, ny):
    s = si.smooth_flow_state(seed, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.8, 1.1, G, 0.3)
    ref = _numpy_binary32_step(*(np.asarray(a, np.float32) for a in (s.h, s.hu, s.hv)), 0.8, 1.1, dt, G)
    got = oracle.run_f32(s.h, s.hu, s.hv, 0.8, 1.1, dt, G, 1)
    for k in range(3):
        assert ref[k].dtype == np.float32
        assert np.array_equal(got[k], ref[k]), k


def test_binary32_window_run_equals_full_run_bitwise():
    nx, ny, n = 40, 30, 7
    bumps = si.multi_bumps(9, 1, nx, ny, 3, sigma_range=(2.0, 5.0))

    def ic(w):
        h = si.bumps_h(nx, ny, 1.0, bumps, w).astype(np.float32)
        return h, np.float32(0.1) * h, np.float32(-0.05) * h

    full = oracle.run_f32(*ic((1, nx, 1, ny)), 1.0, 1.0, 0.05, G, n)
    for window in [(1, 5, 1, 4), (20, 26, 9, 15), (33, 40, 25, 30)]:
        win = oracle.run_window(ic, nx, ny, window, 1.0, 1.0, 0.05, G, n, binary32=True)
        i0, i1, j0, j1 = window
        for k in range(3):
            assert np.array_equal(win[k], full[k][j0 - 1:j1, i0 - 1:i1])


@pytest.mark.parametrize("mistake", ["step1_sign", "drop_pressure", "swap_flux", "ghost_sign"])
def test_per_step_ulp_units_separate_rounding_from_mistakes(mistake):
    """The unit of the GPU-vs-binary32 test (tests/test_gpu_f32_ulp.py): the
    FP64 step differs from the binary32 oracle's step by a few units, while
    each planted mistake (in a numpy copy of the FP64 step) differs by far
    more than the 16 units per step that test allows."""
    from test_gpu_f32_ulp import PER_STEP, _units
    from test_oracle_pins import _planted_step
    s = si.smooth_flow_state(3, 40, 30).rounded_to(np.float32)
    dx, dy = 0.8, 1.1
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3)
    units = _units(s, dx, dy, dt)
    b32 = oracle.run_f32(s.h, s.hu, s.hv, dx, dy, dt, G, 1)
    good = oracle.run(s.h, s.hu, s.hv, dx, dy, dt, G, 1)
    bad = _planted_step(mistake)(s.h, s.hu, s.hv, dx, dy, dt, G)
    r_good = max(float(np.abs(good[k] - b32[k]).max()) / units[k] for k in range(3))
    r_bad = max(float(np.abs(bad[k] - b32[k]).max()) / units[k] for k in range(3))
    assert r_good <= 4.0, r_good
    assert r_bad >= 100 * PER_STEP, (mistake, r_bad)
