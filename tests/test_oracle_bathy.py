"""Pins of the oracle's open sides and bed-slope source (swe_oracle_bathy.c;
variants the paper leaves open, Sec. 2.3 and Sec. 3), against what the
equations fix: a flat bed reduces to the flat-bottom step, a lake at rest
stays at rest (bitwise where the arithmetic is exact, to rounding in
general, while a plausible non-balanced source does not), mass is conserved,
the scheme stays second order over a bed, a uniform flow passes open sides
unchanged and a pulse leaves through them; and a numpy restatement of the
source step equals the C oracle bit for bit."""
import math

import numpy as np
import pytest

import oracle
import swe_inputs as si

G = 9.80


def _bed(nx, ny, seed, amp=0.3):
    bumps = si.multi_bumps(seed, 7, nx, ny, 3, sigma_range=(3.0, 6.0))
    return si.bumps_h(nx, ny, 0.0, bumps) * amp / 0.5


def test_flat_bed_is_the_flat_bottom_step():
    s = si.smooth_flow_state(3, 30, 20)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 40)
    for level in (0.0, 0.37):
        got = oracle.run_bc(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 40, bed=np.full_like(s.h, level))
        for k in range(3):
            assert np.array_equal(got[k], ref[k]), (level, k)


def test_dyadic_lake_at_rest_is_bitwise_steady():
    """Surface 2, bed a multiple of 1/64 in [0, 0.5], g = 8: every operation
    of the step is exact, so the balance of the pressure flux and the source
    holds bit for bit."""
    rng = np.random.default_rng(1)
    b = rng.integers(0, 33, size=(17, 23)) / 64.0
    h = 2.0 - b
    z = np.zeros_like(h)
    out = oracle.run_bc(h, z, z, 1.0, 1.0, 1.0 / 16, 8.0, 300, bed=b)
    assert np.array_equal(out[0], h) and not out[1].any() and not out[2].any()


def _numpy_bathy_step(H, U, V, B, dx, dy, dt, g, mistake=None):
    """One source step restated in numpy on padded arrays with filled ghosts,
    optionally with a planted mistake."""
    hx, hy, lx, ly = 0.5 * dt / dx, 0.5 * dt / dy, dt / dx, dt / dy
    fxu = lambda H, U: U * U / H + 0.5 * g * H * H  # noqa: E731
    fuv = lambda H, U, V: U * V / H  # noqa: E731
    fyv = lambda H, V: V * V / H + 0.5 * g * H * H  # noqa: E731
    sl = lambda A: (A[1:-1, :-1], A[1:-1, 1:])  # noqa: E731
    sd = lambda A: (A[:-1, 1:-1], A[1:, 1:-1])  # noqa: E731
    (Hl, Hr), (Ul, Ur), (Vl, Vr), (Bl, Br) = sl(H), sl(U), sl(V), sl(B)
    s1 = 0.0 if mistake == "no_step1_source" else 1.0
    Hx = 0.5 * (Hl + Hr) + hx * (Ul - Ur)
    Ux = 0.5 * (Ul + Ur) + hx * (fxu(Hl, Ul) - fxu(Hr, Ur)) + s1 * hx * (g * (0.5 * (Hl + Hr)) * (Bl - Br))
    Vx = 0.5 * (Vl + Vr) + hx * (fuv(Hl, Ul, Vl) - fuv(Hr, Ur, Vr))
    (Hd, Hu), (Ud, Uu), (Vd, Vu), (Bd, Bu) = sd(H), sd(U), sd(V), sd(B)
    Hy = 0.5 * (Hd + Hu) + hy * (Vd - Vu)
    Uy = 0.5 * (Ud + Uu) + hy * (fuv(Hd, Ud, Vd) - fuv(Hu, Uu, Vu))
    Vy = 0.5 * (Vd + Vu) + hy * (fyv(Hd, Vd) - fyv(Hu, Vu)) + s1 * hy * (g * (0.5 * (Hd + Hu)) * (Bd - Bu))
    Bx = 0.5 * (B[1:-1, :-1] + B[1:-1, 1:])
    By = 0.5 * (B[:-1, 1:-1] + B[1:, 1:-1])
    if mistake == "cell_depth":       # source with the cell's own depth instead of the face average
        hxs = H[1:-1, 1:-1]
        hys = H[1:-1, 1:-1]
    else:
        hxs = 0.5 * (Hx[:, :-1] + Hx[:, 1:])
        hys = 0.5 * (Hy[:-1] + Hy[1:])
    sgn = -1.0 if mistake == "source_sign" else 1.0
    a, b, c, d = fxu(Hx, Ux), fuv(Hx, Ux, Vx), fuv(Hy, Uy, Vy), fyv(Hy, Vy)
    nh = H[1:-1, 1:-1] + lx * (Ux[:, :-1] - Ux[:, 1:]) + ly * (Vy[:-1] - Vy[1:])
    nu = U[1:-1, 1:-1] + lx * (a[:, :-1] - a[:, 1:]) + ly * (c[:-1] - c[1:]) \
        + sgn * lx * (g * hxs * (Bx[:, :-1] - Bx[:, 1:]))
    nv = V[1:-1, 1:-1] + lx * (b[:, :-1] - b[:, 1:]) + ly * (d[:-1] - d[1:]) \
        + sgn * ly * (g * hys * (By[:-1] - By[1:]))
    return nh, nu, nv


def test_source_step_is_a_numpy_restatement_bit_for_bit():
    s = si.smooth_flow_state(5, 26, 19)
    b = _bed(26, 19, 5)
    H, U, V = oracle.pad(s.h + 0.5), oracle.pad(s.hu), oracle.pad(s.hv)
    oracle.fill_halo(H, U, V)
    B = oracle.pad_bed(b)
    got = oracle.step_padded_bathy(H, U, V, B, 0.8, 1.1, 0.03, G)
    ref = _numpy_bathy_step(H, U, V, B, 0.8, 1.1, 0.03, G)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k]), k


@pytest.mark.parametrize("mistake", [None, "no_step1_source", "cell_depth", "source_sign"])
def test_lake_at_rest_over_a_bed_is_steady_to_rounding(mistake):
    """g = 9.8 and a smooth bed: the balanced source keeps the lake at rest to
    rounding (the momenta stay below 1e-12 of the wave momentum); each
    planted mistake stirs currents many orders larger."""
    nx, ny = 40, 30
    b = _bed(nx, ny, 2)
    h = 1.5 - b
    z = np.zeros_like(h)
    dt = 0.3 / math.sqrt(G * 1.5)
    if mistake is None:
        out = oracle.run_bc(h, z, z, 1.0, 1.0, dt, G, 200, bed=b)
    else:
        H, U, V = oracle.pad(h), oracle.pad(z), oracle.pad(z)
        B = oracle.pad_bed(b)
        for _ in range(200):
            oracle.fill_halo(H, U, V)
            nh, nu, nv = _numpy_bathy_step(H, U, V, B, 1.0, 1.0, dt, G, mistake)
            H[1:-1, 1:-1], U[1:-1, 1:-1], V[1:-1, 1:-1] = nh, nu, nv
        out = (H[1:-1, 1:-1], U[1:-1, 1:-1], V[1:-1, 1:-1])
    wave = 1.5 * math.sqrt(G * 1.5)
    current = max(np.abs(out[1]).max(), np.abs(out[2]).max()) / wave
    if mistake is None:
        assert current <= 1e-12 and np.abs(out[0] - h).max() <= 1e-12
    else:
        assert current >= 1e-6, (mistake, current)


def test_mass_is_conserved_over_a_bed():
    s = si.smooth_flow_state(7, 36, 28)
    b = _bed(36, 28, 7)
    h = s.h + 0.5
    m0 = oracle.mass(h, 0.7, 0.9)
    out = oracle.run_bc(h, s.hu, s.hv, 0.7, 0.9, 0.01, G, 150, bed=b)
    assert abs(oracle.mass(out[0], 0.7, 0.9) - m0) / m0 <= 1e-13
    assert np.abs(out[1]).max() > 1e-3


def test_second_order_over_a_bed():
    def solve(n):
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        X, Y = x[None, :], x[:, None]
        bed = 0.2 * np.exp(-((X - 0.6) ** 2 + (Y - 0.4) ** 2) / (2 * 0.12 ** 2))
        h = 1.0 - bed + 0.05 * np.exp(-((X - 0.4) ** 2 + (Y - 0.55) ** 2) / (2 * 0.08 ** 2))
        z = np.zeros_like(h)
        t_end = 0.06
        dt = 0.25 * dx / math.sqrt(G * 1.1)
        steps = int(math.ceil(t_end / dt))
        return oracle.run_bc(h, z, z, dx, dx, t_end / steps, G, steps, bed=bed)

    def restrict(a):
        return 0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2])

    s = [solve(n) for n in (48, 96, 192)]
    for k in (0, 1, 2):
        e1 = np.sqrt(np.mean((restrict(s[1][k]) - s[0][k]) ** 2))
        e2 = np.sqrt(np.mean((restrict(s[2][k]) - s[1][k]) ** 2))
        assert math.log2(e1 / e2) >= 1.8, (k, math.log2(e1 / e2))


def test_uniform_flow_passes_open_sides_unchanged():
    h = np.full((12, 17), 1.5)
    hu, hv = 0.6 * h, -0.25 * h
    out = oracle.run_bc(h, hu, hv, 1.0, 1.0, 0.05, G, 100, walls=0, open_sides=15)
    for k, ref in enumerate((h, hu, hv)):
        assert np.array_equal(out[k], ref), k
    walled = oracle.run_bc(h, hu, hv, 1.0, 1.0, 0.05, G, 100)
    assert not np.array_equal(walled[1], hu)


def test_a_pulse_leaves_through_open_sides():
    n = 80
    x = np.arange(n) + 0.5
    h = 1.0 + 0.1 * np.exp(-((x[None, :] - 40) ** 2 + (x[:, None] - 40) ** 2) / (2 * 4.0 ** 2))
    z = np.zeros_like(h)
    dt = 0.3 / math.sqrt(G * 1.1)
    steps = int(90 / (math.sqrt(G) * dt))   # the front crosses the half width about twice

    def energy(s):
        eta = s[0] - 1.0
        return float(np.sum(0.5 * G * eta ** 2 + 0.5 * (s[1] ** 2 + s[2] ** 2) / s[0]))

    e0 = energy((h, z, z))
    gone = energy(oracle.run_bc(h, z, z, 1.0, 1.0, dt, G, steps, walls=0, open_sides=15))
    kept = energy(oracle.run_bc(h, z, z, 1.0, 1.0, dt, G, steps))
    assert gone <= 0.03 * e0, gone / e0
    assert kept >= 0.5 * e0, kept / e0


@pytest.mark.parametrize("window", [(1, 6, 1, 5), (18, 25, 9, 14), (35, 40, 26, 30)])
def test_window_run_with_open_sides_and_bed_equals_full_run_bitwise(window):
    nx, ny, n = 40, 30, 6
    bumps = si.multi_bumps(4, 1, nx, ny, 3, sigma_range=(2.0, 5.0))
    mounds = si.multi_bumps(4, 2, nx, ny, 3, amp_range=(0.05, 0.2), sigma_range=(3.0, 6.0))

    def ic(w):
        h = si.bumps_h(nx, ny, 1.2, bumps, w) - si.bumps_h(nx, ny, 0.0, mounds, w)
        return h, 0.1 * h, -0.05 * h

    def bed(w):
        return si.bumps_h(nx, ny, 0.0, mounds, w)

    h, hu, hv = ic((1, nx, 1, ny))
    opens = 1 | 4                                  # left and bottom open, right and top walls
    full = oracle.run_bc(h, hu, hv, 1.0, 1.0, 0.05, G, n, walls=15 & ~opens, open_sides=opens,
                         bed=bed((1, nx, 1, ny)))
    win = oracle.run_window(ic, nx, ny, window, 1.0, 1.0, 0.05, G, n, open_sides=opens, bed=bed)
    i0, i1, j0, j1 = window
    for k in range(3):
        assert np.array_equal(win[k], full[k][j0 - 1:j1, i0 - 1:i1])
