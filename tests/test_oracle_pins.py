"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an
invariant of the equations, a closed-form solution, a textbook special case,
or the index sets printed in Sec. 3.1.  A plausible mistake in the oracle
(a dropped flux term, a wrong sign or factor, a swapped index, a wrong ghost
rule) fails at least one of them; ``test_planted_mistakes_are_caught``
demonstrates that on planted copies of the step.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import swe_inputs as si
from closed_forms import (flux_jacobians, lw_amplification, stoker, textbook_lw_1d)

G = 9.80
HERE = os.path.dirname(os.path.abspath(__file__))


def _random_smooth_state(nx, ny, seed, amp_u=0.3):
    rng = si.SplitMix64(seed, 5)
    bumps = si.multi_bumps(seed, 6, nx, ny, 5, sigma_range=(3.0, 8.0))
    h = si.bumps_h(nx, ny, 1.5, bumps)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    a, b = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
    hu = amp_u * h * np.sin(2 * math.pi * a * y)[:, None] * np.sin(math.pi * x)[None, :]
    hv = -amp_u * h * np.sin(math.pi * y)[:, None] * np.cos(2 * math.pi * b * x)[None, :]
    return h, hu, hv


# ---------------------------------------------------------------------------
# The printed index sets of Sec. 3.1
# ---------------------------------------------------------------------------

def region_cpy(a: np.ndarray, halo):
    """Sec. 2.3 region of an array stored as [y, x]: ``halo = [left, right,
    down, up]`` elements are excluded on each side."""
    l, r, d, u = halo
    ny, nx = a.shape
    return a[d:ny - u, l:nx - r]


def test_sec3_1_statements_match_oracle_faces_and_update():
    fx = json.load(open(os.path.join(HERE, "golden", "sec3_1_region_halos.json")))
    nx, ny, dx, dy, dt = 7, 5, 0.9, 1.3, 0.05
    h, hu, hv = _random_smooth_state(nx, ny, 3)
    H, U, V = oracle.pad(h), oracle.pad(hu), oracle.pad(hv)
    oracle.fill_halo(H, U, V)
    (oH, oU, oV), (Hx, Ux, Vx), (Hy, Uy, Vy) = oracle.step_padded(H, U, V, dx, dy, dt, G)

    s1 = fx["step1"]
    Hx_paper = 0.5 * (region_cpy(H, s1["face_lt"]) + region_cpy(H, s1["face_rt"])) \
        + (0.5 * dt / dx) * (region_cpy(U, s1["face_lt"]) - region_cpy(U, s1["face_rt"]))
    assert Hx_paper.shape == Hx.shape == (ny, nx + 1)
    assert np.array_equal(Hx_paper, Hx)
    # the y analogue of the Hx statement, with face_dn / face_up and V
    Hy_paper = 0.5 * (region_cpy(H, s1["face_dn"]) + region_cpy(H, s1["face_up"])) \
        + (0.5 * dt / dy) * (region_cpy(V, s1["face_dn"]) - region_cpy(V, s1["face_up"]))
    assert Hy_paper.shape == Hy.shape == (ny + 1, nx)
    assert np.array_equal(Hy_paper, Hy)

    s2 = fx["step2"]
    pH = region_cpy(H, s2["halo"]) \
        + (dt / dx) * (region_cpy(Ux, s2["face_lt"]) - region_cpy(Ux, s2["face_rt"])) \
        + (dt / dy) * (region_cpy(Vy, s2["face_dn"]) - region_cpy(Vy, s2["face_up"]))
    assert np.array_equal(pH, oH[1:-1, 1:-1])


# ---------------------------------------------------------------------------
# Reflective ghost rule
# ---------------------------------------------------------------------------

def test_halo_fill_rule_and_nan_corners():
    nx, ny = 6, 4
    rng = np.random.default_rng(0)
    H, U, V = (oracle.pad(rng.uniform(1, 2, (ny, nx))) for _ in range(3))
    oracle.fill_halo(H, U, V)
    I = slice(1, -1)
    assert np.array_equal(H[I, 0], H[I, 1]) and np.array_equal(H[I, -1], H[I, -2])
    assert np.array_equal(U[I, 0], -U[I, 1]) and np.array_equal(U[I, -1], -U[I, -2])
    assert np.array_equal(V[I, 0], V[I, 1]) and np.array_equal(V[I, -1], V[I, -2])
    assert np.array_equal(H[0, I], H[1, I]) and np.array_equal(H[-1, I], H[-2, I])
    assert np.array_equal(U[0, I], U[1, I]) and np.array_equal(U[-1, I], U[-2, I])
    assert np.array_equal(V[0, I], -V[1, I]) and np.array_equal(V[-1, I], -V[-2, I])
    for a in (H, U, V):
        assert np.isnan(a[[0, 0, -1, -1], [0, -1, 0, -1]]).all()


def test_corner_ghosts_never_read():
    # fill_halo plants NaN in the corners; 50 steps stay finite.
    h, hu, hv = _random_smooth_state(9, 11, 4)
    out = oracle.run(h, hu, hv, 1.0, 1.0, 0.02, G, 50)
    assert all(np.isfinite(a).all() for a in out)


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------

def test_lake_at_rest_is_bitwise_steady():
    nx, ny = 37, 23
    h = np.full((ny, nx), 1.7)
    z = np.zeros_like(h)
    out = oracle.run(h, z, z, 0.7, 1.1, 0.03, G, 1000)
    assert np.array_equal(out[0], h)
    assert np.array_equal(out[1], z) and np.array_equal(out[2], z)


@pytest.mark.parametrize("seed", [0, 3, 7])
def test_mass_conserved_with_reflective_walls(seed):
    s = si.single_bump_state(seed)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
    m0 = oracle.mass(s.h, 1.0, 1.0)
    h, hu, hv = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 100)
    assert abs(oracle.mass(h, 1.0, 1.0) - m0) / m0 <= 1e-13
    # a state with momentum in both directions, unequal dx, dy
    h, hu, hv = _random_smooth_state(40, 28, seed)
    m0 = oracle.mass(h, 0.5, 0.8)
    h2, _, _ = oracle.run(h, hu, hv, 0.5, 0.8, 0.01, G, 200)
    assert abs(oracle.mass(h2, 0.5, 0.8) - m0) / m0 <= 1e-13


def test_mirror_symmetry_of_centred_bump_is_bitwise():
    s = si.single_bump_state(0, centred=True)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
    h, hu, hv = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 100)
    assert np.abs(hu).max() > 1e-3  # the bump has moved
    # x-mirror: h even, hu odd, hv even
    assert np.array_equal(h, h[:, ::-1])
    assert np.array_equal(hu, -hu[:, ::-1])
    assert np.array_equal(hv, hv[:, ::-1])
    # y-mirror: h even, hu even, hv odd
    assert np.array_equal(h, h[::-1, :])
    assert np.array_equal(hu, hu[::-1, :])
    assert np.array_equal(hv, -hv[::-1, :])


def test_axis_swap_equivalence():
    # (h, hu, hv, dx, dy) and (h^T, hv^T, hu^T, dy, dx) give transposed results.
    # The update adds the x terms before the y terms (Sec. 3.1 order), so the
    # two runs agree to rounding, not bitwise.
    h, hu, hv = _random_smooth_state(30, 22, 11)
    a = oracle.run(h, hu, hv, 0.6, 0.9, 0.012, G, 60)
    b = oracle.run(h.T.copy(), hv.T.copy(), hu.T.copy(), 0.9, 0.6, 0.012, G, 60)
    scale = [np.abs(a[0]).max(), np.abs(a[1]).max(), np.abs(a[2]).max()]
    assert np.abs(a[0] - b[0].T).max() <= 1e-14 * scale[0]
    assert np.abs(a[1] - b[2].T).max() <= 1e-14 * max(scale)
    assert np.abs(a[2] - b[1].T).max() <= 1e-14 * max(scale)


def test_one_dimensional_reduction_matches_textbook_1d_scheme():
    nx, ny = 160, 3
    x = (np.arange(nx) + 0.5) / nx
    h1 = 1.0 + 0.4 * np.exp(-((x - 0.35) / 0.07) ** 2)
    m1 = 0.2 * np.sin(math.pi * x) * h1
    dx, dt = 1.0 / nx, 0.3 / nx / math.sqrt(G * 1.4)
    h = np.tile(h1, (ny, 1))
    hu = np.tile(m1, (ny, 1))
    hv = np.zeros_like(h)
    H, U, V = oracle.run(h, hu, hv, dx, 0.37, dt, G, 150)
    # V stays exactly zero and every row is identical
    assert np.array_equal(V, np.zeros_like(V))
    assert all(np.array_equal(H[0], H[k]) and np.array_equal(U[0], U[k]) for k in range(ny))
    hr, mr = textbook_lw_1d(h1, m1, dx, dt, G, 150)
    assert np.abs(H[0] - hr).max() <= 1e-13
    assert np.abs(U[0] - mr).max() <= 1e-13


# ---------------------------------------------------------------------------
# Linearised (von Neumann) analysis
# ---------------------------------------------------------------------------

def _fourier_mode(nx, ny, tx, ty, qhat, offset=0.0):
    i = np.arange(1, nx + 1, dtype=np.float64)
    j = np.arange(1, ny + 1, dtype=np.float64)
    phase = np.exp(1j * (tx * (i[None, :] - offset) + ty * (j[:, None] - offset)))
    return [qhat[k] * phase for k in range(3)]


@pytest.mark.parametrize("tx,ty", [(0.7, 0.0), (0.0, 1.1), (0.9, 0.45), (2.3, -1.7)])
def test_linearised_step_matches_amplification_matrix_on_moving_state(tx, ty):
    """About a uniform moving state, one step multiplies a small Fourier mode
    by the LW amplification matrix built from the flux Jacobians (all six
    flux terms enter A or B with a non-zero coefficient here)."""
    nx, ny, dx, dy = 48, 40, 1.0, 0.8
    H0, U0, V0 = 1.5, 0.3 * 1.5, -0.2 * 1.5
    dt = 0.45 * min(dx, dy) / (math.sqrt(G * H0) + 0.3)
    eps = 1e-6
    qhat = np.array([1.0, 0.6 - 0.3j, 0.2 + 0.5j])
    mode = _fourier_mode(nx, ny, tx, ty, qhat)
    base = (H0, U0, V0)
    state = [base[k] + eps * mode[k].real for k in range(3)]
    out = oracle.run(*state, dx, dy, dt, G, 1)
    A, B = flux_jacobians(H0, U0, V0, G)
    Gm = lw_amplification(A, B, dt / dx, dt / dy, tx, ty)
    pred_hat = Gm @ qhat
    pred = _fourier_mode(nx, ny, tx, ty, pred_hat)
    inner = (slice(2, -2), slice(2, -2))  # cells not touched by the walls
    for k in range(3):
        got = (out[k] - base[k])[inner] / eps
        want = pred[k].real[inner]
        assert np.abs(got - want).max() <= 2e-4, k


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 2), (3, 2), (7, 5)])
def test_standing_wave_with_reflective_walls_matches_amplification(mx, my):
    """At rest, the mode h ~ cos(tx (i-1/2)) cos(ty (j-1/2)) with tx = pi mx/nx
    is even about both walls (hu odd in x, hv odd in y), so the reflective
    ghosts are its own continuation and every cell, walls included, follows
    the amplification matrix.  This pins the ghost rule."""
    nx, ny, dx, dy = 32, 24, 1.0, 1.0
    H0 = 2.0
    dt = 0.5 * dx / math.sqrt(G * H0)
    eps = 1e-6
    tx, ty = math.pi * mx / nx, math.pi * my / ny
    A, B = flux_jacobians(H0, 0.0, 0.0, G)
    # real standing wave = sum over the four sign combinations of exp modes
    acc = [np.zeros((ny, nx)) for _ in range(3)]
    init = [np.zeros((ny, nx)) for _ in range(3)]
    for sx in (1, -1):
        for sy in (1, -1):
            qhat = np.array([0.25, 0.0, 0.0], dtype=np.complex128)
            m0 = _fourier_mode(nx, ny, sx * tx, sy * ty, qhat, offset=0.5)
            Gm = lw_amplification(A, B, dt / dx, dt / dy, sx * tx, sy * ty)
            m1 = _fourier_mode(nx, ny, sx * tx, sy * ty, Gm @ qhat, offset=0.5)
            for k in range(3):
                init[k] += m0[k].real
                acc[k] += m1[k].real
    state = [H0 + eps * init[0], eps * init[1], eps * init[2]]
    out = oracle.run(*state, dx, dy, dt, G, 1)
    for k, base in enumerate((H0, 0.0, 0.0)):
        got = (out[k] - base) / eps
        assert np.abs(got - acc[k]).max() <= 2e-4, k


# ---------------------------------------------------------------------------
# Nonlinear closed forms and convergence
# ---------------------------------------------------------------------------

def _dam_break_run(nx, g=G, h_l=2.0, h_r=1.0, t_end=0.075, cfl=0.45):
    ny, L = 2, 1.0
    dx = L / nx
    x = (np.arange(nx) + 0.5) * dx
    h = np.tile(np.where(x < 0.5 * L, h_l, h_r), (ny, 1))
    z = np.zeros_like(h)
    dt0 = oracle.cfl_dt(h, z, z, dx, dx, g, cfl)
    n = int(math.ceil(t_end / dt0))
    dt = t_end / n
    H, U, V = oracle.run(h, z, z, dx, dx, dt, g, n)
    he, ue = stoker((x - 0.5 * L) / t_end, h_l, h_r, g)
    return H[0], U[0], he, ue


def test_stoker_dam_break_l1_and_refinement():
    errs = []
    for nx in (256, 512, 1024):
        h, hu, he, ue = _dam_break_run(nx)
        errs.append(np.abs(h - he).sum() / np.abs(he).sum())
    assert errs[-1] <= 0.02, errs
    assert errs[0] > errs[1] > errs[2], errs
    # the momentum profile too (L1 relative to the peak momentum plateau)
    h, hu, he, ue = _dam_break_run(1024)
    me = he * ue
    assert np.abs(hu - me).sum() / np.abs(me).sum() <= 0.05


def test_linear_wave_speed_is_sqrt_gh():
    nx, ny, dx = 2048, 2, 1.0
    x = (np.arange(nx) + 0.5) * dx
    H0, eps, sig = 1.0, 1e-3, 16.0
    h = np.tile(H0 + eps * np.exp(-(x - 1024.0) ** 2 / (2 * sig * sig)), (ny, 1))
    z = np.zeros_like(h)
    c = math.sqrt(G * H0)
    dt = 0.5 * dx / c

    def peak_position(hrow):
        k = 1024 + int(np.argmax(hrow[1024:]))
        y0, y1, y2 = hrow[k - 1], hrow[k], hrow[k + 1]
        return x[k] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * dx

    n1, n2 = 400, 800
    H1, U1, V1 = oracle.run(h, z, z, dx, dx, dt, G, n1)
    H2, _, _ = oracle.run(H1, U1, V1, dx, dx, dt, G, n2 - n1)
    speed = (peak_position(H2[0]) - peak_position(H1[0])) / ((n2 - n1) * dt)
    assert abs(speed / c - 1.0) <= 0.01, speed / c


def test_second_order_self_convergence():
    def solve(n):
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        r2 = (x[None, :] - 0.45) ** 2 + (x[:, None] - 0.55) ** 2
        h = 1.0 + 0.1 * np.exp(-r2 / (2 * 0.08 ** 2))
        z = np.zeros_like(h)
        t_end = 0.06
        dt = 0.25 * dx / math.sqrt(G * 1.1)
        steps = int(math.ceil(t_end / dt))
        return oracle.run(h, z, z, dx, dx, t_end / steps, G, steps)

    def restrict(a):
        return 0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2])

    s = [solve(n) for n in (48, 96, 192)]
    for k in (0, 1):
        e1 = np.sqrt(np.mean((restrict(s[1][k]) - s[0][k]) ** 2))
        e2 = np.sqrt(np.mean((restrict(s[2][k]) - s[1][k]) ** 2))
        order = math.log2(e1 / e2)
        assert order >= 1.8, (k, order)


# ---------------------------------------------------------------------------
# Mass and CFL
# ---------------------------------------------------------------------------

def test_mass_closed_form():
    nx, ny, dx, dy = 13, 9, 0.5, 0.25
    i = np.arange(1, nx + 1)
    j = np.arange(1, ny + 1)
    h = (i[None, :] + 2.0 * j[:, None]).astype(np.float64)
    exact = (ny * nx * (nx + 1) / 2 + 2 * nx * ny * (ny + 1) / 2) * dx * dy
    assert oracle.mass(h, dx, dy) == exact


def test_cfl_closed_form_and_argmin():
    nx, ny = 10, 7
    h = np.full((ny, nx), 2.0)
    hu = 0.5 * h
    hv = -0.25 * h
    dt = oracle.cfl_dt(h, hu, hv, 1.0, 0.5, G, 0.2)
    c = math.sqrt(G * 2.0)
    assert dt == pytest.approx(0.2 * min(1.0 / (c + 0.5), 0.5 / (c + 0.25)), rel=1e-15)
    h[3, 4] = 8.0  # one deep cell sets the step
    dt = oracle.cfl_dt(h, h * 0, h * 0, 1.0, 1.0, G, 0.3)
    assert dt == pytest.approx(0.3 / math.sqrt(G * 8.0), rel=1e-15)


# ---------------------------------------------------------------------------
# Domain-of-dependence window (used for sampled parity on large grids)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("window", [(1, 5, 1, 4), (20, 26, 9, 15), (33, 40, 25, 30), (12, 12, 30, 30)])
def test_window_run_equals_full_run_bitwise(window):
    nx, ny, n = 40, 30, 7
    bumps = si.multi_bumps(9, 1, nx, ny, 3, sigma_range=(2.0, 5.0))

    def ic(w):
        h = si.bumps_h(nx, ny, 1.0, bumps, w)
        return h, 0.1 * h, -0.05 * h

    h, hu, hv = ic((1, nx, 1, ny))
    full = oracle.run(h, hu, hv, 1.0, 1.0, 0.05, G, n)
    win = oracle.run_window(ic, nx, ny, window, 1.0, 1.0, 0.05, G, n)
    i0, i1, j0, j1 = window
    for k in range(3):
        assert np.array_equal(win[k], full[k][j0 - 1:j1, i0 - 1:i1])


# ---------------------------------------------------------------------------
# The pins above catch plausible mistakes
# ---------------------------------------------------------------------------

def _planted_step(mistake):
    """A numpy copy of one oracle step with one planted mistake."""
    def step(h, hu, hv, dx, dy, dt, g):
        H, U, V = oracle.pad(h), oracle.pad(hu), oracle.pad(hv)
        oracle.fill_halo(H, U, V)
        if mistake == "ghost_sign":
            U[1:-1, 0] = U[1:-1, 1]
        hx, lx = 0.5 * dt / dx, dt / dx
        hy, ly = 0.5 * dt / dy, dt / dy
        sgn = -1.0 if mistake == "step1_sign" else 1.0
        Hl, Hr = H[1:-1, :-1], H[1:-1, 1:]
        Ul, Ur = U[1:-1, :-1], U[1:-1, 1:]
        Vl, Vr = V[1:-1, :-1], V[1:-1, 1:]
        f2 = lambda H, U: U * U / H + (0.0 if mistake == "drop_pressure" else 0.5 * g * H * H)
        f3 = (lambda H, U, V: V * V / H) if mistake == "swap_flux" else (lambda H, U, V: U * V / H)
        Hx = 0.5 * (Hl + Hr) + sgn * hx * (Ul - Ur)
        Ux = 0.5 * (Ul + Ur) + sgn * hx * (f2(Hl, Ul) - f2(Hr, Ur))
        Vx = 0.5 * (Vl + Vr) + sgn * hx * (f3(Hl, Ul, Vl) - f3(Hr, Ur, Vr))
        Hd, Hu = H[:-1, 1:-1], H[1:, 1:-1]
        Ud, Uu = U[:-1, 1:-1], U[1:, 1:-1]
        Vd, Vu = V[:-1, 1:-1], V[1:, 1:-1]
        g3 = lambda H, V: V * V / H + 0.5 * g * H * H
        Hy = 0.5 * (Hd + Hu) + hy * (Vd - Vu)
        Uy = 0.5 * (Ud + Uu) + hy * (Ud * Vd / Hd - Uu * Vu / Hu)
        Vy = 0.5 * (Vd + Vu) + hy * (g3(Hd, Vd) - g3(Hu, Vu))
        fxu = f2(Hx, Ux)
        fxv = f3(Hx, Ux, Vx)
        gyu = Uy * Vy / Hy
        gyv = g3(Hy, Vy)
        nh = H[1:-1, 1:-1] + lx * (Ux[:, :-1] - Ux[:, 1:]) + ly * (Vy[:-1] - Vy[1:])
        nu = U[1:-1, 1:-1] + lx * (fxu[:, :-1] - fxu[:, 1:]) + ly * (gyu[:-1] - gyu[1:])
        nv = V[1:-1, 1:-1] + lx * (fxv[:, :-1] - fxv[:, 1:]) + ly * (gyv[:-1] - gyv[1:])
        return nh, nu, nv
    return step


@pytest.mark.parametrize("mistake", [None, "step1_sign", "drop_pressure", "swap_flux", "ghost_sign"])
def test_planted_mistakes_are_caught(mistake):
    """The correct numpy copy passes the linearised pins; each planted
    mistake fails one of them (moving-state mode or wall standing wave)."""
    step = _planted_step(mistake)
    G_ = G
    # moving-state linear pin
    nx, ny, dx, dy = 24, 20, 1.0, 0.8
    H0, U0, V0 = 1.5, 0.45, -0.3
    dt = 0.45 * 0.8 / (math.sqrt(G_ * H0) + 0.3)
    eps, tx, ty = 1e-6, 0.9, 0.45
    qhat = np.array([1.0, 0.6 - 0.3j, 0.2 + 0.5j])
    mode = _fourier_mode(nx, ny, tx, ty, qhat)
    base = (H0, U0, V0)
    out = step(*[base[k] + eps * mode[k].real for k in range(3)], dx, dy, dt, G_)
    A, B = flux_jacobians(H0, U0, V0, G_)
    pred = _fourier_mode(nx, ny, tx, ty, lw_amplification(A, B, dt / dx, dt / dy, tx, ty) @ qhat)
    inner = (slice(2, -2), slice(2, -2))
    err1 = max(np.abs((out[k] - base[k])[inner] / eps - pred[k].real[inner]).max() for k in range(3))
    # wall standing wave with a flow along x near the wall (hu odd about x walls)
    nx, ny = 16, 12
    tx = math.pi * 3 / nx
    i = np.arange(1, nx + 1) - 0.5
    h = 2.0 + eps * np.tile(np.cos(tx * i), (ny, 1))
    hu = eps * np.tile(np.sin(tx * i), (ny, 1))
    dt = 0.5 / math.sqrt(G_ * 2.0)
    out = step(h, hu, np.zeros_like(h), 1.0, 1.0, dt, G_)
    ref = oracle.run(h, hu, np.zeros_like(h), 1.0, 1.0, dt, G_, 1)
    A, B = flux_jacobians(2.0, 0.0, 0.0, G_)
    acc = [np.zeros((ny, nx)) for _ in range(3)]
    for sx in (1, -1):
        qh = np.array([0.5, -0.5j * sx, 0.0])
        m1 = _fourier_mode(nx, ny, sx * tx, 0.0, lw_amplification(A, B, dt, dt, sx * tx, 0.0) @ qh, offset=0.5)
        for k in range(3):
            acc[k] += m1[k].real
    err2 = max(np.abs((out[k] - (2.0 if k == 0 else 0.0)) / eps - acc[k]).max() for k in range(3))
    caught = err1 > 2e-4 or err2 > 2e-4
    if mistake is None:
        assert not caught, (err1, err2)
        # and the numpy copy agrees with the oracle on the wall case
        assert all(np.abs(out[k] - ref[k]).max() <= 1e-14 for k in range(3))
    else:
        assert caught, (mistake, err1, err2)
