"""GPU parity of the single-grid path (C ABI -> CUDA kernels) against the
FP64 oracle, on the same seeded inputs.

Bars: FP64 within 1e-12 relative per field; FP32 within 2e-5, or, where
binary32 evaluation of the scheme itself misses 2e-5, within twice the
binary32 oracle's own error (``parity.f32_bar``); integer-like facts (lake at
rest, the CFL step) bitwise.
"""

import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import B32_RATIO, G, TOL_F32, TOL_F64, b32_run, f32_bar, rel_errors, run_gpu, scales

pytestmark = pytest.mark.gpu

KERNELS = {"tiled": 2, "naive": 1}


def _oracle(state, dx, dy, dt, n):
    return oracle.run(state.h, state.hu, state.hv, dx, dy, dt, G, n)


@pytest.mark.parametrize("seed", list(range(10)))
def test_128_fp64_100_steps(seed):
    """128x128 bump, FP64, dt from CFL 0.2 at t = 0, 100 steps."""
    s = si.single_bump_state(seed)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
    ref = _oracle(s, 1.0, 1.0, dt, 100)
    got = run_gpu(s, 1.0, 1.0, dt, G, 100, "f64")
    errs = rel_errors(got, ref)
    assert max(errs) <= TOL_F64, errs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_128_fp32_100_steps(seed):
    s = si.single_bump_state(seed)
    s32 = s.rounded_to(np.float32)
    dt = oracle.cfl_dt(s32.h, s32.hu, s32.hv, 1.0, 1.0, G, 0.2)
    ref = _oracle(s32, 1.0, 1.0, dt, 100)
    got = run_gpu(s32, 1.0, 1.0, dt, G, 100, "f32")
    ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s32, 1.0, 1.0, dt, G, 100))
    assert ok, (errs, errs_b32)


@pytest.mark.parametrize("kernel", ["tiled", "naive"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (3, 5), (4, 4), (127, 31), (129, 33),
                                   (130, 66), (200, 97), (257, 129), (64, 200)])
def test_ragged_sizes_with_flow_at_walls(kernel, dtype, nx, ny):
    """Sizes below, at and just past tile multiples, with momentum at every
    wall so the ghost rule is exercised on all four sides."""
    s = si.smooth_flow_state(nx * 1000 + ny, nx, ny)
    dx, dy = 0.8, 1.1
    if dtype == "f32":
        s = s.rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3)
    ref = _oracle(s, dx, dy, dt, 20)
    got = run_gpu(s, dx, dy, dt, G, 20, dtype, KERNELS[kernel])
    if dtype == "f64":
        errs = rel_errors(got, ref)
        assert max(errs) <= TOL_F64, errs
    else:
        ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s, dx, dy, dt, G, 20))
        assert ok, (errs, errs_b32)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_lake_at_rest_bitwise(dtype):
    nx, ny = 300, 170
    s = si.State(np.full((ny, nx), 1.7), np.zeros((ny, nx)), np.zeros((ny, nx)))
    got = run_gpu(s, 0.7, 1.1, 0.03, G, 1000, dtype)
    assert np.array_equal(got[0], s.h.astype(got[0].dtype))
    assert not np.any(got[1]) and not np.any(got[2])


def test_zero_steps_round_trip_is_exact():
    s = si.smooth_flow_state(5, 77, 45)
    for dtype, npd in (("f32", np.float32), ("f64", np.float64)):
        got = run_gpu(s, 1.0, 1.0, 0.01, G, 0, dtype)
        for k, a in enumerate((s.h, s.hu, s.hv)):
            assert np.array_equal(got[k], a.astype(npd))


def test_mirror_symmetry_fp64():
    s = si.single_bump_state(0, centred=True)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.2)
    h, hu, hv = run_gpu(s, 1.0, 1.0, dt, G, 100, "f64")
    scale = np.abs(h).max()
    assert np.abs(h - h[:, ::-1]).max() <= 1e-13 * scale
    assert np.abs(hu + hu[:, ::-1]).max() <= 1e-13 * scale
    assert np.abs(h - h[::-1, :]).max() <= 1e-13 * scale
    assert np.abs(hv + hv[::-1, :]).max() <= 1e-13 * scale


# ---------------------------------------------------------------------------
# FP64 reductions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mass_and_cfl_match_oracle(dtype):
    from paper_1107_2157_gb300 import Grid
    nx, ny, dx, dy = 517, 389, 0.6, 1.3
    s = si.smooth_flow_state(17, nx, ny)
    npd = np.float32 if dtype == "f32" else np.float64
    s = s.rounded_to(npd)
    with Grid(nx, ny, dx, dy, 0.01, G, dtype=dtype) as grid:
        grid.set_state(*(a.astype(npd) for a in (s.h, s.hu, s.hv)))
        m = grid.mass()
        dt = grid.cfl_dt(0.2)
    m_ref = oracle.mass(s.h, dx, dy)
    assert abs(m - m_ref) <= 1e-14 * m_ref
    # the per-cell bounds are correctly rounded FP64 operations on both sides
    assert dt == oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.2)


def test_cfl_rejects_non_positive_depth():
    from paper_1107_2157_gb300 import Grid, SweError
    s = si.smooth_flow_state(3, 40, 30)
    h = s.h.copy()
    h[7, 11] = 0.0
    with Grid(40, 30, 1.0, 1.0, 0.01, G, dtype="f64") as grid:
        grid.set_state(h, s.hu, s.hv)
        with pytest.raises(SweError) as e:
            grid.cfl_dt(0.2)
        assert e.value.status == 5  # SWE_ECHECK


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mass_conservation_on_gpu(dtype):
    from paper_1107_2157_gb300 import Grid
    s = si.single_bump_state(4)
    npd = np.float32 if dtype == "f32" else np.float64
    with Grid(128, 128, 1.0, 1.0, 0.04, G, dtype=dtype) as grid:
        grid.set_state(*(a.astype(npd) for a in (s.h, s.hu, s.hv)))
        m0 = grid.mass()
        grid.step(100)
        m1 = grid.mass()
    drift = abs(m1 - m0) / m0
    assert drift <= (1e-13 if dtype == "f64" else 1e-6), drift


# ---------------------------------------------------------------------------
# Full size, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------

N_FULL = 8192


def _full_windows(n, w=8, seed=12):
    rng = np.random.default_rng(seed)
    corners = [(1, w, 1, w), (n - w + 1, n, 1, w), (1, w, n - w + 1, n), (n - w + 1, n, n - w + 1, n)]
    edges = [(n // 2, n // 2 + w - 1, 1, w), (1, w, n // 3, n // 3 + w - 1),
             (n - w + 1, n, 2 * n // 3, 2 * n // 3 + w - 1), (n // 5, n // 5 + w - 1, n - w + 1, n)]
    inner = []
    for _ in range(4):
        i0, j0 = (int(v) for v in rng.integers(200, n - 200, 2))
        inner.append((i0, i0 + w - 1, j0, j0 + w - 1))
    # tile seams of the 128x32 (FP32) and 64x32 (FP64) tiles
    seams = [(128 * 20 - 3, 128 * 20 + 4, 32 * 50 - 3, 32 * 50 + 4)]
    # on the slopes of the first bumps of the initial state, where the flow
    # after 100 steps is far from still water
    slopes = []
    for b in si.large_grid_bumps(1, n)[:6]:
        for (ox, oy) in ((b.sigma, 0.0), (0.0, -0.5 * b.sigma)):
            i0 = int(min(max(round(b.cx + ox) - w // 2, 1), n - w + 1))
            j0 = int(min(max(round(b.cy + oy) - w // 2, 1), n - w + 1))
            slopes.append((i0, i0 + w - 1, j0, j0 + w - 1))
    return corners + edges + inner + seams + slopes


def window_errors(got, ic, n, dt, steps, windows, dtype):
    """Errors of the full-grid GPU state ``got`` on sampled windows against
    the oracle's exact window values.  The denominators are the parity
    scales (tests/parity.py) of the whole GPU field -- the window oracle does
    not see the whole grid -- and FP32 follows ``parity.f32_bar``: a field
    above 2e-5 must stay within twice the binary32 oracle's own error on the
    same windows."""
    den = scales([np.asarray(a) for a in got])
    worst, worst_b32 = [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]
    refs = []
    for w in windows:
        ref = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps)
        refs.append(ref)
        i0, i1, j0, j1 = w
        for k in range(3):
            sub = np.asarray(got[k][j0 - 1:j1, i0 - 1:i1], np.float64)
            worst[k] = max(worst[k], float(np.abs(sub - ref[k]).max()) / den[k])
    if dtype == "f64":
        return {"ok": max(worst) <= TOL_F64, "errs": worst}
    if max(worst) <= TOL_F32:
        return {"ok": True, "errs": worst}
    for w, ref in zip(windows, refs):
        b = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps, binary32=True)
        for k in range(3):
            worst_b32[k] = max(worst_b32[k], float(np.abs(b[k].astype(np.float64) - ref[k]).max()) / den[k])
    ok = all(worst[k] <= max(TOL_F32, B32_RATIO * worst_b32[k]) for k in range(3))
    return {"ok": ok, "errs": worst, "errs_b32": worst_b32}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_8192_sampled_windows(dtype):
    """8192x8192, 64 bumps: GPU after 100 steps vs exact oracle values on
    sampled windows (domain of dependence), plus mass and positivity after
    1000 steps."""
    from paper_1107_2157_gb300 import Grid
    n, steps = N_FULL, 100
    npd = np.float32 if dtype == "f32" else np.float64
    full = si.large_grid_state(seed=1, n=n)
    h0 = full.h.astype(npd)
    z = np.zeros_like(h0)
    with Grid(n, n, 1.0, 1.0, 0.01, G, dtype=dtype) as grid:
        grid.set_state(h0, z, z)
        dt = grid.cfl_dt(0.2)
        grid.set_dt(dt)
        m0 = grid.mass()
        grid.step(steps)
        got = grid.get_state()
        grid.step(1000 - steps)
        m1 = grid.mass()
        hlast = grid.get_state()[0]
        assert grid.check() == 0
    del full

    def ic(w):
        h = si.large_grid_state(seed=1, n=n, window=w).h.astype(npd).astype(np.float64)
        return h, np.zeros_like(h), np.zeros_like(h)

    errs = window_errors(got, ic, n, dt, steps, _full_windows(n), dtype)
    assert errs["ok"], errs
    assert np.isfinite(hlast).all() and hlast.min() > 0
    assert abs(m1 - m0) / m0 <= (1e-13 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("case", ["flat", "near_ties", "single_peak", "flow"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cfl_exact_on_flat_and_near_tie_states(case, dtype):
    """The CFL reduction screens cells with an FP32 estimate and evaluates
    FP64 only near the maximum; the result must still equal the oracle's
    exact FP64 minimum bitwise, including on plateaus and near-ties."""
    from paper_1107_2157_gb300 import Grid
    nx, ny, dx, dy = 333, 211, 0.9, 1.2
    npd = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(7)
    if case == "flat":
        h = np.full((ny, nx), 1.25); hu = np.full((ny, nx), 0.1); hv = np.full((ny, nx), -0.2)
    elif case == "near_ties":
        h = 1.0 + 1e-7 * rng.standard_normal((ny, nx)); hu = 1e-7 * rng.standard_normal((ny, nx))
        hv = np.zeros((ny, nx))
    elif case == "single_peak":
        h = np.full((ny, nx), 1.0); h[100, 200] = 1.0 + 1e-6; hu = np.zeros((ny, nx)); hv = np.zeros((ny, nx))
        hv[3, 5] = 1e-6
    else:
        s = si.smooth_flow_state(99, nx, ny)
        h, hu, hv = s.h, s.hu, s.hv
    h, hu, hv = (np.ascontiguousarray(a.astype(npd)) for a in (h, hu, hv))
    with Grid(nx, ny, dx, dy, 0.01, G, dtype=dtype) as grid:
        grid.set_state(h, hu, hv)
        dt = grid.cfl_dt(0.2)
    ref = oracle.cfl_dt(h.astype(np.float64), hu.astype(np.float64), hv.astype(np.float64), dx, dy, G, 0.2)
    assert dt == ref, (dt, ref)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_naive_and_tiled_kernels_give_identical_bits(dtype):
    """Every flux product is explicitly rounded, so a cell's update is the
    same function of its neighbours in every kernel and tile shape."""
    s = si.smooth_flow_state(31, 300, 141)
    if dtype == "f32":
        s = s.rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.9, 1.1, G, 0.3)
    a = run_gpu(s, 0.9, 1.1, dt, G, 25, dtype, KERNELS["tiled"])
    b = run_gpu(s, 0.9, 1.1, dt, G, 25, dtype, KERNELS["naive"])
    for k in range(3):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("nx,ny,steps", [(1, 1, 4), (3, 5, 7), (130, 66, 10), (257, 129, 9), (128, 32, 6),
                                         (300, 97, 11), (64, 200, 8)])
def test_two_step_kernel_equals_one_step_kernel_bitwise(dtype, nx, ny, steps):
    """The temporally blocked kernel (two steps per launch, intermediate state
    in shared memory) gives the same bits as one-step launches, also for odd
    step counts and ragged sizes with flow at every wall."""
    s = si.smooth_flow_state(nx * 7 + ny, nx, ny)
    if dtype == "f32":
        s = s.rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.8, 1.1, G, 0.3)
    a = run_gpu(s, 0.8, 1.1, dt, G, steps, dtype, KERNELS["tiled"])
    b = run_gpu(s, 0.8, 1.1, dt, G, steps, dtype, 3)
    for k in range(3):
        assert np.array_equal(a[k], b[k]), k


def test_two_step_kernel_full_size_windows_against_oracle():
    """8192^2 FP32 with the two-step kernel: sampled windows after 100 steps
    against the oracle, as for the one-step kernel."""
    from paper_1107_2157_gb300 import Grid
    n, steps = N_FULL, 100
    full = si.large_grid_state(seed=1, n=n)
    h0 = full.h.astype(np.float32)
    z = np.zeros_like(h0)
    with Grid(n, n, 1.0, 1.0, 0.01, G, dtype="f32", kernel=3) as grid:
        grid.set_state(h0, z, z)
        dt = grid.cfl_dt(0.2)
        grid.set_dt(dt)
        grid.step(steps)
        got = grid.get_state()
        assert grid.check() == 0
    del full

    def ic(w):
        h = si.large_grid_state(seed=1, n=n, window=w).h.astype(np.float32).astype(np.float64)
        return h, np.zeros_like(h), np.zeros_like(h)

    errs = window_errors(got, ic, n, dt, steps, _full_windows(n)[-8:], "f32")
    assert errs["ok"], errs


@pytest.mark.parametrize("nx,ny,steps", [(1, 1, 3), (3, 5, 7), (130, 66, 10), (257, 129, 9), (128, 32, 6),
                                         (300, 97, 11), (8, 200, 5), (1025, 40, 4)])
def test_packed_kernel_equals_plane_kernel_bitwise(nx, ny, steps):
    """The packed-state kernel ((h, hu, hv, 0) cells in one 16-byte vector)
    runs the same strip routine on its box, so it gives the plane kernel's
    bits, for ragged sizes with flow at every wall."""
    s = si.smooth_flow_state(nx * 11 + ny, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.8, 1.1, G, 0.3)
    a = run_gpu(s, 0.8, 1.1, dt, G, steps, "f32", KERNELS["tiled"])
    b = run_gpu(s, 0.8, 1.1, dt, G, steps, "f32", 4)
    for k in range(3):
        assert np.array_equal(a[k], b[k]), k


def test_packed_kernel_reductions_and_fp64_rejection():
    """Mass and CFL of a packed context read the current (packed) state;
    FP64 is not offered in the packed layout."""
    from paper_1107_2157_gb300 import Grid, swe
    s = si.smooth_flow_state(5, 200, 90).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    out = []
    for kernel in (KERNELS["tiled"], 4):
        with Grid(200, 90, 1.0, 1.0, dt, G, dtype="f32", kernel=kernel) as g:
            g.set_state(*(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
            m0 = g.mass()
            g.step(7)
            out.append((m0, g.mass(), g.cfl_dt(0.2), g.query(swe.SWE_Q_KERNEL)))
    assert out[0][:3] == out[1][:3]
    assert out[1][3] == 4
    with pytest.raises(swe.SweError) as e:
        Grid(16, 16, 1.0, 1.0, 0.01, G, dtype="f64", kernel=4)
    assert e.value.status == swe.SWE_EUNSUPPORTED


def test_auto_picks_the_streaming_two_step_kernel_for_fp32_and_fp64():
    from paper_1107_2157_gb300 import Grid, swe
    for dtype, shape in (("f32", 5), ("f64", 6)):
        with Grid(64, 64, 1.0, 1.0, 0.01, G, dtype=dtype) as g:
            assert g.query(swe.SWE_Q_KERNEL) == 3 and g.query(swe.SWE_Q_STEPS_PER_LAUNCH) == 2
            assert g.query(swe.SWE_Q_SHAPE) == shape


@pytest.mark.parametrize("nx,ny", [(1024, 96), (517, 263)])
def test_paired_interior_tiles_equal_the_scalar_naive_kernel(nx, ny):
    """Tiles away from an x-wall take the FP32 pair path (f32x2 arithmetic),
    tiles at a wall and the naive kernel the scalar one: same bits."""
    s = si.smooth_flow_state(nx + ny, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    ref = run_gpu(s, 1.0, 1.0, dt, G, 9, "f32", KERNELS["naive"])
    for kernel in (KERNELS["tiled"], 3, 4):
        got = run_gpu(s, 1.0, 1.0, dt, G, 9, "f32", kernel)
        for k in range(3):
            assert np.array_equal(got[k], ref[k]), (kernel, k)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_narrow_edge_tiles_equal_the_naive_kernel(dtype):
    """A tile that the grid's right side cuts within half (a quarter) of the
    tile width is computed by half- (quarter-) warps working on different
    rows, and the rows of a tile cut short by the top side are shared evenly
    among the warps.  Widths on both sides of each cut and ragged heights give
    the bits of the naive kernel (one thread per cell, no tiles)."""
    tx = 128 if dtype == "f32" else 64
    widths = [1, tx // 4, tx // 4 + 1, tx // 2, tx // 2 + 1, tx - 1, tx + tx // 4, tx + tx // 4 + 1,
              tx + tx // 2, tx + tx // 2 + 1, 2 * tx - 1]
    kernels = (KERNELS["tiled"], 3) + ((4,) if dtype == "f32" else ())
    for i, nx in enumerate(widths):
        ny = 5 + 13 * i
        s = si.smooth_flow_state(700 + i, nx, ny)
        if dtype == "f32":
            s = s.rounded_to(np.float32)
        dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
        ref = run_gpu(s, 1.0, 1.0, dt, G, 7, dtype, KERNELS["naive"])
        for kernel in kernels:
            got = run_gpu(s, 1.0, 1.0, dt, G, 7, dtype, kernel)
            for k in range(3):
                assert np.array_equal(got[k], ref[k]), (nx, ny, kernel, k)


def test_stencil_reciprocal_halves_when_its_argument_doubles():
    """The flux functions carry face states doubled (Coef in swe_device.cuh)
    and so rely on rcp(2x) = rcp(x) / 2 for the approximate FP32 reciprocal
    (exact for IEEE division).  Every significand of the binades of depths
    from 2^-8 to 2^16, each against the next binade, bit for bit; and the
    reciprocal stays within its documented one-ulp bound of the host's 1/x."""
    import torch
    from paper_1107_2157_gb300 import swe
    sig = np.arange(1 << 23, dtype=np.uint32)
    for e in (-8, -1, 0, 1, 3, 15):
        x = ((np.uint32(127 + e) << np.uint32(23)) | sig).view(np.float32)
        both = np.concatenate([x, 2 * x]).astype(np.float32)
        bd = torch.from_numpy(both).cuda()
        o = torch.empty_like(bd)
        swe.check(swe.lib().swe_selftest_div(bd.data_ptr(), bd.data_ptr(), o.data_ptr(), both.size, 4,
                                             swe.current_stream()), "swe_selftest_div")
        got = o.cpu().numpy()
        r1, r2 = got[:x.size], got[x.size:]
        bad = np.flatnonzero((0.5 * r1).view(np.uint32) != r2.view(np.uint32))
        assert bad.size == 0, (e, bad[:5], x[bad[:5]], r1[bad[:5]], r2[bad[:5]])
        exact = 1.0 / x.astype(np.float64)
        ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(r1 - exact) <= ulp), e


@pytest.mark.parametrize("variant,nx,ny", [(0, 1411, 777), (1, 1411, 777), (2, 1411, 777), (3, 1411, 777),
                                           (4, 1411, 777), (4, 130, 12811), (4, 257, 3001)])
def test_every_two_step_shape_equals_the_one_step_kernel_bitwise(variant, nx, ny):
    """Shapes 0..3 take one CTA per tile, shape 4 (the FP64 default) runs
    persistent CTAs that prefetch their next tile: all give the one-step
    kernel's bits, with ragged edges and an odd step count.  The tall grids
    have more tiles than resident CTAs, so each persistent CTA takes
    several."""
    from paper_1107_2157_gb300 import Grid
    steps = 7
    s = si.smooth_flow_state(4321, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.9, 1.1, G, 0.3)
    ref = run_gpu(s, 0.9, 1.1, dt, G, steps, "f32", KERNELS["tiled"])
    with Grid(nx, ny, 0.9, 1.1, dt, G, dtype="f32", kernel=3, variant=variant) as grid:
        grid.set_state(*(np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)))
        grid.step(steps)
        got = grid.get_state()
        assert grid.check() == 0
    for k in range(3):
        assert np.array_equal(got[k], ref[k]), (variant, k)


# widths around the strip ends of the streaming shapes (56 and 120 columns)
STREAM_WIDTHS = sorted({w for k in (1, 2, 3) for out in (56, 120) for w in
                        (k * out - 2, k * out - 1, k * out, k * out + 1, k * out + 2, k * out + 3)})
STREAM_CASES = [(v, nx, ny) for v in (5, 6, 7, 8) for nx, ny in ((1411, 777), (130, 12811), (257, 3001))] + \
    [(v, nx, ny) for v in (5, 7) for nx, ny in [(1, 1), (2, 3), (5, 2), (8, 4099)] +
     [(w, 3 + w % 37) for w in STREAM_WIDTHS]]


@pytest.mark.parametrize("variant,nx,ny", STREAM_CASES)
def test_streaming_two_step_shapes_equal_the_one_step_kernel_bitwise(variant, nx, ny):
    """Shapes 5..8 stream warps up column strips (56 stored columns per warp
    for one cell pair per lane, 120 for two) with the intermediate rows in
    registers and the walls as mirrored ghost columns.  The widths put the
    right wall in every lane position around a strip's end (including the
    width at which a strip's last stored column reads the ghost column), one-
    and two-row grids start and end a run on both walls at once, and the tall
    grids cut each strip into many row ranges: all give the one-step
    kernel's bits."""
    from paper_1107_2157_gb300 import Grid
    steps = 7
    s = si.smooth_flow_state(4321 + nx, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.9, 1.1, G, 0.3)
    ref = run_gpu(s, 0.9, 1.1, dt, G, steps, "f32", KERNELS["tiled"])
    with Grid(nx, ny, 0.9, 1.1, dt, G, dtype="f32", kernel=3, variant=variant) as grid:
        grid.set_state(*(np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)))
        grid.step(steps)
        got = grid.get_state()
        assert grid.check() == 0
    for k in range(3):
        bad = np.argwhere(got[k] != ref[k])
        assert bad.size == 0, (variant, k, bad[:4], got[k][tuple(bad[0])], ref[k][tuple(bad[0])])


STREAM64_WIDTHS = sorted({w for k in (1, 2, 3) for w in (60 * k - 2, 60 * k - 1, 60 * k, 60 * k + 1, 60 * k + 2)})
STREAM64_CASES = [(v, nx, ny) for v in (5, 6) for nx, ny in ((701, 389), (130, 3001))] + \
    [(v, nx, ny) for v in (5,) for nx, ny in [(1, 1), (2, 3), (5, 2), (8, 777)] +
     [(w, 3 + w % 29) for w in STREAM64_WIDTHS]]


@pytest.mark.parametrize("variant,nx,ny", STREAM64_CASES)
def test_fp64_streaming_shapes_equal_the_one_step_kernel_bitwise(variant, nx, ny):
    """FP64 streaming (two cells per lane, 60-column strips): the widths put
    the right wall at every lane position around a strip's end; all give the
    FP64 one-step kernel's bits after an odd number of steps."""
    from paper_1107_2157_gb300 import Grid
    steps = 7
    s = si.smooth_flow_state(977 + nx, nx, ny)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.9, 1.1, G, 0.3)
    ref = run_gpu(s, 0.9, 1.1, dt, G, steps, "f64", KERNELS["tiled"])
    with Grid(nx, ny, 0.9, 1.1, dt, G, dtype="f64", kernel=3, variant=variant) as grid:
        grid.set_state(*(np.ascontiguousarray(a, np.float64) for a in (s.h, s.hu, s.hv)))
        grid.step(steps)
        got = grid.get_state()
        assert grid.check() == 0
    for k in range(3):
        bad = np.argwhere(got[k] != ref[k])
        assert bad.size == 0, (variant, k, bad[:4])


def test_two_step_defaults_and_fp32_only_shapes():
    """The two-step default is streaming shape 5 for FP32 and 6 for FP64,
    and AUTO picks the two-step kernel for both; streaming shapes 7 and 8
    refuse FP64."""
    from paper_1107_2157_gb300 import Grid, SweError, swe
    with Grid(300, 200, 1.0, 1.0, 0.01, G, dtype="f32", kernel=3) as grid:
        assert grid.query(swe.SWE_Q_SHAPE) == 5
    with Grid(300, 200, 1.0, 1.0, 0.01, G, dtype="f64", kernel=3) as grid:
        assert grid.query(swe.SWE_Q_SHAPE) == 6
    for dtype in ("f32", "f64"):
        with Grid(300, 200, 1.0, 1.0, 0.01, G, dtype=dtype) as grid:
            assert grid.query(swe.SWE_Q_KERNEL) == 3 and grid.query(swe.SWE_Q_STEPS_PER_LAUNCH) == 2
    with Grid(300, 200, 1.0, 1.0, 0.01, G, dtype="f32", kernel=2) as grid:
        assert grid.query(swe.SWE_Q_SHAPE) == -1
    for v in (7, 8):
        with pytest.raises(SweError) as e:
            Grid(300, 200, 1.0, 1.0, 0.01, G, dtype="f64", kernel=3, variant=v)
        assert e.value.status == 6  # SWE_EUNSUPPORTED


@pytest.mark.parametrize("dtype,kernel,variant", [("f32", 1, None), ("f32", 2, None), ("f32", 3, None),
                                                   ("f32", 3, 4), ("f32", 4, None), ("f64", 2, None),
                                                   ("f64", 3, None)])
@pytest.mark.parametrize("steps", [0, 1, 6, 7])
def test_run_equals_cfl_step_and_mass_in_turn(dtype, kernel, variant, steps):
    """swe_run keeps the CFL step on the device and the step kernels read
    their coefficients from there: the dt, the state and the mass are those
    of swe_cfl_dt, swe_set_dt, swe_step and swe_mass in turn, bit for bit,
    for every kernel and an even or odd step count."""
    import torch
    from paper_1107_2157_gb300 import Grid
    nx, ny = 389, 263
    npd = np.float32 if dtype == "f32" else np.float64
    s = si.smooth_flow_state(71, nx, ny).rounded_to(npd)
    planes = [np.ascontiguousarray(a, npd) for a in (s.h, s.hu, s.hv)]
    with Grid(nx, ny, 0.8, 1.1, 0.01, G, dtype=dtype, kernel=kernel, variant=variant) as a:
        a.set_state(*planes)
        dt = a.cfl_dt(0.3)
        a.set_dt(dt)
        a.step(steps)
        m = a.mass()
        ref = a.get_state()
    with Grid(nx, ny, 0.8, 1.1, 0.01, G, dtype=dtype, kernel=kernel, variant=variant) as b:
        b.set_state(*planes)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        dt2, m2 = b.run(steps, 0.3, events=ev)
        got = b.get_state()
        assert b.check() == 0
        t = [ev[0].elapsed_time(e) for e in ev[1:]]
        assert 0.0 <= t[0] <= t[1] <= t[2], t
    assert dt2 == dt and m2 == m
    for k in range(3):
        assert np.array_equal(got[k], ref[k]), k


def test_run_leaves_the_state_alone_on_a_bad_depth():
    """A cell with h = 0: swe_run returns SWE_ECHECK with dt 0, the step
    kernels skip, and the state reads back unchanged; a good state run
    afterwards on the same context steps normally."""
    from paper_1107_2157_gb300 import Grid, SweError
    nx, ny = 300, 130
    s = si.smooth_flow_state(5, nx, ny).rounded_to(np.float32)
    h = np.ascontiguousarray(s.h, np.float32)
    h[40, 77] = 0.0
    planes = [h] + [np.ascontiguousarray(a, np.float32) for a in (s.hu, s.hv)]
    with Grid(nx, ny, 1.0, 1.0, 0.01, G, dtype="f32") as grid:
        grid.set_state(*planes)
        with pytest.raises(SweError) as e:
            grid.run(7, 0.2)
        assert e.value.status == 5  # SWE_ECHECK
        got = grid.get_state()
        for k in range(3):
            assert np.array_equal(got[k], planes[k]), k
        h[40, 77] = 1.0
        grid.set_state(*planes)
        dt, m = grid.run(7, 0.2)
        assert dt == oracle.cfl_dt(h.astype(np.float64), s.hu, s.hv, 1.0, 1.0, G, 0.2)
        assert not np.array_equal(grid.get_state()[0], h)


def test_fp32_mass_is_the_exact_sum_on_awkward_data():
    """The FP32 mass sums the depths exactly in 64-bit integers (flushing to
    FP64 only when the largest exponent rises): on depths within a few
    binades, straddling powers of two, with zeros, negative values and row
    tails (nx % 4 != 0), it equals the exactly rounded sum of the same values
    (math.fsum) to a few units in the last place; over 50 binades, where the
    values far below a thread's largest go to its FP64 total, to 1e-14."""
    import math
    from paper_1107_2157_gb300 import Grid
    rng = np.random.default_rng(23)
    nx, ny = 1027, 333
    cases = {
        "one binade": 1.0 + 0.99 * rng.random((ny, nx)),
        "straddling 1 and 2": 0.7 + 1.6 * rng.random((ny, nx)),
        "wide": 2.0 ** rng.uniform(-30, 20, (ny, nx)),
        "signs and zeros": np.where(rng.random((ny, nx)) < 0.3, 0.0, rng.standard_normal((ny, nx))),
    }
    for name, h in cases.items():
        h = h.astype(np.float32)
        z = np.zeros_like(h)
        with Grid(nx, ny, 1.0, 1.0, 0.01, G, dtype="f32") as grid:
            grid.set_state(h, z, z)
            m = grid.mass()
        want = math.fsum(h.astype(np.float64).ravel())
        tol = 1e-14 * abs(want) if name == "wide" else 4 * math.ulp(abs(want))
        assert abs(m - want) <= tol, (name, m, want)


def test_rank_partition_edges_and_ghosts_follow_the_strip_layout():
    """swe_part_edges writes left, right, bottom, top edge strips (h, hu, hv
    each, in row / column order); swe_part_set_ghosts writes only the sides
    in its mask, and a step then reads them: a partition whose every side
    faces another rank, fed the ghosts a wall would give, steps exactly like
    a partition with four walls."""
    import torch
    from paper_1107_2157_gb300 import Partitioned
    from paper_1107_2157_gb300 import partition as P
    nx, ny = 37, 23
    s = si.smooth_flow_state(9, nx, ny).rounded_to(np.float32)
    fields = [np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)]
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    n = 6 * (nx + ny)
    open_p = Partitioned.rank(nx, ny, 0, 1.0, 1.0, dt, G)
    walls_p = Partitioned.rank(nx, ny, 15, 1.0, 1.0, dt, G)
    try:
        for p in (open_p, walls_p):
            p.set_state(*fields)
        edges = torch.empty(n, dtype=torch.float32, device="cuda")
        open_p.edges(edges)
        e = edges.cpu().numpy()
        want = {P.LEFT: [f[:, 0] for f in fields], P.RIGHT: [f[:, -1] for f in fields],
                P.BOTTOM: [f[0, :] for f in fields], P.TOP: [f[-1, :] for f in fields]}
        for side in P.SIDES:
            got = e[P.strip_slice(side, nx, ny)].reshape(3, -1)
            for k in range(3):
                assert np.array_equal(got[k], want[side][k]), (side, k)
        # the reflective ghosts of every side: edge cells, normal momentum negated
        ghosts = np.empty(n, np.float32)
        for side in P.SIDES:
            strip = np.stack(want[side]).copy()
            strip[1 if side in (P.LEFT, P.RIGHT) else 2] *= -1.0
            ghosts[P.strip_slice(side, nx, ny)] = strip.ravel()
        g = torch.from_numpy(ghosts).cuda()
        open_p.set_ghosts(g, 1 | 2)       # left and right now
        open_p.set_ghosts(g, 4 | 8)       # then bottom and top
        open_p.step(1)
        walls_p.step(1)
        a, b = open_p.get_state(), walls_p.get_state()
        for k in range(3):
            assert np.array_equal(a[k], b[k]), k
    finally:
        open_p.close()
        walls_p.close()
