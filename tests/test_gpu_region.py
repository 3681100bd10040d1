"""The step and wall fill written as region statements (swe_region_*)
against the oracle: bit for bit in FP64 against the FP64 oracle and in FP32
against the oracle's binary32 step (every statement operation is one IEEE
round-to-nearest operation in the oracle's order), and within the FP32 bar
of the FP64 oracle, on ragged sizes across every tile shape; plus the Sec.
2.3 semantics that the step reads whatever the ghosts hold, and the FP32
division those statements use."""

import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import B32_RATIO, G, TOL_F32, b32_run, f32_bar, scales_from_max

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (1, 9), (9, 1), (3, 5), (32, 16), (64, 8), (65, 9), (127, 31), (200, 37), (130, 70), (33, 200)]


def _np(dtype):
    from paper_1107_2157_gb300 import swe
    return np.float64 if dtype == swe.SWE_F64 else np.float32


def _upload(planes, arrays):
    """Padded (ny + 2) x (nx + 2) arrays into the planes' first nx + 2 columns."""
    import torch
    for P, a in zip(planes, arrays):
        P[:, :a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a)).to(device=P.device, dtype=P.dtype)


def _download(planes, nx):
    import torch
    torch.cuda.synchronize()
    return [P[:, :nx + 2].cpu().numpy().astype(np.float64) for P in planes]


def _padded(s, npd):
    return [oracle.pad(np.asarray(a, npd).astype(np.float64)) for a in (s.h, s.hu, s.hv)]


def _ok(reg):
    from paper_1107_2157_gb300 import swe
    assert reg.query(swe.SWE_RQ_ERROR) == 0


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_fp64_step_is_the_oracle_bit_for_bit(variant, nx, ny):
    from paper_1107_2157_gb300 import Region, swe
    s = si.smooth_flow_state(nx * 977 + ny, nx, ny)
    dx, dy = 0.8, 1.1
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3)
    H, U, V = _padded(s, np.float64)
    oracle.fill_halo(H, U, V)
    ref, _, _ = oracle.step_padded(H, U, V, dx, dy, dt, G)
    with Region(swe.SWE_F64, nx, ny, variant=variant) as reg:
        a, b = reg.planes(), reg.planes()
        _upload(a, [np.nan_to_num(x) for x in (H, U, V)])  # corner ghosts (NaN in the oracle) are never read
        reg.step(a, b, dx, dy, dt, G)
        got = _download(b, nx)
        _ok(reg)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k][1:-1, 1:-1]), k
        assert not got[k][0].any() and not got[k][-1].any()       # ghosts of the output untouched
        assert not got[k][:, 0].any() and not got[k][:, -1].any()


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (65, 9), (200, 37)])
def test_fp64_run_with_walls_is_the_oracle_bit_for_bit(nx, ny):
    from paper_1107_2157_gb300 import Region, swe
    s = si.smooth_flow_state(nx * 31 + ny, nx, ny)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.25)
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 25)
    with Region(swe.SWE_F64, nx, ny) as reg:
        a, b = reg.planes(), reg.planes()
        _upload(a, _padded(s, np.float64))
        in_b = reg.run(a, b, 25, 1.0, 1.0, dt, G)
        got = _download(b if in_b else a, nx)
        assert in_b == 1
        assert reg.query(swe.SWE_RQ_LAUNCHES) == 50
        _ok(reg)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k]), k


@pytest.mark.parametrize("walls", [0, 1, 2, 4, 8, 5, 10, 15])
@pytest.mark.parametrize("dtype", [0, 1])
def test_wall_fill_is_the_oracle_ghost_rule(walls, dtype):
    from paper_1107_2157_gb300 import Region
    nx, ny = 37, 21
    rng = np.random.default_rng(walls * 2 + dtype)
    npd = _np(dtype)
    arrs = [rng.standard_normal((ny + 2, nx + 2)).astype(npd).astype(np.float64) for _ in range(3)]
    ref = [a.copy() for a in arrs]
    oracle.fill_halo(*ref, walls=walls)
    with Region(dtype, nx, ny) as reg:
        st = reg.planes()
        _upload(st, arrs)
        reg.walls(st, walls)
        got = _download(st, nx)
        _ok(reg)
    corners = np.zeros((ny + 2, nx + 2), bool)
    corners[[0, 0, -1, -1], [0, -1, 0, -1]] = True
    for k in range(3):
        assert np.array_equal(got[k][~corners], ref[k][~corners]), k
        assert np.array_equal(got[k][corners], arrs[k][corners])  # corners untouched


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (65, 9), (127, 31), (257, 129), (64, 200)])
def test_fp32_run_matches_the_oracle(variant, nx, ny):
    from paper_1107_2157_gb300 import Region, swe
    s = si.smooth_flow_state(nx * 1000 + ny, nx, ny).rounded_to(np.float32)
    dx, dy = 0.8, 1.1
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3)
    ref = oracle.run(s.h, s.hu, s.hv, dx, dy, dt, G, 20)
    with Region(swe.SWE_F32, nx, ny, variant=variant) as reg:
        a, b = reg.planes(), reg.planes()
        _upload(a, _padded(s, np.float32))
        in_b = reg.run(a, b, 20, dx, dy, dt, G)
        got = _download(b if in_b else a, nx)
        _ok(reg)
    # bit for bit the oracle's binary32 step, the paper's precision, and so
    # within the FP32 bar against the FP64 oracle (parity.f32_bar)
    ref32 = oracle.run_f32(s.h, s.hu, s.hv, dx, dy, dt, G, 20)
    ok, errs, errs_b32 = f32_bar([g[1:-1, 1:-1] for g in got], ref, ref32)
    assert ok, (errs, errs_b32)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref32[k].astype(np.float64)), k


def test_fp32_tile_shapes_agree_bitwise_and_with_the_hand_kernel():
    """The statements do not depend on the tile shape, so neither do the
    bits; the hand-written kernel (FMA, approximate reciprocal) agrees to
    the FP32 bar."""
    from paper_1107_2157_gb300 import Grid, Region, swe
    nx, ny = 300, 170
    s = si.smooth_flow_state(7, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    outs = []
    for variant in (1, 2, 3, 4, 5):
        with Region(swe.SWE_F32, nx, ny, variant=variant) as reg:
            a, b = reg.planes(), reg.planes()
            _upload(a, _padded(s, np.float32))
            in_b = reg.run(a, b, 15, 1.0, 1.0, dt, G)
            outs.append(_download(b if in_b else a, nx))
    for o in outs[1:]:
        for k in range(3):
            assert np.array_equal(o[k], outs[0][k])
    with Grid(nx, ny, 1.0, 1.0, dt, G, dtype="f32") as grid:
        grid.set_state(*(np.ascontiguousarray(x, np.float32) for x in (s.h, s.hu, s.hv)))
        grid.step(15)
        hand = grid.get_state()
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, 15)
    b32 = b32_run(s, 1.0, 1.0, dt, G, 15)
    ok_region, e_region, _ = f32_bar([x[1:-1, 1:-1] for x in outs[0]], ref, b32)
    ok_hand, e_hand, e_b32 = f32_bar(hand, ref, b32)
    assert ok_region and ok_hand, (e_region, e_hand, e_b32)


def test_step_reads_the_ghosts_it_is_given():
    """Sec. 2.3: boundary conditions stay outside the kernel.  A window of a
    larger grid, its ghost ring holding the true neighbour cells, steps to
    exactly the larger grid's values on the window (FP64, bitwise)."""
    from paper_1107_2157_gb300 import Region, swe
    NX, NY = 150, 110
    s = si.smooth_flow_state(99, NX, NY)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    full = _padded(s, np.float64)
    oracle.fill_halo(*full)
    ref, _, _ = oracle.step_padded(*full, 1.0, 1.0, dt, G)
    i0, i1, j0, j1 = 37, 120, 20, 95             # 1-based inclusive window of interior cells
    nx, ny = i1 - i0 + 1, j1 - j0 + 1
    win = [F[j0 - 1:j1 + 2, i0 - 1:i1 + 2] for F in full]
    with Region(swe.SWE_F64, nx, ny) as reg:
        a, b = reg.planes(), reg.planes()
        _upload(a, win)
        reg.step(a, b, 1.0, 1.0, dt, G)
        got = _download(b, nx)
        _ok(reg)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k][j0:j1 + 1, i0:i1 + 1]), k


def test_rejects_misaligned_planes_and_counts_launches():
    import torch
    from paper_1107_2157_gb300 import Region, swe
    with Region(swe.SWE_F32, 40, 30) as reg:
        a, b = reg.planes(), reg.planes()
        bad = [a[0].data_ptr() + 4, a[1].data_ptr(), a[2].data_ptr()]
        with pytest.raises(swe.SweError) as e:
            reg.step(bad, b, 1.0, 1.0, 0.01, G)
        assert e.value.status == swe.SWE_EINVAL
        with pytest.raises(swe.SweError):
            reg.walls(a, 16)
        assert reg.query(swe.SWE_RQ_LAUNCHES) == 0
        for P in a:
            P.fill_(1.0)
        reg.run(a, b, 3, 1.0, 1.0, 0.01, G)
        torch.cuda.synchronize()
        assert reg.query(swe.SWE_RQ_LAUNCHES) == 6
        assert reg.query(swe.SWE_RQ_TILE_X) == 32 and reg.query(swe.SWE_RQ_TILE_Y) == 32
        _ok(reg)


N_FULL = 8192


def test_full_size_fp32_region_run_sampled_windows():
    """The benchmark's region launch configuration: 8192 x 8192 FP32, 64
    bumps at rest, walls + step per step; after 60 steps, exact oracle
    values on sampled windows (domain of dependence)."""
    import torch
    from paper_1107_2157_gb300 import Region, swe
    n, steps = N_FULL, 60
    full = si.large_grid_state(seed=1, n=n)
    h0 = full.h.astype(np.float32)
    del full
    dt = oracle.cfl_dt(h0[::8, ::8], 0 * h0[::8, ::8], 0 * h0[::8, ::8], 1.0, 1.0, G, 0.2)
    with Region(swe.SWE_F32, n, n) as reg:
        a, b = reg.planes(), reg.planes()
        a[0][1:-1, 1:n + 1] = torch.from_numpy(h0).cuda()
        in_b = reg.run(a, b, steps, 1.0, 1.0, dt, G)
        res = b if in_b else a
        torch.cuda.synchronize()
        _ok(reg)
        wins = [(1, 48, 1, 48), (8145, 8192, 8145, 8192), (4000, 4100, 1, 40), (1, 40, 3000, 3090),
                (2000, 2100, 5000, 5100), (8150, 8192, 100, 200)]
        got = {w: [P[w[2]:w[3] + 1, w[0]:w[1] + 1].cpu().numpy().astype(np.float64) for P in res] for w in wins}
        # parity scales of the whole fields (the window oracle sees windows only)
        den = scales_from_max([float(P[1:-1, 1:n + 1].abs().max()) for P in res])

    def ic(w):
        h = si.large_grid_state(seed=1, n=n, window=w).h.astype(np.float32).astype(np.float64)
        return h, np.zeros_like(h), np.zeros_like(h)

    for w in wins:
        ref = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps)
        ref32 = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps, binary32=True)
        for k in range(3):
            # bit for bit the binary32 oracle, hence within the FP32 bar
            assert np.array_equal(got[w][k], ref32[k].astype(np.float64)), (w, k)
            err = np.abs(got[w][k] - ref[k]).max() / den[k]
            err_b32 = np.abs(ref32[k].astype(np.float64) - ref[k]).max() / den[k]
            assert err <= max(TOL_F32, B32_RATIO * err_b32), (w, k, err, err_b32)


def _div_cases(seed):
    """Operand pairs for the division test: random bit patterns (every class:
    zeros, subnormals, infinities, NaNs), random magnitudes across the
    binary32 range and across the statements' fast-path range and its
    edges, near-midpoint quotients (a = RN(b m)
    for m halfway between two floats: the hardest rounding decisions), and
    special values against each other."""
    rng = np.random.default_rng(seed)
    n = 1 << 21
    out = []
    out.append(rng.integers(0, 2 ** 32, size=(2, n), dtype=np.uint64).astype(np.uint32).view(np.float32))
    e = rng.integers(-110, 128, size=(2, n))
    m = rng.uniform(1.0, 2.0, size=(2, n)) * rng.choice([-1.0, 1.0], size=(2, n))
    out.append(np.ldexp(m, e).astype(np.float32))
    # inside the fast path's range (2^-100 <= |a| < 2^100, 2^-20 <= |b| < 2^20) and just outside it
    e = np.stack([rng.integers(-101, 101, n), rng.integers(-21, 21, n)])
    m = rng.uniform(1.0, 2.0, size=(2, n)) * rng.choice([-1.0, 1.0], size=(2, n))
    out.append(np.ldexp(m, e).astype(np.float32))
    b = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-30, 30, n)).astype(np.float32)
    q = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-30, 30, n)).astype(np.float32)
    q_up = np.nextafter(q, np.float32(np.inf))
    mid = (q.astype(np.float64) + q_up.astype(np.float64)) / 2            # exact in float64
    a = (b.astype(np.float64) * mid).astype(np.float32)                   # b (24 bits) x mid (25 bits) is exact in float64
    a2 = np.nextafter(a, np.float32(np.inf))
    out.append(np.stack([np.concatenate([a, a2]), np.concatenate([b, b])]))
    ones = np.uint32(0x3FFFFFFF) + (np.arange(64, dtype=np.uint32) << 23)  # significand all ones, many binades
    sp = np.concatenate([np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0, 0.5, 3.0,
                                   np.finfo(np.float32).max, np.finfo(np.float32).tiny, 1e-45, 1e-40, 2.0 ** -100,
                                   2.0 ** -101, 2.0 ** 126, 2.0 ** 127, 2.0 ** -20, 2.0 ** 20, 2.0 ** 100,
                                   np.nextafter(np.float32(2.0 ** -20), np.float32(0)),
                                   np.nextafter(np.float32(2.0 ** 20), np.float32(0)),
                                   np.nextafter(np.float32(2.0 ** 100), np.float32(0))], np.float32),
                         ones.view(np.float32)])
    A, B = np.meshgrid(sp, sp)
    out.append(np.stack([A.ravel(), B.ravel()]))
    return np.concatenate(out, axis=1).astype(np.float32)


def test_fp32_division_reciprocal_step_is_correctly_rounded_for_every_significand():
    """The statements' division finishes with one FMA (Markstein's theorem),
    which needs its reciprocal to be RN(1/b).  Every significand but the
    all-ones one (which the division sends to __fdiv_rn), in the lowest,
    middle and highest binade of the fast range: the reciprocal step equals
    the host's RN(1/b) (1/b in float64, then rounded to float32: 1/b is never
    within 2^-49 relative of a float32 midpoint, so the double rounding is
    exact)."""
    import torch
    from paper_1107_2157_gb300 import swe
    sig = np.arange((1 << 23) - 1, dtype=np.uint32)  # all significands but 0x7fffff
    outs = []
    for e in (-20, 0, 19):
        b = ((np.uint32(127 + e) << np.uint32(23)) | sig).view(np.float32)
        bd = torch.from_numpy(b).cuda()
        o = torch.empty_like(bd)
        swe.check(swe.lib().swe_selftest_div(bd.data_ptr(), bd.data_ptr(), o.data_ptr(), b.size, 3,
                                             swe.current_stream()), "swe_selftest_div")
        want = (1.0 / b.astype(np.float64)).astype(np.float32)
        got = o.cpu().numpy()
        bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
        assert bad.size == 0, (e, bad[:5], b[bad[:5]], got[bad[:5]], want[bad[:5]])


def test_fp32_division_is_correctly_rounded():
    """The statements' FP32 division (FMA scheme with an exact rounding test),
    alone and on element pairs as the paired evaluation takes it, against
    CUDA's __fdiv_rn and the host's IEEE division, bit for bit."""
    import torch
    from paper_1107_2157_gb300 import swe
    ab = _div_cases(5)
    n = ab.shape[1]
    a, b = (torch.from_numpy(np.ascontiguousarray(ab[k])).cuda() for k in range(2))
    if n % 2:
        ab = ab[:, :-1]
        n -= 1
        a, b = a[:n], b[:n]
    outs = []
    for which in (0, 1, 2):
        o = torch.empty_like(a)
        swe.check(swe.lib().swe_selftest_div(a.data_ptr(), b.data_ptr(), o.data_ptr(), n, which,
                                             swe.current_stream()), "swe_selftest_div")
        outs.append(o.cpu().numpy())
    with np.errstate(all="ignore"):
        host = ab[0] / ab[1]
    mine, cuda, paired = outs
    nan = np.isnan(host)
    for got in (mine, cuda, paired):
        assert np.array_equal(np.isnan(got), nan)
        assert np.array_equal(got[~nan].view(np.uint32), host[~nan].view(np.uint32))
