"""Open sides and the step over a bottom topography in the region front end
(swe_region_boundary, swe_region_step_bed, swe_region_run_bc) against the
FP64 oracle of swe_oracle_bathy.c: FP64 bit for bit, FP32 within the FP32
bar; the lake at rest over a bed on the GPU; and the benchmark's topography
launch at 8192^2 on sampled windows."""
import math

import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import G, TOL_F32, f32_bar, scales_from_max

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (3, 5), (32, 16), (65, 9), (127, 31), (200, 37), (33, 200)]


def _upload(planes, arrays):
    import torch
    for P, a in zip(planes, arrays):
        P[:, :a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a)).to(device=P.device, dtype=P.dtype)


def _download(planes, nx):
    import torch
    torch.cuda.synchronize()
    return [P[:, :nx + 2].cpu().numpy().astype(np.float64) for P in planes]


def _bed_plane(reg, b):
    """The bed as a plane of the region's layout, ghosts copying the edges."""
    import torch
    P = reg.planes()[0]
    B = np.nan_to_num(oracle.pad_bed(b))
    P[:, :B.shape[1]] = torch.from_numpy(B).to(device=P.device, dtype=P.dtype)
    return P


def _case(nx, ny, seed):
    s = si.smooth_flow_state(seed, nx, ny)
    mounds = si.multi_bumps(seed, 9, nx, ny, 3, amp_range=(0.05, 0.3), sigma_range=(2.0, 6.0))
    b = si.bumps_h(nx, ny, 0.0, mounds)
    return s, b


def _ok(reg):
    from paper_1107_2157_gb300 import swe
    assert reg.query(swe.SWE_RQ_ERROR) == 0


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_fp64_bed_step_is_the_oracle_bit_for_bit(variant, nx, ny):
    from paper_1107_2157_gb300 import Region, swe
    s, b = _case(nx, ny, nx * 31 + ny)
    H, U, V = oracle.pad(s.h + 0.5), oracle.pad(s.hu), oracle.pad(s.hv)
    oracle.fill_halo(H, U, V)
    B = oracle.pad_bed(b)
    dt = 0.25 / math.sqrt(G * 3.0)
    ref = oracle.step_padded_bathy(H, U, V, B, 0.8, 1.1, dt, G)
    with Region(swe.SWE_F64, nx, ny, variant=variant) as reg:
        a, o = reg.planes(), reg.planes()
        _upload(a, [np.nan_to_num(x) for x in (H, U, V)])
        reg.step_bed(a, _bed_plane(reg, b), o, 0.8, 1.1, dt, G)
        got = _download(o, nx)
        _ok(reg)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k][1:-1, 1:-1]), k


@pytest.mark.parametrize("kinds", [(2, 2, 2, 2), (2, 1, 2, 1), (1, 2, 1, 2), (1, 1, 1, 1)])
@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (65, 9), (130, 70)])
def test_fp64_run_with_open_sides_and_bed_is_the_oracle_bit_for_bit(kinds, nx, ny):
    from paper_1107_2157_gb300 import Region, swe
    s, b = _case(nx, ny, nx + 7 * ny)
    h = s.h + 0.5
    dt = oracle.cfl_dt(h, s.hu, s.hv, 1.0, 1.0, G, 0.25)
    walls = sum(1 << i for i in range(4) if kinds[i] == 1)
    opens = sum(1 << i for i in range(4) if kinds[i] == 2)
    ref = oracle.run_bc(h, s.hu, s.hv, 1.0, 1.0, dt, G, 25, walls=walls, open_sides=opens, bed=b)
    with Region(swe.SWE_F64, nx, ny) as reg:
        a, o = reg.planes(), reg.planes()
        _upload(a, [oracle.pad(x) for x in (h, s.hu, s.hv)])
        in_b = reg.run_bc(a, o, 25, 1.0, 1.0, dt, G, kinds=kinds, bed=_bed_plane(reg, b))
        got = _download(o if in_b else a, nx)
        _ok(reg)
    for k in range(3):
        assert np.array_equal(got[k][1:-1, 1:-1], ref[k]), k


@pytest.mark.parametrize("variant", [1, 3, 5])
def test_fp32_run_with_open_sides_and_bed_matches_the_oracle(variant):
    from paper_1107_2157_gb300 import Region, swe
    nx, ny = 257, 129
    s, b = _case(nx, ny, 11)
    st = si.State(s.h + 0.5, s.hu, s.hv).rounded_to(np.float32)
    b32 = b.astype(np.float32).astype(np.float64)
    dt = oracle.cfl_dt(st.h, st.hu, st.hv, 1.0, 1.0, G, 0.25)
    ref = oracle.run_bc(st.h, st.hu, st.hv, 1.0, 1.0, dt, G, 20, walls=2 | 8, open_sides=1 | 4, bed=b32)
    with Region(swe.SWE_F32, nx, ny, variant=variant) as reg:
        a, o = reg.planes(), reg.planes()
        _upload(a, [oracle.pad(x) for x in (st.h, st.hu, st.hv)])
        in_b = reg.run_bc(a, o, 20, 1.0, 1.0, dt, G, kinds=(2, 1, 2, 1), bed=_bed_plane(reg, b32))
        got = _download(o if in_b else a, nx)
        _ok(reg)
    ok, errs, _ = f32_bar([g[1:-1, 1:-1] for g in got], ref)
    assert ok, errs


@pytest.mark.parametrize("dtype", [0, 1])
def test_boundary_kinds_are_the_oracle_fills(dtype):
    from paper_1107_2157_gb300 import Region
    nx, ny = 37, 21
    rng = np.random.default_rng(dtype)
    npd = np.float32 if dtype == 0 else np.float64
    arrs = [rng.standard_normal((ny + 2, nx + 2)).astype(npd).astype(np.float64) for _ in range(3)]
    for kinds in [(2, 2, 2, 2), (1, 2, 0, 2), (0, 0, 2, 1), (2, 0, 0, 0)]:
        ref = [a.copy() for a in arrs]
        walls = sum(1 << i for i in range(4) if kinds[i] == 1)
        opens = sum(1 << i for i in range(4) if kinds[i] == 2)
        oracle.fill_halo(*ref, walls=walls)
        oracle.fill_open(*ref, sides=opens)
        with Region(dtype, nx, ny) as reg:
            st = reg.planes()
            _upload(st, arrs)
            reg.boundary(st, kinds)
            got = _download(st, nx)
            _ok(reg)
        corners = np.zeros((ny + 2, nx + 2), bool)
        corners[[0, 0, -1, -1], [0, -1, 0, -1]] = True
        for k in range(3):
            assert np.array_equal(got[k][~corners], ref[k][~corners]), (kinds, k)


@pytest.mark.parametrize("dtype,bound", [(0, 1e-4), (1, 1e-12)])
def test_lake_at_rest_over_a_bed_stays_at_rest(dtype, bound):
    from paper_1107_2157_gb300 import Region
    nx, ny = 200, 150
    mounds = si.multi_bumps(3, 9, nx, ny, 6, amp_range=(0.1, 0.4), sigma_range=(5.0, 20.0))
    b = si.bumps_h(nx, ny, 0.0, mounds)
    npd = np.float32 if dtype == 0 else np.float64
    b = b.astype(npd).astype(np.float64)
    h = (1.5 - b).astype(npd).astype(np.float64)
    z = np.zeros_like(h)
    dt = 0.3 / math.sqrt(G * 1.5)
    with Region(dtype, nx, ny) as reg:
        a, o = reg.planes(), reg.planes()
        _upload(a, [oracle.pad(x) for x in (h, z, z)])
        in_b = reg.run_bc(a, o, 300, 1.0, 1.0, dt, G, kinds=(1, 2, 1, 2), bed=_bed_plane(reg, b))
        got = _download(o if in_b else a, nx)
        _ok(reg)
    wave = 1.5 * math.sqrt(G * 1.5)
    current = max(np.abs(got[1][1:-1, 1:-1]).max(), np.abs(got[2][1:-1, 1:-1]).max()) / wave
    assert current <= bound, current


def test_rejects_bad_kinds_and_missing_bed():
    from paper_1107_2157_gb300 import Region, swe
    with Region(swe.SWE_F32, 20, 10) as reg:
        a, o = reg.planes(), reg.planes()
        with pytest.raises(swe.SweError):
            reg.boundary(a, (3, 0, 0, 0))
        with pytest.raises(swe.SweError):
            reg.boundary(a, (-1, 0, 0, 0))
        with pytest.raises(swe.SweError):
            reg.step_bed(a, 0, o, 1.0, 1.0, 0.01, G)
        assert reg.query(swe.SWE_RQ_LAUNCHES) == 0


def test_full_size_fp32_topography_run_sampled_windows():
    """The benchmark's topography launch: 8192 x 8192 FP32, the default
    workload's surface over 32 bed mounds, left and right sides open, bottom
    and top walls; after 40 steps, exact FP64 oracle values on sampled
    windows (domain of dependence), FP32 bar."""
    import torch
    from paper_1107_2157_gb300 import Region, swe
    n, steps = 8192, 40
    st = si.large_grid_bed_state(n=n)
    h0 = st.h.astype(np.float32)
    del st
    bed = si.large_grid_bed(n=n).astype(np.float32)
    assert h0.min() > 0.3
    dt = 0.2 / math.sqrt(G * float(h0.max()))
    kinds = (2, 2, 1, 1)
    with Region(swe.SWE_F32, n, n) as reg:
        a, b = reg.planes(), reg.planes()
        B = reg.planes()[0]
        a[0][1:-1, 1:n + 1] = torch.from_numpy(h0).cuda()
        B[1:-1, 1:n + 1] = torch.from_numpy(bed).cuda()
        B[0], B[-1] = B[1], B[-2]
        B[:, 0], B[:, n + 1] = B[:, 1], B[:, n]
        in_b = reg.run_bc(a, b, steps, 1.0, 1.0, dt, G, kinds=kinds, bed=B)
        res = b if in_b else a
        torch.cuda.synchronize()
        _ok(reg)
        wins = [(1, 40, 1, 40), (8153, 8192, 8153, 8192), (1, 40, 4000, 4060), (8160, 8192, 2000, 2050),
                (3000, 3080, 5000, 5080)]
        got = {w: [P[w[2]:w[3] + 1, w[0]:w[1] + 1].cpu().numpy().astype(np.float64) for P in res] for w in wins}
        # parity scales of the whole fields (the window oracle sees windows only)
        den = scales_from_max([float(P[1:-1, 1:n + 1].abs().max()) for P in res])

    def ic(w):
        h = si.large_grid_bed_state(n=n, window=w).h.astype(np.float32).astype(np.float64)
        return h, np.zeros_like(h), np.zeros_like(h)

    def bedw(w):
        return si.large_grid_bed(n=n, window=w).astype(np.float32).astype(np.float64)

    for w in wins:
        ref = oracle.run_window(ic, n, n, w, 1.0, 1.0, dt, G, steps, open_sides=1 | 2, bed=bedw)
        for k in range(3):
            err = np.abs(got[w][k] - ref[k]).max() / den[k]
            assert err <= TOL_F32, (w, k, err)
