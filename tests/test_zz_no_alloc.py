"""swe_mass_noalloc: the FP64 mass of a caller-owned device plane, computed
with scratch in a static device array instead of allocated memory.

Callers that cannot allocate device memory (their GPU memory is owned by
another allocator, or their loop cannot afford the synchronisation that
cudaMalloc/cudaFree may cause) call this entry point with their own buffers.
The test calls it through the C ABI on two different grids, twice in a row,
and checks each result against swe_mass of the same state, within the 1e-14
relative bound the other mass tests use.  This file sorts last so that a run
stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

import swe_inputs as si

pytestmark = pytest.mark.gpu


def _grid_with_state(nx, ny, dx, dy, dtype, seed):
    from paper_1107_2157_gb300 import Grid
    npd = np.float32 if dtype == "f32" else np.float64
    s = si.smooth_flow_state(seed, nx, ny)
    grid = Grid(nx, ny, dx, dy, 0.01, 9.8, dtype=dtype)
    grid.set_state(*(a.astype(npd) for a in (s.h, s.hu, s.hv)))
    return grid


def test_noalloc_mass_matches_swe_mass_on_two_calls_in_a_row():
    import torch
    from paper_1107_2157_gb300 import swe

    cases = [(700, 513, 0.6, 1.3, "f32", 21), (257, 1030, 1.1, 0.9, "f64", 22)]
    grids = [_grid_with_state(*c) for c in cases]
    try:
        refs = [g.mass() for g in grids]
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for rep in range(2):
            out.fill_(float("nan"))
            for k, ((nx, ny, dx, dy, dtype, _), g) in enumerate(zip(cases, grids)):
                swe.swe_mass_noalloc(swe.SWE_F32 if dtype == "f32" else swe.SWE_F64,
                                     g.query(swe.SWE_Q_STATE_PTR), nx, ny, g.query(swe.SWE_Q_PITCH),
                                     dx, dy, out.data_ptr() + 8 * k, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for k in range(2):
                assert abs(got[k] - refs[k]) <= 1e-14 * abs(refs[k]), (rep, k, got[k], refs[k])
    finally:
        for g in grids:
            g.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    from paper_1107_2157_gb300 import swe

    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = swe.lib().swe_mass_noalloc
    # wider than SWE_NOALLOC_MAX_DIM (the buffer is never touched: rejected on the host)
    assert f(swe.SWE_F32, buf.data_ptr(), 70000, 1, 70000, 1.0, 1.0, out.data_ptr(), None) == swe.SWE_EINVAL
    assert f(swe.SWE_F32, buf.data_ptr(), 4, 4, 3, 1.0, 1.0, out.data_ptr(), None) == swe.SWE_EINVAL
    assert f(swe.SWE_F32, ctypes.c_void_p(0), 4, 4, 4, 1.0, 1.0, out.data_ptr(), None) == swe.SWE_EINVAL
    assert f(7, buf.data_ptr(), 4, 4, 4, 1.0, 1.0, out.data_ptr(), None) == swe.SWE_EINVAL
