"""One grid split into px x py ghosted partitions on one device (swe_part_*:
halo kernel + step kernel) against the single-grid kernel (bitwise) and the
FP64 oracle."""
import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import G, b32_run, f32_bar, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("px,py", [(1, 1), (2, 2), (3, 5), (7, 1), (1, 4), (300, 1)])
def test_partitioned_equals_single_grid_bitwise(px, py):
    from paper_1107_2157_gb300 import Partitioned, swe
    nx, ny, steps = 300, 97, 11
    s = si.smooth_flow_state(41, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 0.9, 1.1, G, 0.3)
    ref = run_gpu(s, 0.9, 1.1, dt, G, steps, "f32", 2)
    with Partitioned(nx, ny, px, py, 0.9, 1.1, dt, G) as p:
        p.set_state(*(np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)))
        p.step(steps)
        got = p.get_state()
        assert p.query(swe.SWE_PQ_PARTS) == px * py
        xs = [a * nx // px for a in range(px + 1)]
        ys = [b * ny // py for b in range(py + 1)]
        halo = sum(2 * (xs[a + 1] - xs[a]) + 2 * (ys[b + 1] - ys[b]) for a in range(px) for b in range(py))
        assert p.query(swe.SWE_PQ_HALO_CELLS) == halo
        assert p.query(swe.SWE_PQ_LAUNCHES) == 2 * steps
    for k in range(3):
        assert np.array_equal(got[k], ref[k]), k


def test_partitioned_matches_oracle():
    from paper_1107_2157_gb300 import Partitioned
    nx, ny, steps = 129, 64, 40
    s = si.smooth_flow_state(42, nx, ny).rounded_to(np.float32)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, G, 0.3)
    with Partitioned(nx, ny, 4, 3, 1.0, 1.0, dt, G) as p:
        p.set_state(*(np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)))
        p.step(steps)
        got = p.get_state()
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, G, steps)
    ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s, 1.0, 1.0, dt, G, steps))
    assert ok, (errs, errs_b32)


def test_partition_arguments_are_checked():
    from paper_1107_2157_gb300 import Partitioned, swe
    for args in ((10, 10, 11, 1), (10, 10, 1, 0), (0, 10, 1, 1)):
        with pytest.raises(swe.SweError) as e:
            Partitioned(*args, 1.0, 1.0, 0.01, G)
        assert e.value.status == swe.SWE_EINVAL
