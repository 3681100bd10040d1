"""Parity at the full workload sizes, in the launch configurations bench.py
times: the 512-grid ensemble (tuned persistent launch, 500 steps) and the
fused learned serving (1024 instances of 256^2 in one launch), on sampled
instances the oracle computes one by one."""
import numpy as np
import pytest

import oracle
import swe_inputs as si
from oracle import learned, nn
from parity import G, b32_run, f32_bar

pytestmark = pytest.mark.gpu


def test_ensemble_512_full_size_sampled_instances():
    from paper_1107_2157_gb300 import Batch
    sizes = si.ensemble_sizes(seed=2, count=512)
    steps = 500
    b = Batch(sizes, 1.0, 1.0, 0.01, G)
    try:
        for i, (nx, ny) in enumerate(sizes):
            st = si.ensemble_state(2, i, nx, ny)
            b.set_state(i, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)))
        dts = b.cfl_dt(0.2)
        b.set_dt(dts)
        b.tune()
        b.step(steps)
        rc, flags = b.status()
        assert rc == 0 and not flags.any()
        areas = [nx * ny for nx, ny in sizes]
        rng = np.random.default_rng(0)
        sample = sorted({int(np.argmax(areas)), int(np.argmin(areas))} |
                        set(int(i) for i in rng.choice(len(sizes), 6, replace=False)))
        for i in sample:
            nx, ny = sizes[i]
            st = si.ensemble_state(2, i, nx, ny).rounded_to(np.float32)
            dt = oracle.cfl_dt(st.h, st.hu, st.hv, 1.0, 1.0, G, 0.2)
            assert dt == dts[i]
            ref = oracle.run(st.h, st.hu, st.hv, 1.0, 1.0, dt, G, steps)
            ok, errs, errs_b32 = f32_bar(b.get_state(i), ref, b32_run(st, 1.0, 1.0, dt, G, steps))
            assert ok, (i, sizes[i], errs, errs_b32)
    finally:
        b.close()


NORM = (0.0, 5e-4, 1.4e-3, 1.2e-5, 3e-5)


def _serving_batch(n, N, seed0):
    from paper_1107_2157_gb300 import Batch
    b = Batch([(N, N)] * n, 4.0, 4.0, 0.16, 9.8)
    for i in range(n):
        st = si.corrector_training_state(seed0 + i, N)
        b.set_state(i, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)))
    return b


def test_learned_serving_full_size():
    """1024 instances of 256^2: one fused step against the oracle on
    sampled instances; then 63 steps in one launch equal 63 one-step
    launches bit for bit (the pending mass offset carried inside a launch
    and settled between launches give the same state), keep the mass and
    raise no flag."""
    from paper_1107_2157_gb300 import Net, swe
    n, N = 1024, 256
    params = nn.init_params(11, out_scale=1.0)
    net = Net(1, 8, 8)
    net.set_params(swe.flatten_params(params))
    net.set_norm(*NORM)
    a = _serving_batch(n, N, 10000)
    c = _serving_batch(n, N, 10000)
    try:
        m0 = a.mass()
        a.learned_step(net, 1)
        po = {k: (learned.bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
              for k, v in params.items()}
        for i in (0, 517, 1023):
            st = si.corrector_training_state(10000 + i, N).rounded_to(np.float32)
            (rh, ru, rv), d = learned.corrected_step(st.h, st.hu, st.hv, 4.0, 4.0, 0.16, 9.8, po, NORM)
            plain = oracle.run(st.h, st.hu, st.hv, 4.0, 4.0, 0.16, 9.8, 1)
            got = a.get_state(i)
            for k, ref in enumerate((rh, ru, rv)):
                dg = got[k].astype(np.float64) - plain[k]
                assert np.linalg.norm(dg - d[k]) <= 2e-2 * np.linalg.norm(d[k]) + 1e-6 * np.linalg.norm(plain[k]), (i, k)
        a.learned_step(net, 63)
        c.learned_step(net, 1)
        for _ in range(63):
            c.learned_step(net, 1)
        rc, flags = a.status()
        assert rc == 0 and not flags.any()
        drift = np.abs(a.mass() - m0) / m0
        assert (drift <= 1e-5).all(), drift.max()
        for i in (0, 100, 517, 1023):
            x, y = a.get_state(i), c.get_state(i)
            for k in range(3):
                assert np.array_equal(x[k], y[k]), (i, k)
    finally:
        a.close()
        c.close()
        net.close()
