"""The fused learned coarse step (swe_batch_learned_step: Lax-Wendroff step,
corrector network and corrected update in one persistent launch) against
the FP64 oracle of the learned step (oracle/learned.py), against the plain
batched step (zero network: bitwise) and against the unfused GPU path."""
import math

import numpy as np
import pytest

import oracle
import swe_inputs as si
from oracle import learned, nn

pytestmark = pytest.mark.gpu
G = 9.8


def _params_oracle(params):
    """The network's precision: bf16 weights, fp32 biases (as float64)."""
    return {k: (learned.bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
            for k, v in params.items()}


def _states(sizes, seed):
    return [si.smooth_flow_state(seed + i, nx, ny).rounded_to(np.float32) for i, (nx, ny) in enumerate(sizes)]


def _batch(states, dx, dts):
    from paper_1107_2157_gb300 import Batch
    b = Batch([(s.nx, s.ny) for s in states], dx, dx, dts, G)
    for i, s in enumerate(states):
        b.set_state(i, *(np.ascontiguousarray(a, np.float32) for a in (s.h, s.hu, s.hv)))
    return b


def _dts(states, dx):
    return np.array([oracle.cfl_dt(s.h, s.hu, s.hv, dx, dx, G, 0.2) for s in states])


def _norm(states, dx, dts):
    """Input scales from the oracle's plain increments (RMS over instances);
    output scales of the order of a coarse step's truncation error."""
    inc_h, inc_u = [], []
    for s, dt in zip(states, dts):
        lw = oracle.run(s.h, s.hu, s.hv, dx, dx, dt, G, 1)
        inc_h.append(np.sqrt(np.mean((lw[0] - s.h) ** 2)))
        inc_u.append(np.sqrt(np.mean((lw[1] - s.hu) ** 2 + (lw[2] - s.hv) ** 2) / 2))
    sh, su = float(np.median(inc_h)), float(np.median(inc_u))
    return (0.0, sh, su, 0.05 * sh, 0.05 * su)


def _net(params, norm):
    from paper_1107_2157_gb300 import Net, swe
    net = Net(1, 8, 8)  # the fused step does not use the net's image buffers
    net.set_params(swe.flatten_params(params))
    net.set_norm(*norm)
    return net


def _zero_params():
    return {k: np.zeros_like(v) for k, v in nn.init_params(0).items()}


SIZES_WIDE = [(256, 40), (200, 37), (129, 3), (256, 1), (140, 64)]
SIZES_NARROW = [(128, 33), (97, 50), (1, 7), (5, 1), (64, 128)]


@pytest.mark.parametrize("sizes", [SIZES_WIDE, SIZES_NARROW])
@pytest.mark.parametrize("project", [True, False])
def test_zero_network_is_bitwise_the_plain_batched_step(sizes, project):
    states = _states(sizes, 10)
    dts = _dts(states, 1.0)
    with _batch(states, 1.0, dts) as fused, _batch(states, 1.0, dts) as plain:
        net = _net(_zero_params(), (0.0, 1e-3, 1e-3, 1e-2, 1e-2))
        try:
            fused.learned_step(net, 5, project_mass=project)
            plain.step(5)
            rc, flags = fused.status()
            assert rc == 0 and not flags.any()
            for i in range(len(sizes)):
                a, b = fused.get_state(i), plain.get_state(i)
                for k in range(3):
                    assert np.array_equal(a[k], b[k]), (sizes[i], k)
        finally:
            net.close()


def _compare_with_oracle(states, dx, dts, params, norm, n_steps, project=True):
    po = _params_oracle(params)
    with _batch(states, dx, dts) as b:
        net = _net(params, norm)
        try:
            b.learned_step(net, n_steps, project_mass=project)
            rc, flags = b.status()
            assert rc == 0 and not flags.any(), flags
            got = [b.get_state(i) for i in range(len(states))]
        finally:
            net.close()
    worst = []
    for i, s in enumerate(states):
        ref = learned.corrected_run(s.h, s.hu, s.hv, dx, dx, dts[i], G, po, norm, n_steps, project)
        plain = oracle.run(s.h, s.hu, s.hv, dx, dx, dts[i], G, n_steps)
        for k in range(3):
            d_ref = ref[k] - plain[k]                       # the oracle's total correction
            d_gpu = got[i][k].astype(np.float64) - plain[k]
            scale = float(np.max(np.abs(d_ref)))
            assert scale > 0.0
            err = float(np.max(np.abs(d_gpu - d_ref)))
            # bf16 activations (relative 2^-8 per layer) on the correction,
            # plus the FP32 Lax-Wendroff rounding on the state
            bound = 3e-2 * scale + 4e-6 * float(np.max(np.abs(ref[0])))
            assert err <= bound, (s.nx, s.ny, k, err, scale)
            num = float(np.linalg.norm(d_gpu - d_ref))
            worst.append(num / float(np.linalg.norm(d_ref)))
    return worst


@pytest.mark.parametrize("sizes", [SIZES_WIDE, SIZES_NARROW])
def test_one_fused_step_matches_the_oracle(sizes):
    states = _states(sizes, 20)
    dts = _dts(states, 1.0)
    norm = _norm(states, 1.0, dts)
    rel = _compare_with_oracle(states, 1.0, dts, nn.init_params(3, out_scale=1.0), norm, 1)
    assert max(rel) <= 2e-2, rel


def test_three_fused_steps_match_the_oracle_coarse_spacing():
    sizes = [(256, 48), (173, 21)]
    states = _states(sizes, 30)
    dts = _dts(states, 4.0)
    norm = _norm(states, 4.0, dts)
    rel = _compare_with_oracle(states, 4.0, dts, nn.init_params(4, out_scale=1.0), norm, 3)
    assert max(rel) <= 3e-2, rel


def test_fused_agrees_with_the_unfused_path():
    """Same steps as batch step + prep_input(base) + correct per step; the
    FP32 accumulation order inside the network (the fused kernel starts each
    accumulator from the bias and sums by input row) and of the per-image
    h-correction sum differ, so the two agree to the bf16 resolution of the
    network's activations, measured on the correction."""
    import torch
    from paper_1107_2157_gb300 import Net, swe
    n, nx, ny = 3, 200, 96
    states = _states([(nx, ny)] * n, 40)
    dts = np.full(n, min(_dts(states, 4.0)))
    norm = _norm(states, 4.0, dts)
    params = nn.init_params(6, out_scale=1.0)
    K = 4
    with _batch(states, 4.0, dts) as fused, _batch(states, 4.0, dts) as unf, _batch(states, 4.0, dts) as plain:
        plain.step(K)
        net = Net(n, ny, nx)
        try:
            net.set_params(swe.flatten_params(params))
            net.set_norm(*norm)
            fused.learned_step(net, K)
            for _ in range(K):
                c0 = unf.state_ptr(0)[0]
                unf.step(1)
                p0, plane, pitch = unf.state_ptr(0)
                img = (unf.state_ptr(1)[0] - p0) // 4
                net.prep_input(n, p0, img, plane, pitch, base_ptr=c0)
                net.correct(n, p0, img, plane, pitch, project_mass=True)
            torch.cuda.synchronize()
            assert net.check() == 0
            for i in range(n):
                a, b, p = fused.get_state(i), unf.get_state(i), plain.get_state(i)
                for k in range(3):
                    corr = float(np.max(np.abs(b[k].astype(np.float64) - p[k])))
                    diff = float(np.max(np.abs(a[k].astype(np.float64) - b[k])))
                    assert corr > 0.0
                    assert diff <= 2e-2 * corr + 1e-6 * float(np.max(np.abs(b[0]))), (i, k, diff, corr)
        finally:
            net.close()


def test_fused_step_keeps_mass_with_the_projection():
    sizes = [(256, 64), (150, 40)]
    states = _states(sizes, 50)
    dts = _dts(states, 4.0)
    norm = _norm(states, 4.0, dts)
    params = nn.init_params(7, out_scale=1.0)
    drift = {}
    for project in (True, False):
        with _batch(states, 4.0, dts) as b:
            net = _net(params, norm)
            try:
                m0 = b.mass()
                b.learned_step(net, 8, project_mass=project)
                m1 = b.mass()
            finally:
                net.close()
        drift[project] = np.abs(m1 - m0) / m0
    assert (drift[True] <= 2e-6).all(), drift        # FP32 rounding of the stored depth
    assert (drift[False] > 10 * drift[True]).any(), drift


def test_fused_flags_a_nonpositive_depth_for_that_instance_only():
    sizes = [(64, 48), (50, 50), (70, 30)]
    states = _states(sizes, 60)
    s1 = states[1]
    s1.h[:, :25] = 1e-3
    s1.hu[:, 20:25] = 2.0
    dts = np.array([0.01, 0.05, 0.01])
    with _batch(states, 1.0, dts) as b:
        net = _net(_zero_params(), (0.0, 1e-3, 1e-3, 1e-2, 1e-2))
        try:
            b.learned_step(net, 3)
            rc, flags = b.status()
        finally:
            net.close()
    assert rc == 0
    assert flags[1] & 1 and not flags[0] and not flags[2]


def test_fused_rejects_instances_wider_than_256_and_is_one_launch():
    from paper_1107_2157_gb300 import swe
    states = _states([(257, 8), (16, 16)], 70)
    with _batch(states, 1.0, _dts(states, 1.0)) as b:
        net = _net(_zero_params(), (0.0, 1e-3, 1e-3, 1e-2, 1e-2))
        try:
            with pytest.raises(swe.SweError) as e:
                b.learned_step(net, 1)
            assert e.value.status == swe.SWE_EUNSUPPORTED
        finally:
            net.close()
    states = _states([(100, 20)] * 3, 71)
    with _batch(states, 1.0, _dts(states, 1.0)) as b:
        net = _net(_zero_params(), (0.0, 1e-3, 1e-3, 1e-2, 1e-2))
        try:
            before = b.query(swe.SWE_BQ_LAUNCHES)
            b.learned_step(net, 7)
            assert b.query(swe.SWE_BQ_LAUNCHES) == before + 1
        finally:
            net.close()
