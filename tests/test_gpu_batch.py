"""Batched ensembles (one persistent launch over many uneven grids) against
the FP64 oracle and against the single-grid kernel."""
import json

import numpy as np
import pytest

import oracle
import swe_inputs as si
from parity import G, b32_run, f32_bar

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (65, 1000), (3, 7), (1, 1), (257, 129), (128, 32), (300, 77), (1024, 64), (129, 129),
         (40, 513), (777, 211), (96, 96)]


def _states(sizes, seed=5):
    return [si.smooth_flow_state(seed * 1000 + i, nx, ny).rounded_to(np.float32)
            for i, (nx, ny) in enumerate(sizes)]


def _dts(states, dxs, dys):
    return np.array([oracle.cfl_dt(s.h, s.hu, s.hv, dx, dy, G, 0.3) for s, dx, dy in zip(states, dxs, dys)])


def _make_batch(sizes, states, dxs, dys, dts):
    from paper_1107_2157_gb300 import Batch
    b = Batch(sizes, dxs, dys, dts, G)
    for i, s in enumerate(states):
        b.set_state(i, *(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
    return b


def test_batch_matches_oracle_per_instance():
    states = _states(SIZES)
    dxs = np.linspace(0.7, 1.3, len(SIZES))
    dys = np.linspace(1.2, 0.8, len(SIZES))
    dts = _dts(states, dxs, dys)
    steps = 20
    with _make_batch(SIZES, states, dxs, dys, dts) as b:
        b.step(steps)
        rc, flags = b.status()
        assert rc == 0 and not flags.any()
        for i, s in enumerate(states):
            got = b.get_state(i)
            ref = oracle.run(s.h, s.hu, s.hv, dxs[i], dys[i], dts[i], G, steps)
            ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s, dxs[i], dys[i], dts[i], G, steps))
            assert ok, (i, SIZES[i], errs, errs_b32)


def test_every_variant_is_bitwise_equal_to_the_single_grid_kernel():
    """Each cell's update is a fixed function of its neighbours, so the tile
    shape, staging depth and CTA count cannot change a bit."""
    from paper_1107_2157_gb300 import Grid, swe
    sizes = SIZES[:8]
    states = _states(sizes, seed=6)
    dxs, dys = np.ones(len(sizes)), np.ones(len(sizes))
    dts = _dts(states, dxs, dys)
    steps = 15  # odd: ends in the other buffer
    refs = []
    for i, s in enumerate(states):
        with Grid(sizes[i][0], sizes[i][1], 1.0, 1.0, dts[i], G, dtype="f32") as g:
            g.set_state(*(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
            g.step(steps)
            refs.append(g.get_state())
    with _make_batch(sizes, states, dxs, dys, dts) as b:
        nvar = b.query(swe.SWE_BQ_VARIANT_COUNT)
        for v in range(nvar):
            for cps in (1, 2):
                b.configure(v, cps)
                for i, s in enumerate(states):
                    b.set_state(i, *(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
                b.step(steps)
                rc, flags = b.status()
                assert rc == 0 and not flags.any()
                for i in range(len(sizes)):
                    got = b.get_state(i)
                    for k in range(3):
                        assert np.array_equal(got[k], refs[i][k]), (v, cps, i, k)


def test_batch_reductions_match_oracle():
    states = _states(SIZES, seed=8)
    dxs = np.linspace(0.5, 1.5, len(SIZES))
    dys = np.linspace(1.1, 0.9, len(SIZES))
    with _make_batch(SIZES, states, dxs, dys, np.full(len(SIZES), 0.01)) as b:
        m = b.mass()
        d = b.cfl_dt(0.2)
    for i, s in enumerate(states):
        mr = oracle.mass(s.h, dxs[i], dys[i])
        assert abs(m[i] - mr) <= 1e-14 * mr
        assert d[i] == oracle.cfl_dt(s.h, s.hu, s.hv, dxs[i], dys[i], G, 0.2)


def test_nonpositive_depth_is_flagged_for_that_instance_only():
    sizes = [(64, 48), (50, 50), (70, 30)]
    states = _states(sizes, seed=9)
    # instance 1: a nearly dry region drained by a strong outflow
    s1 = states[1]
    s1.h[:, :25] = 1e-3
    s1.hu[:, 20:25] = 2.0
    dts = np.array([0.01, 0.05, 0.01])
    with _make_batch(sizes, states, np.ones(3), np.ones(3), dts) as b:
        b.step(3)
        rc, flags = b.status()
    assert rc == 0
    assert flags[1] & 1 and not flags[0] and not flags[2]


def test_tuner_picks_a_variant_and_caches_it(tmp_path):
    from paper_1107_2157_gb300 import swe
    sizes = SIZES
    states = _states(sizes, seed=10)
    dxs, dys = np.ones(len(sizes)), np.ones(len(sizes))
    dts = _dts(states, dxs, dys)
    cache = str(tmp_path / "tune.jsonl")
    with _make_batch(sizes, states, dxs, dys, dts) as b:
        nvar = b.query(swe.SWE_BQ_VARIANT_COUNT)
        before = [b.get_state(i) for i in range(len(sizes))]
        b.tune(cache)
        assert b.query(swe.SWE_BQ_TUNED) == 1
        # the state is restored after the trials
        for i in range(len(sizes)):
            after = b.get_state(i)
            assert all(np.array_equal(a, c) for a, c in zip(after, before[i]))
    lines = [json.loads(x) for x in open(cache)]
    winners = [ln for ln in lines if "variant" in ln]
    trials = [ln for ln in lines if "trials" in ln]
    assert len(winners) == 1 and winners[0]["ctas_per_sm"] >= 1
    # every variant (both temporal-blocking depths) was timed
    assert len(trials) == 1
    assert {t["v"] for t in trials[0]["trials"]} == set(range(nvar))
    assert {t["depth"] for t in trials[0]["trials"]} == {1, 2}
    best = min(trials[0]["trials"], key=lambda t: t["ms"])
    assert (best["v"], best["cps"]) == (winners[0]["variant"], winners[0]["ctas_per_sm"])
    with _make_batch(sizes, states, dxs, dys, dts) as b2:
        b2.tune(cache)
        assert b2.query(swe.SWE_BQ_TUNED) == 2
        assert b2.query(swe.SWE_BQ_VARIANT) == winners[0]["variant"]
        assert b2.query(swe.SWE_BQ_DEPTH) == best["depth"]


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_give_up_and_report(which):
    """A wait on a barrier that nothing completes returns SWE_ETIMEOUT after
    its limit instead of hanging; the context stays usable afterwards."""
    import torch
    from paper_1107_2157_gb300 import swe
    rc = swe.lib().swe_selftest_wait(which, 2.0, None)
    assert rc == swe.SWE_ETIMEOUT
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0


def test_graph_replay_is_used_and_repeatable():
    from paper_1107_2157_gb300 import swe
    sizes = SIZES[:5]
    states = _states(sizes, seed=11)
    dxs, dys = np.ones(len(sizes)), np.ones(len(sizes))
    dts = _dts(states, dxs, dys)
    with _make_batch(sizes, states, dxs, dys, dts) as b:
        b.step(4)
        b.step(4)  # replays the captured graph
        a = [b.get_state(i) for i in range(len(sizes))]
        graph = b.query(swe.SWE_BQ_GRAPH)
    with _make_batch(sizes, states, dxs, dys, dts) as b:
        b.step(8)
        c = [b.get_state(i) for i in range(len(sizes))]
    for i in range(len(sizes)):
        assert all(np.array_equal(x, y) for x, y in zip(a[i], c[i]))
    print("graph capture in use:", graph)


def test_narrow_last_column_strips_equal_the_naive_kernel():
    """Instances whose last 128-wide column strip holds 1, 32, 33, 64 or 65
    cells (half- and quarter-warp tiles) and whose last tile row is short:
    every variant gives the bits of the naive single-grid kernel."""
    from paper_1107_2157_gb300 import Grid, swe
    sizes = [(129, 45), (160, 33), (161, 70), (192, 17), (193, 100), (32, 31), (33, 9), (64, 65), (65, 130)]
    states = _states(sizes, seed=11)
    dxs, dys = np.ones(len(sizes)), np.ones(len(sizes))
    dts = _dts(states, dxs, dys)
    steps = 9
    refs = []
    for i, s in enumerate(states):
        with Grid(sizes[i][0], sizes[i][1], 1.0, 1.0, dts[i], G, dtype="f32", kernel=swe.SWE_KERNEL_NAIVE) as g:
            g.set_state(*(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
            g.step(steps)
            refs.append(g.get_state())
    with _make_batch(sizes, states, dxs, dys, dts) as b:
        for v in range(b.query(swe.SWE_BQ_VARIANT_COUNT)):
            b.configure(v, 2)
            for i, s in enumerate(states):
                b.set_state(i, *(a.astype(np.float32) for a in (s.h, s.hu, s.hv)))
            b.step(steps)
            rc, flags = b.status()
            assert rc == 0 and not flags.any()
            for i in range(len(sizes)):
                got = b.get_state(i)
                for k in range(3):
                    assert np.array_equal(got[k], refs[i][k]), (v, sizes[i], k)
