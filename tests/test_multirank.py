"""Multi-process logic on the CPU (gloo): the replicas of bench.py meet only
in their timings (a max over ranks); a grid decomposed across ranks
exchanges one-cell halo strips with its neighbours and gives the
single-domain result bit for bit."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r's job took (1 + r) s, steps (0.5 + r) s, e2e (2 + 3 r) s
        t = bench.aggregate_over_ranks([1.0 + rank, 0.5 + rank, 2.0 + 3 * rank], world)
        out[rank] = (t, bench.whole_job_rate(world, 1000, 10, t[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        t, rate = out[r]
        assert t == [2.0, 1.5, 5.0]
        assert rate == pytest.approx(2 * 1000 * 10 / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks([3.0, 1.0], 1) == [3.0, 1.0]
    assert bench.whole_job_rate(1, 100, 4, 2.0) == 200.0


def _halo_rank(rank, world, port, px, py, nx, ny, steps, out):
    """One partition per rank: exchange the ghost strips that face other
    ranks over gloo, fill the wall ghosts with the oracle's reflective rule,
    then one oracle step (FP64) on the ghosted arrays, ``steps`` times; the
    interior goes back to the parent."""
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import swe_inputs as si
    from paper_1107_2157_gb300 import partition as P
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = si.smooth_flow_state(3, nx, ny)
        dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, 9.8, 0.3)
        a, b = P.coords(rank, px)
        x0, x1 = P.bounds(nx, px, a)
        y0, y1 = P.bounds(ny, py, b)
        fields = []
        for full in (s.h, s.hu, s.hv):
            F = torch.zeros((y1 - y0 + 2, x1 - x0 + 2), dtype=torch.float64)
            F[1:-1, 1:-1] = torch.from_numpy(np.ascontiguousarray(full[y0:y1, x0:x1]))
            fields.append(F)
        walls = P.wall_mask(rank, px, py)
        for _ in range(steps):
            P.exchange_halo(fields, rank, px, py)
            arrs = [np.ascontiguousarray(F.numpy()) for F in fields]
            oracle.fill_halo(*arrs, walls=walls)
            (oH, oU, oV), _, _ = oracle.step_padded(*arrs, 1.0, 1.0, dt, 9.8)
            fields = [torch.from_numpy(x) for x in (oH, oU, oV)]
        out[rank] = [F[1:-1, 1:-1].numpy().copy() for F in fields]
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 2), (3, 1), (1, 3)])
def test_gloo_ranks_with_halo_exchange_equal_the_single_domain_bitwise(px, py):
    """Partitions on separate processes, ghost strips exchanged with
    torch.distributed (gloo) in the library's strip layout, each stepped by
    the FP64 oracle: the gathered state equals the oracle on the whole grid
    bit for bit, walls included.  (tests/test_gpu_multirank.py runs the same
    exchange around the library's CUDA step.)"""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    import swe_inputs as si
    from paper_1107_2157_gb300 import partition as P
    nx, ny, steps, world = 37, 23, 6, px * py
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_halo_rank, args=(r, world, port, px, py, nx, ny, steps, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs)
    s = si.smooth_flow_state(3, nx, ny)
    dt = oracle.cfl_dt(s.h, s.hu, s.hv, 1.0, 1.0, 9.8, 0.3)
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, dt, 9.8, steps)
    got = [np.zeros((ny, nx)) for _ in range(3)]
    for r in range(world):
        a, b = P.coords(r, px)
        x0, x1 = P.bounds(nx, px, a)
        y0, y1 = P.bounds(ny, py, b)
        for k in range(3):
            got[k][y0:y1, x0:x1] = out[r][k]
    for k in range(3):
        assert np.array_equal(got[k], ref[k]), k


def test_partition_layout_covers_the_grid_once():
    sys.path.insert(0, ROOT)
    from paper_1107_2157_gb300 import partition as P
    for n, p in ((37, 3), (8, 8), (1000, 7)):
        spans = [P.bounds(n, p, a) for a in range(p)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(spans[i][1] == spans[i + 1][0] and spans[i][1] > spans[i][0] for i in range(p - 1))
    nb = P.neighbours(4, 3, 3)  # the centre of a 3 x 3 layout
    assert nb == {P.LEFT: 3, P.RIGHT: 5, P.BOTTOM: 1, P.TOP: 7}
    assert P.neighbours(0, 3, 3) == {P.LEFT: None, P.RIGHT: 1, P.BOTTOM: None, P.TOP: 3}
    assert P.wall_mask(4, 3, 3) == 0 and P.wall_mask(0, 3, 3) == 1 | 4 and P.wall_mask(0, 1, 1) == 15
    # strips tile the buffer of 6 (nx + ny) floats in the order left, right, bottom, top
    sl = [P.strip_slice(s, 7, 5) for s in P.SIDES]
    assert [(x.start, x.stop) for x in sl] == [(0, 15), (15, 30), (30, 51), (51, 72)]
