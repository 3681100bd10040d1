"""The multi-GPU path of bench.py runs independent replicas (the grids do
not exchange data); across ranks only the timings meet, as a max.  Checked
here with two gloo ranks on the CPU."""
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
