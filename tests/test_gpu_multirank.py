"""A grid decomposed across processes, each rank stepping its partition with
the library's CUDA kernels (swe_part_create_rank: wall ghosts and the TMA
tile step on the GPU) and exchanging the edge strips that face other ranks
over torch.distributed (gloo, through host memory) before every step -- the
layout of Sec. 4.1 and Fig. 1.  The ranks share one GPU here; no kernel
waits on another rank (the exchange is on the host between launches).  The
gathered state equals the single-grid CUDA step bit for bit and the FP64
oracle within the FP32 bar."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

NX, NY, STEPS, DX, DY, G = 300, 97, 11, 0.9, 1.1, 9.8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _state():
    import oracle
    import swe_inputs as si
    s = si.smooth_flow_state(41, NX, NY).rounded_to(np.float32)
    return s, oracle.cfl_dt(s.h, s.hu, s.hv, DX, DY, G, 0.3)


def _gpu_rank(rank, world, port, px, py, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1107_2157_gb300 import Partitioned
    from paper_1107_2157_gb300 import partition as P
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, dt = _state()
        a, b = P.coords(rank, px)
        x0, x1 = P.bounds(NX, px, a)
        y0, y1 = P.bounds(NY, py, b)
        part = Partitioned.rank(x1 - x0, y1 - y0, P.wall_mask(rank, px, py), DX, DY, dt, G)
        try:
            part.set_state(*(np.ascontiguousarray(f[y0:y1, x0:x1], np.float32) for f in (s.h, s.hu, s.hv)))
            n = 6 * (part.nx + part.ny)
            edges = torch.empty(n, dtype=torch.float32, device="cuda")
            ghosts = torch.zeros(n, dtype=torch.float32, device="cuda")
            for _ in range(STEPS):
                P.exchange_ghosts(part, rank, px, py, edges, ghosts)
                part.step(1)
            out[rank] = part.get_state()
            out["launches%d" % rank] = part.query(2)
        finally:
            part.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2)])
def test_ranks_stepping_on_the_gpu_equal_the_single_grid_bitwise(px, py):
    from paper_1107_2157_gb300 import partition as P
    from parity import b32_run, f32_bar, run_gpu
    import oracle
    world = px * py
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, world, port, px, py, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = [np.zeros((NY, NX), np.float32) for _ in range(3)]
    for r in range(world):
        a, b = P.coords(r, px)
        x0, x1 = P.bounds(NX, px, a)
        y0, y1 = P.bounds(NY, py, b)
        for k in range(3):
            got[k][y0:y1, x0:x1] = out[r][k]
        assert out["launches%d" % r] == 2 * STEPS
    s, dt = _state()
    single = run_gpu(s, DX, DY, dt, G, STEPS, "f32", 2)
    for k in range(3):
        assert np.array_equal(got[k], single[k]), k
    ref = oracle.run(s.h, s.hu, s.hv, DX, DY, dt, G, STEPS)
    ok, errs, errs_b32 = f32_bar(got, ref, b32_run(s, DX, DY, dt, G, STEPS))
    assert ok, (errs, errs_b32)


def test_rank_partition_arguments_are_checked():
    import torch
    from paper_1107_2157_gb300 import Partitioned, swe
    with pytest.raises(swe.SweError) as e:
        Partitioned.rank(10, 10, 16, 1.0, 1.0, 0.01, G)
    assert e.value.status == swe.SWE_EINVAL
    part = Partitioned.rank(10, 7, 15, 1.0, 1.0, 0.01, G)
    try:
        with pytest.raises(ValueError):
            part.edges(torch.empty(5, dtype=torch.float32, device="cuda"))
        buf = torch.zeros(6 * 17, dtype=torch.float32, device="cuda")
        with pytest.raises(swe.SweError):
            part.set_ghosts(buf, 16)
    finally:
        part.close()
    many = Partitioned(20, 20, 2, 1, 1.0, 1.0, 0.01, G)
    try:
        with pytest.raises(swe.SweError):
            many.edges(torch.zeros(6 * 40, dtype=torch.float32, device="cuda"))
    finally:
        many.close()
