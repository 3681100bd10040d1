"""Partitions of one grid across ranks, and the exchange of edge strips
between neighbouring partitions over torch.distributed (NCCL between GPUs,
gloo between CPU processes): the host side of a decomposed multi-GPU run.

Sec. 4.1 (with Fig. 1) lays out the global array in MPI partitions, each
with its halo; this module is that layout for the two-step Lax-Wendroff
stencil (Sec. 3), whose halo is one cell wide.  A rank holds one partition
in a library context (``swe.Partitioned.rank``: swe_part_create_rank),
which fills its wall ghosts and takes the step on the GPU; before each step
``exchange_ghosts`` moves the edge strips that face other ranks.

Layout: px x py partitions, rank r at (a, b) = (r % px, r // px); partition
(a, b) holds columns [a nx // px, (a+1) nx // px) and rows
[b ny // py, (b+1) ny // py) -- the split swe_part_create uses.  A ghost
next to another partition receives that partition's edge cell; a ghost on
the grid boundary is a reflective wall, filled by whoever takes the step.
Corner ghosts are never read by the stencil.

Strip buffer (the library's layout, 6 (nx + ny) floats): the left, right,
bottom and top strips one after another, each holding h, hu, hv along the
side (ny cells for left and right, nx for bottom and top).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

LEFT, RIGHT, BOTTOM, TOP = "left", "right", "bottom", "top"
SIDES = (LEFT, RIGHT, BOTTOM, TOP)
_BIT = {LEFT: 1, RIGHT: 2, BOTTOM: 4, TOP: 8}
_OPPOSITE = {LEFT: RIGHT, RIGHT: LEFT, BOTTOM: TOP, TOP: BOTTOM}


def bounds(n: int, p: int, a: int) -> Tuple[int, int]:
    """[lo, hi) of part a of n cells split p ways."""
    return a * n // p, (a + 1) * n // p


def coords(rank: int, px: int) -> Tuple[int, int]:
    return rank % px, rank // px


def neighbours(rank: int, px: int, py: int) -> Dict[str, Optional[int]]:
    """The rank across each side of this rank's partition (None: the grid boundary)."""
    a, b = coords(rank, px)
    return {LEFT: rank - 1 if a > 0 else None, RIGHT: rank + 1 if a + 1 < px else None,
            BOTTOM: rank - px if b > 0 else None, TOP: rank + px if b + 1 < py else None}


def wall_mask(rank: int, px: int, py: int) -> int:
    """Bitmask (1 left, 2 right, 4 bottom, 8 top) of the sides on the grid boundary."""
    return sum(_BIT[s] for s, other in neighbours(rank, px, py).items() if other is None)


def strip_slice(side: str, nx: int, ny: int) -> slice:
    """Where a side's strip (h, hu, hv) sits in the strip buffer."""
    off = {LEFT: 0, RIGHT: 3 * ny, BOTTOM: 6 * ny, TOP: 6 * ny + 3 * nx}[side]
    return slice(off, off + (3 * ny if side in (LEFT, RIGHT) else 3 * nx))


def _swap_strips(edges, ghosts, rank, px, py, nx, ny, group=None, via_host=False) -> int:
    """Sends this rank's edge strips to the neighbours and receives theirs
    into ``ghosts``; returns the bitmask of the sides received."""
    import torch.distributed as dist
    nb = neighbours(rank, px, py)
    reqs, recvs, mask = [], [], 0
    for side, other in nb.items():
        if other is None:
            continue
        send = edges[strip_slice(side, nx, ny)]
        recv = ghosts[strip_slice(side, nx, ny)]
        if via_host:
            send, recv_h = send.cpu(), recv.new_empty(recv.shape, device="cpu")
        else:
            send, recv_h = send.contiguous(), recv
        reqs.append(dist.isend(send, other, group=group))
        reqs.append(dist.irecv(recv_h, other, group=group))
        recvs.append((recv, recv_h))
        mask |= _BIT[side]
    for r in reqs:
        r.wait()
    for recv, recv_h in recvs:
        if recv_h is not recv:
            recv.copy_(recv_h)
    return mask


def exchange_ghosts(part, rank: int, px: int, py: int, edges, ghosts, group=None, via_host=None) -> None:
    """Before a step of the rank's library partition ``part``: reads its edge
    strips into ``edges``, swaps them with the neighbouring ranks and writes
    the received strips into its ghost ring.  ``edges`` and ``ghosts`` are
    float32 CUDA tensors of 6 (nx + ny) elements.  With gloo (``via_host``,
    the default when the group's backend is gloo) the strips travel through
    host memory.  Every rank of the group calls it at the same step."""
    import torch
    import torch.distributed as dist
    if via_host is None:
        via_host = dist.get_backend(group) == "gloo"
    part.edges(edges)
    if via_host:
        torch.cuda.current_stream().synchronize()
    mask = _swap_strips(edges, ghosts, rank, px, py, part.nx, part.ny, group, via_host)
    if mask:
        part.set_ghosts(ghosts, mask)


def exchange_halo(fields: List, rank: int, px: int, py: int, group=None) -> None:
    """The same exchange for host arrays: fills the ghosts of this rank's
    (H, U, V) -- torch tensors of (rows + 2) x (cols + 2) -- that face
    another rank from that rank's edge cells.  Wall ghosts are left to the
    code that takes the step."""
    import torch
    H, U, V = fields
    ny, nx = H.shape[0] - 2, H.shape[1] - 2
    edges = torch.empty(6 * (nx + ny), dtype=H.dtype)
    ghosts = torch.empty_like(edges)
    for side in SIDES:
        sl = strip_slice(side, nx, ny)
        edges[sl] = torch.cat([_edge(F, side) for F in (H, U, V)])
    mask = _swap_strips(edges, ghosts, rank, px, py, nx, ny, group)
    for side in SIDES:
        if mask & _BIT[side]:
            strip = ghosts[strip_slice(side, nx, ny)].view(3, -1)
            for k, F in enumerate((H, U, V)):
                _ghost(F, side).copy_(strip[k])


def _edge(F, side):
    """This partition's interior cells along ``side`` (a view)."""
    if side == LEFT:
        return F[1:-1, 1]
    if side == RIGHT:
        return F[1:-1, -2]
    if side == BOTTOM:
        return F[1, 1:-1]
    return F[-2, 1:-1]


def _ghost(F, side):
    """The ghost cells along ``side`` (a view)."""
    if side == LEFT:
        return F[1:-1, 0]
    if side == RIGHT:
        return F[1:-1, -1]
    if side == BOTTOM:
        return F[0, 1:-1]
    return F[-1, 1:-1]
