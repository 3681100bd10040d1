"""Partitions of one grid across ranks, and the halo exchange between
neighbouring partitions over torch.distributed (NCCL between GPUs, gloo
between CPU processes): the host side of a decomposed multi-GPU run.

Sec. 4.1 (with Fig. 1) lays out the global array in MPI partitions, each
with its halo; this module is that layout for the two-step Lax-Wendroff
stencil (Sec. 3), whose halo is one cell wide.  The library's swe_part_*
functions hold all partitions of a grid on one device and exchange halos
with a kernel; a rank of a multi-process run holds one partition and calls
``exchange_halo`` before each step.

Layout: px x py partitions, rank r at (a, b) = (r % px, r // px); partition
(a, b) holds columns [a nx // px, (a+1) nx // px) and rows
[b ny // py, (b+1) ny // py) -- the split swe_part_create uses.  Its arrays
are (rows + 2) x (cols + 2) with a one-cell ghost ring; ghosts next to
another partition receive that partition's edge cells, ghosts on the grid
boundary are the reflective mirror of their own edge cell (h and the
tangential momentum copied, the normal momentum negated).  Corner ghosts
are never read by the stencil and are left alone.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

LEFT, RIGHT, BOTTOM, TOP = "left", "right", "bottom", "top"
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


def exchange_halo(fields: List, rank: int, px: int, py: int, group=None) -> None:
    """Fills the ghost ring of this rank's (H, U, V) -- torch tensors of
    (rows + 2) x (cols + 2) on the rank's device -- from the neighbouring
    ranks' edge cells, and on the grid boundary with the reflective mirror.
    Every rank of the group calls it at the same step."""
    import torch
    import torch.distributed as dist
    H, U, V = fields
    nb = neighbours(rank, px, py)
    reqs, recvs = [], []
    for side, other in nb.items():
        if other is None:
            continue
        send = torch.stack([_edge(F, side) for F in (H, U, V)]).contiguous()
        recv = torch.empty_like(send)
        reqs.append(dist.isend(send, other, group=group))
        reqs.append(dist.irecv(recv, other, group=group))
        recvs.append((side, recv, send))
    for side, other in nb.items():
        if other is not None:
            continue
        normal = U if side in (LEFT, RIGHT) else V
        for F in (H, U, V):
            g = _ghost(F, side)
            g.copy_(-_edge(F, side) if F is normal else _edge(F, side))
    for r in reqs:
        r.wait()
    for side, recv, _ in recvs:
        for k, F in enumerate((H, U, V)):
            _ghost(F, side).copy_(recv[k])
