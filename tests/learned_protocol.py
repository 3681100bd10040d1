"""A model of the synchronisation of the fused learned step
(learned_step_kernel in paper_1107_2157_gb300/csrc/swe_learned.cu), explored
over every interleaving.

Agents, each running the kernel's per-tick program in order:
  G0   compute group 0: the Lax-Wendroff row (network input x0), its share
       of layer 1's epilogue (E1) and the output stage (E3)
  G1   compute group 1: its share of E1 and all of layer 2's epilogue (E2)
  MMA  the issuing warp: per batch, wait RDY1 -> layer 1's MMAs -> commit L1,
       wait RDY2 -> layer 2 -> commit L2, wait RDY3 -> layer 3 -> commit L3
  PIPE the tensor core: runs the issued MMAs and commits in issue order; a
       commit's barrier completes once every MMA issued before it has run

A group is one agent: its warps run the same program, and a warp's arrival
for batch t+1 always follows its own wait on batch t, so warps of one group
cannot mix phases.  Barriers are modelled as the hardware has them: an
arrive-count barrier completes a phase at its expected count, and a wait
passes when the parity of the current phase differs from the awaited
phase's parity.  State tags say what each resource holds:
  x0[slot], a1[group][slot], a2[slot]   the ring rows (sweep, row) and
                                        whether their MMA has read them
  acc1[group][block], acc2[block], acc3[block]
                                        the TMEM accumulator blocks: the
                                        (sweep, output row) they are armed
                                        for and the MMAs added so far
Checked in every reachable state: a ring row is not overwritten before its
MMA read it, and an MMA reads the row it expects; an MMA adds to a block
armed for its output row; an epilogue reads a block only once all of its
row's MMAs have run; every wait sees its barrier at the awaited phase or
one past it (a parity wait is otherwise ambiguous); no state is stuck
before every agent has finished.
"""
from __future__ import annotations

from collections import deque

N_RDY = {"RDY1": 16, "RDY2": 8, "RDY3": 8}  # warps arriving per phase
BARS = ("RDY1", "RDY2", "RDY3", "L1", "L2", "L3", "FIN")


def programs(H, S, mutate=None):
    """Per-agent op lists for S sweeps (steps) of one H-row instance."""
    T = H + 6
    g0, g1, mma = [], [], []
    nb = 0  # batches of the finished sweeps
    for k in range(S):
        g0.append(("arm", 0, k))
        g1.append(("arm", 1, k))
        for t in range(T):
            pub = t + 1 < T
            if t < H:
                g0.append(("lw", k, t))
            if t >= 1 and mutate != "g0_no_l1_wait":
                g0.append(("wait", "L1", nb + t - 1))
            if 0 <= t - 2 < H:
                g0.append(("e1", 0, k, t - 2))
            if pub:
                g0.append(("arrive", "RDY1", 8))
            if t >= 1:
                g0.append(("wait", "L3", nb + t - 1))
            if 0 <= t - 6 < H:
                g0.append(("e3", k, t - 6))
            if pub and mutate != "g0_no_rdy3":
                g0.append(("arrive", "RDY3", 8))
            if t >= 1:
                g1.append(("wait", "L1", nb + t - 1))
            if 0 <= t - 2 < H:
                g1.append(("e1", 1, k, t - 2))
            if pub:
                g1.append(("arrive", "RDY1", 8))
            if t >= 1 and mutate != "g1_no_l2_wait":
                g1.append(("wait", "L2", nb + t - 1))
            if 0 <= t - 4 < H:
                g1.append(("e2", k, t - 4))
            if pub:
                g1.append(("arrive", "RDY2", 8))
        for t in range(T - 1):
            b = nb + t
            mma.append(("wait", "RDY1", b))
            if t < H:
                mma.append(("issue", ("mma", 1, k, t)))
            mma.append(("issue", ("commit", "L1")))
            if mutate != "mma_no_rdy2_wait":
                mma.append(("wait", "RDY2", b))
            if 0 <= t - 2 < H:
                mma.append(("issue", ("mma", 2, k, t - 2)))
            mma.append(("issue", ("commit", "L2")))
            mma.append(("wait", "RDY3", b))
            if 0 <= t - 4 < H:
                mma.append(("issue", ("mma", 3, k, t - 4)))
            mma.append(("issue", ("commit", "L3")))
        nb += T - 1
    mma.append(("issue", ("commit", "FIN")))
    mma.append(("wait", "FIN", 0))
    return [tuple(g0), tuple(g1), tuple(mma)]


class Violation(AssertionError):
    pass


def _contrib(r, H):
    """MMAs (input rows r-1, r, r+1 inside the grid) that complete output row r."""
    return sum(1 for j in (r - 1, r, r + 1) if 0 <= j < H)


def _write_ring(slot_val, k, r, what):
    if slot_val is not None and not slot_val[2]:
        raise Violation("%s row %s overwritten by sweep %d row %d before its MMA read it" % (what, slot_val[:2], k, r))
    return (k, r, False)


def _read_ring(slot_val, k, r, what):
    if slot_val is None or slot_val[:2] != (k, r) or slot_val[2]:
        raise Violation("MMA expected %s row %s, found %s" % (what, (k, r), slot_val))
    return (k, r, True)


def _add(block, k, o, what):
    if block is None or block[:2] != (k, o):
        raise Violation("MMA adds to %s output row %s, block armed for %s" % (what, (k, o), block))
    return (k, o, block[2] + 1)


def _read_acc(block, k, r, H, what):
    if block is None or block != (k, r, _contrib(r, H)):
        raise Violation("%s reads row %s from block %s (needs %d MMAs)" % (what, (k, r), block, _contrib(r, H)))
    return (k, r + 3, 0)  # re-armed for the row three on


def successors(state, progs, H):
    """(next state) for every enabled step of every agent."""
    pcs, queue, bars, x0, a1, a2, acc1, acc2, acc3 = state
    out = []
    bar_i = {b: i for i, b in enumerate(BARS)}
    for ag in range(3):
        pc = pcs[ag]
        if pc >= len(progs[ag]):
            continue
        op = progs[ag][pc]
        npcs = pcs[:ag] + (pc + 1,) + pcs[ag + 1:]
        kind = op[0]
        if kind == "wait":
            c, _ = bars[bar_i[op[1]]]
            p = op[2]
            if c not in (p, p + 1):
                raise Violation("agent %d waits for %s phase %d with %d phases complete" % (ag, op[1], p, c))
            if (c & 1) != (p & 1):  # the awaited phase is complete
                out.append((npcs, queue, bars, x0, a1, a2, acc1, acc2, acc3))
        elif kind == "arrive":
            i = bar_i[op[1]]
            c, a = bars[i]
            a += op[2]
            if a > N_RDY[op[1]]:
                raise Violation("%s over-arrived" % op[1])
            if a == N_RDY[op[1]]:
                c, a = c + 1, 0
            nbars = bars[:i] + ((c, a),) + bars[i + 1:]
            out.append((npcs, queue, nbars, x0, a1, a2, acc1, acc2, acc3))
        elif kind == "issue":
            out.append((npcs, queue + (op[1],), bars, x0, a1, a2, acc1, acc2, acc3))
        elif kind == "arm":
            g, k = op[1], op[2]
            fresh = tuple((k, b, 0) for b in range(3))
            nacc1 = tuple(fresh if gg == g else acc1[gg] for gg in range(2))
            if g == 0:
                out.append((npcs, queue, bars, x0, a1, a2, nacc1, acc2, fresh))
            else:
                out.append((npcs, queue, bars, x0, a1, a2, nacc1, fresh, acc3))
        elif kind == "lw":
            k, t = op[1], op[2]
            nx0 = list(x0)
            nx0[t % 2] = _write_ring(x0[t % 2], k, t, "x0")
            out.append((npcs, queue, bars, tuple(nx0), a1, a2, acc1, acc2, acc3))
        elif kind == "e1":
            g, k, r = op[1], op[2], op[3]
            blocks = list(acc1[g])
            blocks[r % 3] = _read_acc(blocks[r % 3], k, r, H, "E1")
            nacc1 = tuple(tuple(blocks) if gg == g else acc1[gg] for gg in range(2))
            ring = list(a1[g])
            ring[r % 2] = _write_ring(ring[r % 2], k, r, "a1")
            na1 = tuple(tuple(ring) if gg == g else a1[gg] for gg in range(2))
            out.append((npcs, queue, bars, x0, na1, a2, nacc1, acc2, acc3))
        elif kind == "e2":
            k, r = op[1], op[2]
            blocks = list(acc2)
            blocks[r % 3] = _read_acc(blocks[r % 3], k, r, H, "E2")
            ring = list(a2)
            ring[r % 2] = _write_ring(ring[r % 2], k, r, "a2")
            out.append((npcs, queue, bars, x0, a1, tuple(ring), acc1, tuple(blocks), acc3))
        elif kind == "e3":
            k, r = op[1], op[2]
            blocks = list(acc3)
            blocks[r % 3] = _read_acc(blocks[r % 3], k, r, H, "E3")
            out.append((npcs, queue, bars, x0, a1, a2, acc1, acc2, tuple(blocks)))
        else:
            raise ValueError(op)
    # the tensor pipe runs the oldest issued operation
    if queue:
        head, rest = queue[0], queue[1:]
        if head[0] == "commit":
            i = bar_i[head[1]]
            c, a = bars[i]
            nbars = bars[:i] + ((c + 1, a),) + bars[i + 1:]
            out.append((pcs, rest, nbars, x0, a1, a2, acc1, acc2, acc3))
        else:
            _, layer, k, j = head
            outs = [o for o in (j + 1, j, j - 1) if o >= 0]
            if layer == 1:
                nx0 = list(x0)
                nx0[j % 2] = _read_ring(x0[j % 2], k, j, "x0")
                nacc1 = []
                for g in range(2):
                    blocks = list(acc1[g])
                    for o in outs:
                        blocks[o % 3] = _add(blocks[o % 3], k, o, "acc1")
                    nacc1.append(tuple(blocks))
                out.append((pcs, rest, bars, tuple(nx0), a1, a2, tuple(nacc1), acc2, acc3))
            elif layer == 2:
                na1 = []
                for g in range(2):
                    ring = list(a1[g])
                    ring[j % 2] = _read_ring(ring[j % 2], k, j, "a1")
                    na1.append(tuple(ring))
                blocks = list(acc2)
                for o in outs:
                    blocks[o % 3] = _add(blocks[o % 3], k, o, "acc2")
                out.append((pcs, rest, bars, x0, tuple(na1), a2, acc1, tuple(blocks), acc3))
            else:
                ring = list(a2)
                ring[j % 2] = _read_ring(ring[j % 2], k, j, "a2")
                blocks = list(acc3)
                for o in outs:
                    blocks[o % 3] = _add(blocks[o % 3], k, o, "acc3")
                out.append((pcs, rest, bars, x0, a1, tuple(ring), acc1, acc2, tuple(blocks)))
    return out


def explore(H, S, mutate=None, limit=5_000_000):
    """Breadth-first search of every interleaving; returns the number of
    states, or raises Violation (a hazard, an ambiguous wait or a stuck
    state)."""
    progs = programs(H, S, mutate)
    empty_acc = (None, None, None)
    start = ((0, 0, 0), (), tuple((0, 0) for _ in BARS), (None, None), ((None, None), (None, None)), (None, None),
             (empty_acc, empty_acc), empty_acc, empty_acc)
    seen = {start}
    todo = deque([start])
    ends = tuple(len(p) for p in progs)
    while todo:
        s = todo.popleft()
        nxt = successors(s, progs, H)
        if not nxt:
            if s[0] != ends or s[1]:
                raise Violation("stuck at program counters %s of %s, %d operations queued" % (s[0], ends, len(s[1])))
            continue
        for n in nxt:
            if n not in seen:
                seen.add(n)
                todo.append(n)
                if len(seen) > limit:
                    raise RuntimeError("state limit")
    return len(seen)
