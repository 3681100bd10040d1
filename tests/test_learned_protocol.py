"""The fused learned step's synchronisation (swe_learned.cu), checked on
the CPU over every interleaving of its agents (tests/learned_protocol.py):
no ring row is overwritten before its MMA has read it, no epilogue reads an
accumulator block before its MMAs have run or misses a re-arm, no barrier
wait is ambiguous in parity, and nothing deadlocks -- for instances of 1 to
9 rows (the first and last rows of a sweep, where the pipeline's stages
overlap, and steady-state ticks) over two sweeps.  Each planted change to
the protocol (a missing wait or arrival) is caught."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import learned_protocol as lp  # noqa: E402


@pytest.mark.parametrize("H", [1, 2, 3, 4, 5, 6, 7, 9])
def test_every_interleaving_is_hazard_free(H):
    assert lp.explore(H, 2) > 0


@pytest.mark.parametrize("mutate", ["g0_no_l1_wait", "g1_no_l2_wait", "mma_no_rdy2_wait", "g0_no_rdy3"])
def test_a_broken_protocol_is_caught(mutate):
    with pytest.raises(lp.Violation):
        lp.explore(3, 2, mutate=mutate)
