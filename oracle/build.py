"""Build the oracle's C library (test infrastructure; see oracle/__init__.py).

The oracle is compiled with -ffp-contract=off so that each floating-point
operation is one IEEE operation (FP64, or binary32 in swe_oracle_f32.c) in
source order.  OpenMP is used only to
spread the row loops of the step over host threads; it does not change any
result (no reductions run in parallel).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "swe_oracle.c")
SRCS = [SRC, os.path.join(HERE, "swe_oracle_f32.c"), os.path.join(HERE, "swe_oracle_bathy.c")]
LIB = os.path.join(HERE, "_swe_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the oracle's C sources into oracle/_swe_oracle.so if out of date."""
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS)
            and os.path.getmtime(LIB) >= os.path.getmtime(__file__)):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
            "-fPIC", "-shared"] + SRCS + ["-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
