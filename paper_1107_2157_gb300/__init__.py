"""GB300 (sm_103a) shallow-water Lax-Wendroff library: Python binding.

The compute path is libswe.so (hand-written CUDA behind the C ABI of
include/swe.h); this package only marshals arguments to it.
"""
from .swe import *  # noqa: F401,F403
from .swe import Batch, Grid, Net, Region, SweError, lib  # noqa: F401
