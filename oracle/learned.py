"""FP64 oracle of the learned coarse step (TEST INFRASTRUCTURE).

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this module; it shares no code with the CUDA library.

One learned coarse step of a state c (no counterpart in the paper; it
corrects the Lax-Wendroff step of Sec. 3):

    l   = LW(c)                                  the oracle's two-step Lax-Wendroff step
    x0  = Q((l_h - c_h)/sh, (l_hu - c_hu)/su, (l_hv - c_hv)/su)
    r   = NN(x0)                                 oracle.nn.forward
    d   = (oh r_h, ou r_hu, ou r_hv)
    d_h = d_h - mean(d_h)                        only with the mass projection
    c'  = l + d

Q rounds to bf16 (nearest even), the precision in which the network reads
its input; the caller passes weights already rounded to the network's
precision.  The scales (h0, sh, su, oh, ou) are the network's normalisation
(h0 is unused: the input is the increment).
"""
from __future__ import annotations

import numpy as np

from . import nn
from . import run as lw_run


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bf16 (ties to even) through float32; float64 out."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def corrected_step(h, hu, hv, dx, dy, dt, g, params, norm, project_mass=True):
    """One learned coarse step of one grid (interior arrays); returns
    (h, hu, hv) in FP64 and the correction d that was added."""
    c = [np.asarray(a, np.float64) for a in (h, hu, hv)]
    lw = lw_run(c[0], c[1], c[2], dx, dy, dt, g, 1)
    _, sh, su, oh, ou = (float(v) for v in norm)
    x0 = np.stack([(lw[0] - c[0]) / sh, (lw[1] - c[1]) / su, (lw[2] - c[2]) / su])[None]
    r, _ = nn.forward(params, bf16_round(x0))
    d = r[0] * np.array([oh, ou, ou])[:, None, None]
    if project_mass:
        d[0] = d[0] - d[0].mean()
    return tuple(lw[k] + d[k] for k in range(3)), d


def corrected_run(h, hu, hv, dx, dy, dt, g, params, norm, n_steps, project_mass=True):
    """n_steps learned coarse steps; returns (h, hu, hv) in FP64."""
    s = tuple(np.asarray(a, np.float64) for a in (h, hu, hv))
    for _ in range(n_steps):
        s, _ = corrected_step(*s, dx, dy, dt, g, params, norm, project_mass)
    return s
