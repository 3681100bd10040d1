"""Seeded synthetic initial states for the shallow-water workloads.

This module is shared by the CPU oracle runs and the GPU runs. It only draws
random numbers and evaluates initial conditions; it contains none of the
Lax-Wendroff arithmetic (no fluxes, no face states, no time step).

Conventions (shared by every caller):
  * interior cell (i, j), i = 1..nx (x, fastest in memory), j = 1..ny;
  * arrays returned here are interior-only, shape (ny, nx), float64;
  * cell centres sit at x = (i - 1/2) dx, y = (j - 1/2) dy; bump centres and
    widths are expressed in cell units.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), keyed by (seed, stream), so
that every instance of an ensemble has its own reproducible stream.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class SplitMix64:
    """Counter-based SplitMix64 stream keyed by (seed, stream)."""

    def __init__(self, seed: int, stream: int = 0):
        self.state = _mix((seed * _GOLDEN + 0x632BE59BD9B4E019) & _MASK)
        self.state = (self.state ^ _mix((stream + 1) * 0xD1B54A32D192ED03 & _MASK)) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        return _mix(self.state)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) with 53 random bits."""
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi]."""
        span = hi - lo + 1
        return lo + (self.next_u64() % span)


@dataclasses.dataclass(frozen=True)
class Bump:
    """Gaussian bump amp * exp(-r^2 / (2 sigma^2)), centre/sigma in cells."""

    cx: float
    cy: float
    amp: float
    sigma: float


# A bump contributes only within this many sigmas of its centre (exp(-72) is
# below 1e-31, far under FP64 resolution of the base depth).
BUMP_CUTOFF_SIGMAS = 12.0


def bumps_h(nx: int, ny: int, base: float, bumps: Sequence[Bump],
            window: Tuple[int, int, int, int] | None = None) -> np.ndarray:
    """Depth field base + sum of separable Gaussian bumps.

    ``window = (i0, i1, j0, j1)`` (1-based, inclusive) evaluates only that
    sub-rectangle; every element gets bitwise the same value it has in the full
    field, so a window can stand in for the full grid.  Indices outside
    1..nx / 1..ny are allowed (they are evaluated by the same formula).
    """
    if window is None:
        window = (1, nx, 1, ny)
    i0, i1, j0, j1 = window
    h = np.full((j1 - j0 + 1, i1 - i0 + 1), float(base), dtype=np.float64)
    for b in bumps:
        reach = BUMP_CUTOFF_SIGMAS * b.sigma
        # bump box in 1-based cell indices (independent of the window)
        bi0 = max(int(math.floor(b.cx + 0.5 - reach)), -(1 << 30))
        bi1 = int(math.ceil(b.cx + 0.5 + reach))
        bj0 = int(math.floor(b.cy + 0.5 - reach))
        bj1 = int(math.ceil(b.cy + 0.5 + reach))
        wi0, wi1 = max(bi0, i0), min(bi1, i1)
        wj0, wj1 = max(bj0, j0), min(bj1, j1)
        if wi0 > wi1 or wj0 > wj1:
            continue
        xi = np.arange(wi0, wi1 + 1, dtype=np.float64) - 0.5 - b.cx
        yj = np.arange(wj0, wj1 + 1, dtype=np.float64) - 0.5 - b.cy
        inv2s2 = 1.0 / (2.0 * b.sigma * b.sigma)
        ex = np.exp(-(xi * xi) * inv2s2)
        ey = np.exp(-(yj * yj) * inv2s2)
        h[wj0 - j0:wj1 - j0 + 1, wi0 - i0:wi1 - i0 + 1] += b.amp * np.outer(ey, ex)
    return h


@dataclasses.dataclass
class State:
    """Interior-only initial state (h, hu, hv), each (ny, nx) float64."""

    h: np.ndarray
    hu: np.ndarray
    hv: np.ndarray

    @property
    def nx(self) -> int:
        return self.h.shape[1]

    @property
    def ny(self) -> int:
        return self.h.shape[0]

    def astype(self, dtype) -> "State":
        return State(self.h.astype(dtype), self.hu.astype(dtype), self.hv.astype(dtype))

    def rounded_to(self, dtype) -> "State":
        """Values rounded to ``dtype`` and returned as float64 (what an
        FP32 device buffer holds after upload, seen exactly in FP64)."""
        return State(*(np.asarray(a, dtype=dtype).astype(np.float64)
                       for a in (self.h, self.hu, self.hv)))


def _at_rest(h: np.ndarray) -> State:
    return State(h, np.zeros_like(h), np.zeros_like(h))


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

def single_bump_state(seed: int, n: int = 128, base: float = 2.0, amp: float = 0.5,
                      sigma: float = 8.0, max_offset: float = 16.0,
                      centred: bool = False) -> State:
    """128x128 workload: one bump of width 8 cells, centre offset U[-16,16]^2."""
    rng = SplitMix64(seed, 0)
    ox = 0.0 if centred else rng.uniform(-max_offset, max_offset)
    oy = 0.0 if centred else rng.uniform(-max_offset, max_offset)
    b = Bump(cx=n / 2.0 + ox, cy=n / 2.0 + oy, amp=amp, sigma=sigma)
    return _at_rest(bumps_h(n, n, base, [b]))


def multi_bumps(seed: int, stream: int, nx: int, ny: int, count: int,
                amp_range=(0.05, 0.5), sigma_range=(8.0, 64.0)) -> List[Bump]:
    """``count`` bumps with centres uniform over the domain."""
    rng = SplitMix64(seed, stream)
    out = []
    for _ in range(count):
        cx = rng.uniform(0.0, float(nx))
        cy = rng.uniform(0.0, float(ny))
        amp = rng.uniform(*amp_range)
        sig = rng.uniform(*sigma_range)
        out.append(Bump(cx, cy, amp, sig))
    return out


def large_grid_bumps(seed: int = 1, n: int = 8192, count: int = 64) -> List[Bump]:
    """8192x8192 workload: h = 1 + 64 bumps, amp U[0.05,0.5], sigma U[8,64]."""
    return multi_bumps(seed, 0, n, n, count)


def large_grid_state(seed: int = 1, n: int = 8192, count: int = 64,
                     window=None) -> State:
    h = bumps_h(n, n, 1.0, large_grid_bumps(seed, n, count), window)
    return _at_rest(h)


def large_grid_bed(seed: int = 2, n: int = 8192, count: int = 32, window=None) -> np.ndarray:
    """Bed elevation of the topography workload: 32 Gaussian mounds on a zero
    base, amp U[0.02, 0.2], sigma U[16, 128] (well below the still-water
    surface at 1)."""
    bumps = multi_bumps(seed, 0xBED, n, n, count, amp_range=(0.02, 0.2), sigma_range=(16.0, 128.0))
    return bumps_h(n, n, 0.0, bumps, window)


def large_grid_bed_state(seed: int = 1, bed_seed: int = 2, n: int = 8192, window=None) -> State:
    """The default workload's surface (1 + 64 bumps) over the bed of
    ``large_grid_bed``: depth = surface - bed, at rest."""
    surface = bumps_h(n, n, 1.0, large_grid_bumps(seed, n), window)
    return _at_rest(surface - large_grid_bed(bed_seed, n, window=window))


def ensemble_sizes(seed: int = 2, count: int = 512, lo: int = 64, hi: int = 1024):
    """Instance sizes (nx, ny), each uniform over the integers [lo, hi]."""
    rng = SplitMix64(seed, 0xE5E)
    return [(rng.integer(lo, hi), rng.integer(lo, hi)) for _ in range(count)]


def ensemble_bumps(seed: int, instance: int, nx: int, ny: int, count: int = 4) -> List[Bump]:
    """Per-instance bumps: sigma U[8, min(64, min(nx,ny)/8)]."""
    smax = min(64.0, min(nx, ny) / 8.0)
    return multi_bumps(seed, 1000 + instance, nx, ny, count, sigma_range=(8.0, max(8.0, smax)))


def ensemble_state(seed: int, instance: int, nx: int, ny: int) -> State:
    return _at_rest(bumps_h(nx, ny, 1.0, ensemble_bumps(seed, instance, nx, ny)))


def dam_break_state(seed: int, n: int, h_high: float = 2.0, h_low: float = 1.0) -> State:
    """Hard step across a random line: a uniform point and a uniform angle."""
    rng = SplitMix64(seed, 0xDA3)
    px = rng.uniform(0.0, float(n))
    py = rng.uniform(0.0, float(n))
    ang = rng.uniform(0.0, 2.0 * math.pi)
    nxv, nyv = math.cos(ang), math.sin(ang)
    xs = np.arange(1, n + 1, dtype=np.float64) - 0.5 - px
    ys = np.arange(1, n + 1, dtype=np.float64) - 0.5 - py
    side = ys[:, None] * nyv + xs[None, :] * nxv
    h = np.where(side < 0.0, h_high, h_low).astype(np.float64)
    return _at_rest(h)


def corrector_training_state(seed: int, n: int = 1024, dam_fraction: float = 0.1,
                             bump_count: int = 8) -> State:
    """Fine-grid training trajectories: bumps (sigma U[8,64]) or, with
    probability ``dam_fraction`` drawn from the seed, a dam-break step."""
    rng = SplitMix64(seed, 0xC0DE)
    if rng.uniform() < dam_fraction:
        return dam_break_state(seed, n)
    return _at_rest(bumps_h(n, n, 1.0, multi_bumps(seed, 7, n, n, bump_count)))


def smooth_flow_state(seed: int, nx: int, ny: int, amp_u: float = 0.3) -> State:
    """A smooth state with momentum in both directions (nonzero at the walls),
    for edge and ragged-size tests: h = 1.5 + bumps, hu and hv sinusoidal."""
    rng = SplitMix64(seed, 0x5F)
    smax = max(1.5, min(nx, ny) / 4.0)
    bumps = multi_bumps(seed, 0x60, nx, ny, 3, sigma_range=(1.0, smax))
    h = bumps_h(nx, ny, 1.5, bumps)
    x = (np.arange(nx, dtype=np.float64) + 0.5) / nx
    y = (np.arange(ny, dtype=np.float64) + 0.5) / ny
    a, b = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
    hu = amp_u * h * (np.cos(math.pi * a * y)[:, None] * np.cos(0.7 * math.pi * x)[None, :])
    hv = amp_u * h * (np.sin(0.9 * math.pi * y)[:, None] * np.cos(math.pi * b * x)[None, :])
    return State(h, hu, hv)


def corrector_states(seeds, n: int = 1024, dam_fraction: float = 0.1) -> List[State]:
    """Initial fine states of the corrector's training / evaluation
    trajectories (one per seed)."""
    return [corrector_training_state(s, n, dam_fraction) for s in seeds]
