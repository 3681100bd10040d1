"""Closed-form and textbook results that pin the oracle from outside.

Nothing here calls the oracle; each function is an independent statement of
a known result:
  * ``stoker``: the exact 1D wet-wet dam-break solution of the shallow-water
    equations (rarefaction + shock), the standard Riemann solution found in
    LeVeque, "Finite Volume Methods for Hyperbolic Problems" (2002), Ch. 13;
  * ``lw_amplification``: the von Neumann amplification matrix of the
    two-step Lax-Wendroff scheme applied to the linearised 2D equations;
  * ``textbook_lw_1d``: an independent 1D Richtmyer two-step code for the 1D
    shallow-water equations with reflective walls.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Stoker dam break
# ---------------------------------------------------------------------------

def stoker_middle_state(h_l: float, h_r: float, g: float):
    """Middle depth/velocity of the dam break with u_l = u_r = 0.

    Left rarefaction: u_m = 2 (sqrt(g h_l) - sqrt(g h_m)).
    Right shock:      u_m = (h_m - h_r) sqrt(g (h_m + h_r) / (2 h_m h_r)).
    Solved for h_m in (h_r, h_l) by bisection."""
    def f(hm):
        return 2.0 * (math.sqrt(g * h_l) - math.sqrt(g * hm)) - \
            (hm - h_r) * math.sqrt(g * (hm + h_r) / (2.0 * hm * h_r))
    lo, hi = h_r, h_l
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    hm = 0.5 * (lo + hi)
    um = 2.0 * (math.sqrt(g * h_l) - math.sqrt(g * hm))
    return hm, um


def stoker(xi: np.ndarray, h_l: float, h_r: float, g: float):
    """Exact (h, u) at similarity coordinate xi = (x - x_dam) / t."""
    hm, um = stoker_middle_state(h_l, h_r, g)
    cl = math.sqrt(g * h_l)
    cm = math.sqrt(g * hm)
    s = hm * um / (hm - h_r)  # shock speed from mass Rankine-Hugoniot (u_r = 0)
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    left = xi < -cl
    fan = (xi >= -cl) & (xi <= um - cm)
    mid = (xi > um - cm) & (xi < s)
    right = xi >= s
    h[left], u[left] = h_l, 0.0
    h[fan] = (2.0 * cl - xi[fan]) ** 2 / (9.0 * g)
    u[fan] = 2.0 / 3.0 * (xi[fan] + cl)
    h[mid], u[mid] = hm, um
    h[right], u[right] = h_r, 0.0
    return h, u


# ---------------------------------------------------------------------------
# Linear stability (von Neumann) analysis
# ---------------------------------------------------------------------------

def flux_jacobians(H0: float, U0: float, V0: float, g: float):
    """Jacobians A = dF/dq, B = dG/dq of the 2D shallow-water fluxes at the
    state q0 = (h, hu, hv), with u = U0/H0, v = V0/H0."""
    u, v = U0 / H0, V0 / H0
    A = np.array([[0.0, 1.0, 0.0],
                  [g * H0 - u * u, 2.0 * u, 0.0],
                  [-u * v, v, u]])
    B = np.array([[0.0, 0.0, 1.0],
                  [-u * v, v, u],
                  [g * H0 - v * v, 0.0, 2.0 * v]])
    return A, B


def lw_amplification(A, B, lx: float, ly: float, tx: float, ty: float):
    """Amplification matrix of the two-step Lax-Wendroff scheme for the
    linear system q_t + A q_x + B q_y = 0 and the mode exp(i (tx*i + ty*j)).

    With face states q_{i+1/2} = (q_i + q_{i+1})/2 - (lx/2) A (q_{i+1} - q_i)
    and the update q' = q - lx A (q_{i+1/2} - q_{i-1/2}) - ly B (...), the
    face difference of the mode is [i sin(tx) + lx A (1 - cos(tx))] q, hence
        G = I - i lx sin(tx) A - lx^2 (1 - cos tx) A^2
              - i ly sin(ty) B - ly^2 (1 - cos ty) B^2,
    with lx = dt/dx, ly = dt/dy."""
    I = np.eye(3, dtype=np.complex128)
    return (I - 1j * lx * math.sin(tx) * A - lx * lx * (1.0 - math.cos(tx)) * (A @ A)
            - 1j * ly * math.sin(ty) * B - ly * ly * (1.0 - math.cos(ty)) * (B @ B))


# ---------------------------------------------------------------------------
# Independent 1D two-step Lax-Wendroff (Richtmyer) code
# ---------------------------------------------------------------------------

def textbook_lw_1d(h: np.ndarray, m: np.ndarray, dx: float, dt: float, g: float, n_steps: int):
    """1D shallow water q = (h, m = hu), f(q) = (m, m^2/h + g h^2/2), with
    reflective walls (ghost h mirrored, ghost m negated).  Two-step
    Richtmyer: half step to the faces, then a conservative full step."""
    h = h.astype(np.float64).copy()
    m = m.astype(np.float64).copy()
    for _ in range(n_steps):
        hg = np.concatenate(([h[0]], h, [h[-1]]))
        mg = np.concatenate(([-m[0]], m, [-m[-1]]))
        f1 = mg
        f2 = mg ** 2 / hg + 0.5 * g * hg ** 2
        hf = (hg[:-1] + hg[1:]) / 2 - dt / (2 * dx) * (f1[1:] - f1[:-1])
        mf = (mg[:-1] + mg[1:]) / 2 - dt / (2 * dx) * (f2[1:] - f2[:-1])
        F1 = mf
        F2 = mf ** 2 / hf + 0.5 * g * hf ** 2
        h = h - dt / dx * (F1[1:] - F1[:-1])
        m = m - dt / dx * (F2[1:] - F2[:-1])
    return h, m
