"""FP64 oracle for the learned coarse-grid corrector (TEST INFRASTRUCTURE).

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this module; it shares no code with the CUDA library.

The corrector is a plain three-layer convolutional network on a coarse
shallow-water state (no counterpart in the paper; the paper's method is the
Lax-Wendroff step of Sec. 3, which the network corrects):

    x0 = normalised (h, hu, hv)                       3 channels
    z1 = conv3x3(x0; W1, b1),  a1 = gelu(z1)          32 channels
    z2 = conv3x3(a1; W2, b2),  a2 = gelu(z2)          32 channels
    r  = conv3x3(a2; W3, b3)                          3 channels

conv3x3 is a cross-correlation with zero padding (outside the grid the
input is 0):  y[n, o, i, j] = b[o] + sum_{c, dy, dx} W[dy+1, dx+1, c, o] *
x[n, c, i+dy, j+dx], with i the row (y) and j the column (x) index.
Weights are stored as W[ky, kx, c_in, c_out].  gelu is the exact erf form
0.5 z (1 + erf(z / sqrt 2)).  The loss is the mean squared error over all
elements, optionally weighted per image (``image_weights``).  Arrays are
NCHW float64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[..., i, j] = x[..., i+dy, j+dx], zero where that is outside."""
    out = np.zeros_like(x)
    H, W = x.shape[-2], x.shape[-1]
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    if i0 < i1 and j0 < j1:
        out[..., i0:i1, j0:j1] = x[..., i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return out


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3 cross-correlation, x (N, C, H, W), W (3, 3, C, O)."""
    y = np.zeros((x.shape[0], W.shape[3], x.shape[2], x.shape[3]))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nchw,co->nohw", shift(x, ky - 1, kx - 1), W[ky, kx])
    return y + b[None, :, None, None]


def conv3x3_input_grad(dy: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in x: dx[n, c, i, j] = sum_{o, taps}
    W[ky, kx, c, o] * dy[n, o, i - (ky-1), j - (kx-1)]."""
    dx = np.zeros((dy.shape[0], W.shape[2], dy.shape[2], dy.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dx += np.einsum("nohw,co->nchw", shift(dy, -(ky - 1), -(kx - 1)), W[ky, kx])
    return dx


def conv3x3_weight_grad(x: np.ndarray, dy: np.ndarray):
    """dW[ky, kx, c, o] = sum_{n,i,j} x[n, c, i+ky-1, j+kx-1] dy[n, o, i, j];
    db[o] = sum dy[n, o, :, :]."""
    dW = np.zeros((3, 3, x.shape[1], dy.shape[1]))
    for ky in range(3):
        for kx in range(3):
            dW[ky, kx] = np.einsum("nchw,nohw->co", shift(x, ky - 1, kx - 1), dy)
    return dW, dy.sum(axis=(0, 2, 3))


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * np.exp(-0.5 * z * z) * INV_SQRT_2PI


def forward(params, x0):
    """Returns (r, cache).  params = dict W1,b1,W2,b2,W3,b3."""
    z1 = conv3x3(x0, params["W1"], params["b1"])
    a1 = gelu(z1)
    z2 = conv3x3(a1, params["W2"], params["b2"])
    a2 = gelu(z2)
    r = conv3x3(a2, params["W3"], params["b3"])
    return r, dict(x0=x0, z1=z1, a1=a1, z2=z2, a2=a2)


def image_weights(t, power, floor):
    """Per-image loss weights w_i = max(ms_i, floor)^(-power/2), ms_i the
    mean square of image i's target (all channels)."""
    ms = np.mean(np.asarray(t, np.float64).reshape(t.shape[0], -1) ** 2, axis=1)
    return np.maximum(ms, floor) ** (-0.5 * power)


def loss(r, t, w=None):
    """mean over all elements of w_i (r - t)^2 (w = None: plain MSE)."""
    d2 = (r - t) ** 2
    if w is not None:
        d2 = d2 * np.asarray(w, np.float64)[:, None, None, None]
    return float(np.mean(d2))


def backward(params, cache, r, t, w=None):
    """Gradients of loss(r, t, w) w.r.t. every parameter."""
    dr = 2.0 * (r - t) / r.size
    if w is not None:
        dr = dr * np.asarray(w, np.float64)[:, None, None, None]
    g = {}
    g["W3"], g["b3"] = conv3x3_weight_grad(cache["a2"], dr)
    dz2 = conv3x3_input_grad(dr, params["W3"]) * gelu_grad(cache["z2"])
    g["W2"], g["b2"] = conv3x3_weight_grad(cache["a1"], dz2)
    dz1 = conv3x3_input_grad(dz2, params["W2"]) * gelu_grad(cache["z1"])
    g["W1"], g["b1"] = conv3x3_weight_grad(cache["x0"], dz1)
    return g, dict(dr=dr, dz2=dz2, dz1=dz1)


def init_params(seed: int, cin=3, hidden=32, cout=3, out_scale=0.1):
    """He-style initialisation from numpy's PCG64 (inputs of the tests)."""
    rng = np.random.default_rng(seed)

    def w(ci, co, scale):
        return rng.standard_normal((3, 3, ci, co)) * scale / math.sqrt(9 * ci)

    return dict(W1=w(cin, hidden, math.sqrt(2.0)), b1=0.01 * rng.standard_normal(hidden),
                W2=w(hidden, hidden, math.sqrt(2.0)), b2=0.01 * rng.standard_normal(hidden),
                W3=w(hidden, cout, out_scale), b3=np.zeros(cout))


def block_average(u: np.ndarray, f: int) -> np.ndarray:
    """f x f block average of the last two axes (sizes divisible by f)."""
    H, W = u.shape[-2], u.shape[-1]
    v = u.reshape(u.shape[:-2] + (H // f, f, W // f, f))
    return v.sum(axis=(-3, -1)) / float(f * f)


def area_matrix(n_src: int, n_dst: int) -> np.ndarray:
    """R[X, i] = |[X f, (X+1) f) & [i, i+1)| / f, f = n_src / n_dst: the
    overlap-weighted mean of source cells over destination cell X."""
    f = n_src / n_dst
    R = np.zeros((n_dst, n_src))
    for X in range(n_dst):
        a, b = X * f, (X + 1) * f
        for i in range(int(np.floor(a)), min(n_src, int(np.ceil(b)))):
            R[X, i] = (min(b, i + 1) - max(a, i)) / f
    return R


def area_average(u: np.ndarray, h_dst: int, w_dst: int) -> np.ndarray:
    """Area-weighted average of the last two axes onto h_dst x w_dst cells
    covering the same domain (any ratio >= 1): R_y u R_x^T."""
    Ry = area_matrix(u.shape[-2], h_dst)
    Rx = area_matrix(u.shape[-1], w_dst)
    return Ry @ np.asarray(u, np.float64) @ Rx.T


def downsample4(u: np.ndarray) -> np.ndarray:
    """4x4 block average of the last two axes (sizes divisible by 4)."""
    return block_average(u, 4)
