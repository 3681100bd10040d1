"""Pins of the corrector network oracle (oracle/nn.py) and the 4x4 block
average: library special cases, closed forms and finite differences."""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import nn


def test_single_channel_conv_is_scipy_correlate_with_zero_fill():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 1, 9, 13))
    W = rng.standard_normal((3, 3, 1, 1))
    y = nn.conv3x3(x, W, np.zeros(1))
    ref = correlate2d(x[0, 0], W[:, :, 0, 0], mode="same", boundary="fill", fillvalue=0.0)
    assert np.allclose(y[0, 0], ref, rtol=0, atol=1e-13)


def test_multichannel_conv_sums_single_channel_convs():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 6, 7))
    W = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    y = nn.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, c], W[:, :, c, o], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_input_grad_is_the_adjoint_of_conv():
    # <conv(x), y> = <x, conv^T(y)> for the zero-padded linear map
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 5, 7, 6))
    W = rng.standard_normal((3, 3, 5, 4))
    y = rng.standard_normal((2, 4, 7, 6))
    lhs = np.sum(nn.conv3x3(x, W, np.zeros(4)) * y)
    rhs = np.sum(x * nn.conv3x3_input_grad(y, W))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_gelu_limits_and_slope():
    assert nn.gelu(np.array(0.0)) == 0.0
    assert abs(nn.gelu(np.array(10.0)) - 10.0) < 1e-15
    assert abs(nn.gelu(np.array(-10.0))) < 1e-20
    assert abs(nn.gelu_grad(np.array(0.0)) - 0.5) < 1e-16
    # exact value at 1: Phi(1) = 0.841344746068543
    assert abs(nn.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (nn.gelu(z + h) - nn.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, nn.gelu_grad(z), atol=1e-8)


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3"])
def test_backward_matches_central_differences(name):
    rng = np.random.default_rng(3)
    params = nn.init_params(4, hidden=6, out_scale=1.0)
    x0 = rng.standard_normal((2, 3, 8, 8))
    t = rng.standard_normal((2, 3, 8, 8))
    r, cache = nn.forward(params, x0)
    grads, _ = nn.backward(params, cache, r, t)
    p = params[name]
    idx = [tuple(rng.integers(0, s) for s in p.shape) for _ in range(6)]
    for ix in idx:
        old = p[ix]
        h = 1e-5
        p[ix] = old + h
        lp = nn.loss(nn.forward(params, x0)[0], t)
        p[ix] = old - h
        lm = nn.loss(nn.forward(params, x0)[0], t)
        p[ix] = old
        fd = (lp - lm) / (2 * h)
        g = grads[name][ix]
        assert abs(fd - g) <= 1e-6 * max(abs(fd), 1e-3), (name, ix, fd, g)


def test_downsample_preserves_sums_constants_and_linear_fields():
    rng = np.random.default_rng(5)
    u = rng.standard_normal((3, 16, 24))
    d = nn.downsample4(u)
    assert d.shape == (3, 4, 6)
    assert np.allclose(d.sum(axis=(1, 2)) * 16, u.sum(axis=(1, 2)))
    assert np.array_equal(nn.downsample4(np.full((8, 8), 2.5)), np.full((2, 2), 2.5))
    i = np.arange(16)[:, None]
    j = np.arange(12)[None, :]
    lin = 0.3 * i - 0.7 * j + 1.0
    d = nn.downsample4(lin.astype(np.float64))
    I = np.arange(4)[:, None] * 4 + 1.5
    J = np.arange(3)[None, :] * 4 + 1.5
    assert np.allclose(d, 0.3 * I - 0.7 * J + 1.0, atol=1e-14)
