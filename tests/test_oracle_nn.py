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


def test_bf16_rounding_is_nearest_even():
    from oracle.learned import bf16_round
    one = 1.0
    ulp = 2.0 ** -7                      # bf16 spacing at 1
    x = np.array([one, one + ulp, one + ulp / 2, one + 3 * ulp / 2, -(one + ulp / 2), 0.0, 3.0e38, 1e-40])
    got = bf16_round(x)
    assert got[0] == one and got[1] == one + ulp
    assert got[2] == one                 # tie -> even mantissa
    assert got[3] == one + 2 * ulp       # tie -> even mantissa
    assert got[4] == -one
    assert got[5] == 0.0
    assert np.isfinite(got[6])
    assert got[7] == 2.0 ** -133         # subnormal: the bf16 spacing there is 2^-133
    rng = np.random.default_rng(11)
    v = rng.standard_normal(1000)
    r = bf16_round(v)
    assert np.all(np.abs(r - v) <= 2.0 ** -8 * np.abs(v) * (1 + 1e-6))  # unit roundoff of 8 significant bits


def _learned_state(seed, nx, ny):
    import swe_inputs as si
    return si.smooth_flow_state(seed, nx, ny)


def test_learned_step_with_zero_network_is_the_lax_wendroff_step():
    import oracle
    from oracle import learned
    s = _learned_state(1, 13, 9)
    p = {k: np.zeros_like(v) for k, v in nn.init_params(0).items()}
    got, d = learned.corrected_step(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, p, (0, 1e-3, 1e-3, 1e-2, 1e-2))
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, 1)
    for k in range(3):
        assert np.array_equal(got[k], ref[k])
    assert not d.any()


def test_learned_step_constant_output_scaling_and_projection():
    """W3 = 0 makes the network output its bias b3 everywhere: the h
    correction oh*b3[0] is removed by the projection, the momentum
    corrections are ou*b3[1:] exactly."""
    import oracle
    from oracle import learned
    s = _learned_state(2, 11, 7)
    p = nn.init_params(3)
    p["W3"] = np.zeros_like(p["W3"])
    p["b3"] = np.array([0.5, -0.25, 2.0])
    norm = (0.0, 1e-3, 1e-3, 1e-2, 4e-2)
    ref = oracle.run(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, 1)
    got, _ = learned.corrected_step(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, p, norm, project_mass=True)
    assert np.allclose(got[0], ref[0], rtol=0, atol=1e-15)
    assert np.allclose(got[1], ref[1] + 4e-2 * -0.25, rtol=0, atol=1e-15)
    assert np.allclose(got[2], ref[2] + 4e-2 * 2.0, rtol=0, atol=1e-15)
    got, _ = learned.corrected_step(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, p, norm, project_mass=False)
    assert np.allclose(got[0], ref[0] + 1e-2 * 0.5, rtol=0, atol=1e-15)


def test_learned_step_keeps_mass_under_projection():
    import oracle
    from oracle import learned
    s = _learned_state(4, 17, 12)
    p = nn.init_params(5, out_scale=1.0)
    norm = (0.0, 1e-3, 1e-3, 1e-2, 1e-2)
    m0 = oracle.mass(s.h, 1.0, 1.0)
    got = learned.corrected_run(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, p, norm, 3)
    assert abs(oracle.mass(got[0], 1.0, 1.0) - m0) <= 1e-13 * m0
    free, _ = learned.corrected_step(s.h, s.hu, s.hv, 1.0, 1.0, 0.05, 9.8, p, norm, project_mass=False)
    assert abs(oracle.mass(free[0], 1.0, 1.0) - m0) > 1e-9 * m0  # the network alone does not
