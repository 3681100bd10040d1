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


def test_image_weights_closed_form():
    t = np.stack([np.full((3, 4, 5), 0.5), np.full((3, 4, 5), 3.0), np.zeros((3, 4, 5))])
    w = nn.image_weights(t, 2.0, 1.0)
    assert np.allclose(w, [1.0, 1.0 / 9.0, 1.0], rtol=1e-15)     # floor 1 -> 0.25 counts as 1
    w1 = nn.image_weights(t, 1.0, 0.01)
    assert np.allclose(w1, [2.0, 1.0 / 3.0, 10.0], rtol=1e-15)
    assert np.array_equal(nn.image_weights(t, 0.0, 1.0), np.ones(3))


def test_weighted_backward_matches_central_differences():
    rng = np.random.default_rng(13)
    params = nn.init_params(8, hidden=6, out_scale=1.0)
    x0 = rng.standard_normal((3, 3, 7, 6))
    t = rng.standard_normal((3, 3, 7, 6)) * np.array([0.5, 2.0, 10.0])[:, None, None, None]
    w = nn.image_weights(t, 1.0, 1.0)
    r, cache = nn.forward(params, x0)
    grads, _ = nn.backward(params, cache, r, t, w)
    for name in ("W1", "b2", "W3"):
        p = params[name]
        for ix in [tuple(rng.integers(0, s) for s in p.shape) for _ in range(4)]:
            old = p[ix]
            h = 1e-5
            p[ix] = old + h
            lp = nn.loss(nn.forward(params, x0)[0], t, w)
            p[ix] = old - h
            lm = nn.loss(nn.forward(params, x0)[0], t, w)
            p[ix] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[name][ix]) <= 1e-6 * max(abs(fd), 1e-3), (name, ix)


def test_area_average_pins():
    """Worked 1D case, integer ratios = block average, constants and
    integrals kept, and a brute-force subdivision for fractional ratios."""
    u = np.arange(5, dtype=np.float64)[None, :]                # 5 -> 2 cells, f = 2.5
    d = nn.area_average(u, 1, 2)
    assert np.allclose(d, [[(0 + 1 + 0.5 * 2) / 2.5, (0.5 * 2 + 3 + 4) / 2.5]], rtol=0, atol=1e-15)
    rng = np.random.default_rng(17)
    v = rng.standard_normal((2, 3, 12, 18))
    assert np.allclose(nn.area_average(v, 4, 6), nn.block_average(v, 3), atol=1e-14)
    for (hs, ws, hd, wd) in [(16, 20, 5, 6), (1024, 1024, 320, 384), (9, 7, 9, 3), (768, 768, 256, 256)]:
        w = rng.standard_normal((hs, ws))
        a = nn.area_average(w, hd, wd)
        assert abs(a.sum() * (hs / hd) * (ws / wd) - w.sum()) <= 1e-9 * np.abs(w).sum()
        assert np.allclose(nn.area_average(np.full((hs, ws), 1.7), hd, wd), 1.7, atol=1e-13)
    # brute force: split every source cell into 10 x 10 equal parts (the
    # same piecewise-constant field); ratios 2.5 and 3.2 then become the
    # integer block sizes 25 and 32 of a plain block average
    w = rng.standard_normal((10, 16))
    fine = np.repeat(np.repeat(w, 10, axis=0), 10, axis=1)     # 100 x 160
    ref = fine.reshape(4, 25, 5, 32).mean(axis=(1, 3))
    assert np.allclose(nn.area_average(w, 4, 5), ref, atol=1e-13)
