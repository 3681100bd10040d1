"""The corrector network's tcgen05 kernels against the FP64 oracle
(oracle/nn.py): forward output, loss and every parameter gradient, on the
same bf16-rounded weights and inputs.  GPU activations are rounded to bf16
between layers, so the bars are relative L2 <= 2e-2 and cosine >= 0.999."""
import numpy as np
import pytest

from oracle import nn

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round to the nearest bf16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _state(n, H, W, seed):
    rng = np.random.default_rng(seed)
    y = np.linspace(0, 1, H)[:, None]
    x = np.linspace(0, 1, W)[None, :]
    out = np.zeros((n, 3, H, W))
    for i in range(n):
        a, b, c = rng.uniform(1, 4, 3)
        out[i, 0] = 1.0 + 0.3 * np.sin(a * np.pi * x + b) * np.cos(c * np.pi * y) + 0.05 * rng.standard_normal((H, W))
        out[i, 1] = 0.2 * np.cos(b * np.pi * x) * np.sin(a * np.pi * y) + 0.05 * rng.standard_normal((H, W))
        out[i, 2] = -0.2 * np.sin(c * np.pi * x * y) + 0.05 * rng.standard_normal((H, W))
    return out.astype(np.float32)


NORM = (1.0, 0.5, 0.3, 1.0, 1.0)


def _oracle_inputs(state):
    h0, sh, su = NORM[:3]
    x0 = np.stack([(state[:, 0] - h0) / sh, state[:, 1] / su, state[:, 2] / su], axis=1)
    return bf16_round(x0.astype(np.float32))


def _oracle_params(params):
    return {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
            for k, v in params.items()}


def _net_with(params, n, H, W):
    from paper_1107_2157_gb300 import Net, swe
    net = Net(n, H, W)
    net.set_params(swe.flatten_params(params))
    net.set_norm(*NORM)
    return net


@pytest.mark.parametrize("n,H,W", [(2, 9, 300), (3, 16, 128), (1, 5, 40)])
def test_forward_matches_oracle(n, H, W):
    import torch
    params = nn.init_params(3, out_scale=1.0)
    st = _state(n, H, W, 1)
    dev = torch.from_numpy(st).cuda()
    resid = torch.zeros((n, 3, H, W), dtype=torch.float32, device="cuda")
    with _net_with(params, n, H, W) as net:
        net.prep_input(n, dev.data_ptr(), 3 * H * W, H * W, W)  # state mode (no base)
        net.infer(n, resid.data_ptr())
        assert net.check() == 0
    got = resid.cpu().numpy()
    ref, _ = nn.forward(_oracle_params(params), _oracle_inputs(st))
    for i in range(n):
        assert rel_l2(got[i], ref[i]) <= 2e-2, (i, rel_l2(got[i], ref[i]))
        assert cosine(got[i], ref[i]) >= 0.999


@pytest.mark.parametrize("power,n,H,W", [(0.0, 2, 12, 260), (1.0, 2, 12, 260), (2.0, 2, 12, 260),
                                         (1.0, 4, 130, 390)])
def test_backward_matches_oracle(power, n, H, W):
    """Loss, residual and every gradient against the FP64 oracle.  The
    weight gradients run on the tensor cores in persistent CTAs of 128 x 4
    pixel tiles: 12 x 260 has ragged tiles in x and y, 4 x 130 x 390 has more
    tiles than CTAs, so CTAs accumulate several tiles in TMEM."""
    import torch
    params = nn.init_params(5, out_scale=1.0)
    st = _state(n, H, W, 2)
    rng = np.random.default_rng(9)
    scale = np.where(np.arange(n) % 2 == 0, 1.0, 6.0)[:, None, None, None]  # images of unequal loss weight
    target = (rng.standard_normal((n, 3, H, W)) * scale).astype(np.float32)
    dev = torch.from_numpy(st).cuda()
    tdev = torch.from_numpy(target).cuda()
    r_dev = torch.zeros((n, 3, H, W), dtype=torch.float32, device="cuda")
    from paper_1107_2157_gb300 import swe
    with _net_with(params, n, H, W) as net:
        net.set_loss_weighting(power, 1.0)
        net.prep_input(n, dev.data_ptr(), 3 * H * W, H * W, W)  # state mode (no base)
        loss, g = net.train_step(n, tdev.data_ptr(), update=False, want_grads=True, resid_ptr=r_dev.data_ptr())
    op = _oracle_params(params)
    r, cache = nn.forward(op, _oracle_inputs(st))
    w = nn.image_weights(target, power, 1.0) if power else None
    ref_loss = nn.loss(r, target, w)
    grads, _ = nn.backward(op, cache, r, target, w)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    assert rel_l2(r_dev.cpu().numpy(), r) <= 2e-2
    gg = swe.unflatten_params(g)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel_l2(gg[k], grads[k]) <= 2e-2, (k, rel_l2(gg[k], grads[k]))
        assert cosine(gg[k], grads[k]) >= 0.999, (k, cosine(gg[k], grads[k]))


@pytest.mark.parametrize("factor", [2, 3, 4])
def test_block_average_matches_oracle(factor):
    import torch
    from paper_1107_2157_gb300 import swe
    n, Hc, Wc, F = 3, 12, 20, factor
    rng = np.random.default_rng(4)
    fine = rng.standard_normal((n, 3, F * Hc, F * Wc)).astype(np.float32)
    fdev = torch.from_numpy(fine).cuda()
    cdev = torch.zeros((n, 3, Hc, Wc), dtype=torch.float32, device="cuda")
    swe.swe_downsample(F, fdev.data_ptr(), 3 * F * F * Hc * Wc, F * F * Hc * Wc, F * Wc, cdev.data_ptr(),
                       3 * Hc * Wc, Hc * Wc, Wc, Wc, Hc, n)
    torch.cuda.synchronize()
    ref = nn.block_average(fine.astype(np.float64), F)
    assert np.abs(cdev.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def test_training_reduces_the_loss_on_a_fixed_batch():
    import torch
    n, H, W = 4, 32, 128
    params = nn.init_params(7, out_scale=0.1)
    st = _state(n, H, W, 3)
    # a smooth, learnable target: a fixed linear filter of the input
    x0 = _oracle_inputs(st)
    target = (0.5 * nn.shift(x0, 0, 1) - 0.5 * nn.shift(x0, 0, -1)).astype(np.float32)
    dev = torch.from_numpy(st).cuda()
    tdev = torch.from_numpy(np.ascontiguousarray(target)).cuda()
    with _net_with(params, n, H, W) as net:
        net.prep_input(n, dev.data_ptr(), 3 * H * W, H * W, W)  # state mode (no base)
        first, _ = net.train_step(n, tdev.data_ptr(), lr=3e-3)
        for _ in range(300):
            last, _ = net.train_step(n, tdev.data_ptr(), lr=3e-3)
    assert last < first / 5, (first, last)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_device_erf_and_gelu_within_published_bound(which):
    """The network's erf (Abramowitz & Stegun 7.1.26, |error| <= 1.5e-7), the
    forward GELU (erf from A&S 7.1.27) and GELU' (7.1.26), against scipy's
    erf in FP64."""
    import torch
    from scipy.special import erf
    from paper_1107_2157_gb300 import swe
    z = np.concatenate([np.linspace(-8, 8, 20001), [0.0, 1e-8, -1e-8, 30.0, -30.0]]).astype(np.float32)
    zd = torch.from_numpy(z).cuda()
    out = torch.zeros_like(zd)
    swe.check(swe.lib().swe_selftest_gelu(zd.data_ptr(), out.data_ptr(), z.size, which, None), "gelu")
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    x = z.astype(np.float64)
    if which == 0:
        ref, tol = erf(x), 1.5e-7 + 4e-7  # published bound + FP32 evaluation
        assert np.abs(got - ref).max() <= tol
    elif which == 1:
        # forward GELU with erf from A&S 7.1.27: 6.9e-4 from the formula (2.3e-4 |z|
        # beyond |z| = 1), plus FP32 evaluation
        ref = nn.gelu(x)
        assert np.all(np.abs(got - ref) <= 7e-4 * np.maximum(1.0, np.abs(x)) + 1e-6 * np.abs(x))
        assert np.abs(got - ref).max() <= 7e-4
    else:
        ref = nn.gelu_grad(x)
        assert np.abs(got - ref).max() <= 2e-6


@pytest.mark.parametrize("shape", [(1024, 1024, 320, 384), (40, 30, 15, 12), (96, 96, 96, 32), (7, 9, 3, 4)])
def test_area_resample_matches_oracle(shape):
    import torch
    from paper_1107_2157_gb300 import swe
    Hs, Ws, Hd, Wd = shape
    n = 2
    rng = np.random.default_rng(21)
    src = rng.standard_normal((n, 3, Hs, Ws)).astype(np.float32)
    sd = torch.from_numpy(src).cuda()
    dd = torch.zeros((n, 3, Hd, Wd), dtype=torch.float32, device="cuda")
    swe.swe_resample(sd.data_ptr(), 3 * Hs * Ws, Hs * Ws, Ws, Ws, Hs, dd.data_ptr(), 3 * Hd * Wd, Hd * Wd, Wd, Wd, Hd, n)
    torch.cuda.synchronize()
    ref = nn.area_average(src.astype(np.float64), Hd, Wd)
    assert np.abs(dd.cpu().numpy() - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
