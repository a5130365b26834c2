"""Pins of the closure oracle (oracle/closure.py):
  * forward convolution equals torch.nn.functional.conv3d on circularly padded
    input (an independent library routine), in FP64;
  * every gradient (weights, biases, through both ReLUs) equals central finite
    differences of the loss;
  * the input gradient of a convolution equals its adjoint (<dy, conv(x)> =
    <conv^T(dy), x> with zero bias);
  * Adam equals torch.optim.Adam on the same gradients;
  * bfloat16 rounding equals torch's float -> bfloat16 conversion;
  * the shell spectrum of a single Fourier mode puts |A|^2/4 per component in shell |k|.
"""
import math

import numpy as np
import pytest

from oracle import closure

torch = pytest.importorskip("torch")


def _x(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_torch_circular():
    import torch.nn.functional as F
    x = _x((5, 6, 7, 8), 1)
    W = _x((4, 5, 3, 3, 3), 2)
    b = _x((4,), 3)
    y = closure.conv3d(x, W, b)
    xt = torch.from_numpy(x)[None]
    xp = F.pad(xt, (1, 1, 1, 1, 1, 1), mode="circular")
    yt = F.conv3d(xp, torch.from_numpy(W), torch.from_numpy(b))[0].numpy()
    np.testing.assert_allclose(y, yt, rtol=1e-12, atol=1e-12)


def test_input_grad_is_adjoint():
    x = _x((3, 5, 4, 6), 4)
    dy = _x((2, 5, 4, 6), 5)
    W = _x((2, 3, 3, 3, 3), 6)
    lhs = np.sum(dy * closure.conv3d(x, W, np.zeros(2)))
    rhs = np.sum(closure.conv3d_input_grad(dy, W) * x)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gradients_match_finite_differences():
    net = closure.Net.init(7, channels=(3, 4, 4, 2))
    x = _x((3, 4, 5, 3), 8)
    t = _x((2, 4, 5, 3), 9)
    loss, grads = net.loss_and_grads(x, t)
    rng = np.random.default_rng(10)
    h = 1e-6
    for li in range(3):
        for pi in range(2):
            arr = net.params[li][pi]
            for _ in range(4):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = net.loss_and_grads(x, t)
                arr[idx] = old - h
                lm, _ = net.loss_and_grads(x, t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][pi][idx]
                assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (li, pi, idx, fd, an)


def test_adam_matches_torch():
    shapes = [(3, 2), (4,)]
    rng = np.random.default_rng(11)
    params = [rng.standard_normal(s) for s in shapes]
    tp = [torch.tensor(p, requires_grad=True) for p in params]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    ad = closure.Adam(shapes, lr=1e-2)
    for it in range(5):
        grads = [rng.standard_normal(s) for s in shapes]
        for p, g in zip(tp, grads):
            p.grad = torch.tensor(g)
        opt.step()
        params = ad.step(params, grads)
        for p, q in zip(params, tp):
            np.testing.assert_allclose(p, q.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_bf16_round_matches_torch():
    a = np.concatenate([_x((1000,), 12) * 10.0 ** np.arange(-5, 5).repeat(100),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -0.0, 65504.0]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(closure.bf16_round(a), ref)


def test_spectrum_of_single_mode():
    n = 16
    z, y, x = np.meshgrid(*[np.arange(n) * 2 * math.pi / n] * 3, indexing="ij")
    v = np.zeros((3, n, n, n))
    v[1] = 0.7 * np.cos(3 * x)
    E = closure.energy_spectrum(v)
    assert abs(E[3] - 0.5 * 0.7 ** 2 / 2) < 1e-14
    assert abs(E.sum() - E[3]) < 1e-14


def _spread_case(n, seed):
    from paper_2103_01597_gb300 import synthetic
    net = closure.Net.init(seed)
    net = closure.Net.unflat(net.flat().astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(seed)
    x = synthetic.turbulent_state(n, seed, kmax=3, amp=0.5)
    x = (x / (0.5 + rng.random(8))[:, None, None, None]).astype(np.float32).astype(np.float64)
    t = rng.standard_normal(x.shape)
    return net, x, t


@pytest.mark.parametrize("n,seed", [((16, 12, 10), 6), ((12, 8, 6), 3), ((10, 10, 10), 11)])
def test_bf16_rounding_spread_calibrates_the_gpu_tolerance(n, seed):
    """The GPU closure tests accept a tensor within 4 (L2) and 6 (max norm)
    rounding spreads of the configuration-precision oracle.  The oracle's own
    evaluation with bfloat16 at the kernels' rounding points -- one
    deterministic instance of that rounding -- must sit well inside (measured:
    L2 <= 1.7, max <= 2.8), and the spread must be a small but non-zero part
    of each tensor, so the criterion still catches a wrong term."""
    net, x, t = _spread_case(n, seed)
    _, gk = net.loss_and_grads(x, t, bf16="kernel")
    _, gc = net.loss_and_grads(x, t, bf16="config")
    sg = net.rounding_spread(x, t, samples=16)
    yk, _ = net.forward(x, bf16="kernel")
    yc, _ = net.forward(x, bf16="config")
    sy = net.rounding_spread(x, samples=16)
    pairs = [(yk, yc, sy)] + [(gk[li][a], gc[li][a], sg[li][a]) for li in range(3) for a in range(2)]
    for g, o, s in pairs:
        d = g - o
        assert np.linalg.norm(d) <= 2.5 * np.linalg.norm(s)
        assert np.max(np.abs(d)) <= 4.0 * np.max(s)
        assert 1e-5 < np.max(s) / np.max(np.abs(o)) < 0.1
