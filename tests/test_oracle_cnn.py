"""Pins of the oracle's learned correction (residual CNN over Pi_F): periodic
3x3 convolution, its adjoint and parameter gradients, pixel shuffle, Adam and
the whole loss gradient, against torch CPU library routines in FP64 and central
finite differences; the zero-initialised last layer reproduces Pi_F exactly."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _torch_conv(x, W, b):
    xt = torch.tensor(x)[None]
    xt = F.pad(xt, (1, 1, 1, 1), mode="circular")
    return F.conv2d(xt, torch.tensor(W), torch.tensor(b))[0]


@pytest.mark.parametrize("cin,cout,n", [(8, 32, 6), (3, 5, 4), (2, 2, 9)])
def test_conv_matches_library_convolution(cin, cout, n):
    rng = np.random.default_rng(cin * n)
    x, W, b = rng.standard_normal((cin, n, n)), rng.standard_normal((cout, cin, 3, 3)), rng.standard_normal(cout)
    ref = _torch_conv(x, W, b).numpy()
    np.testing.assert_allclose(O.conv3x3(x, W, b), ref, atol=1e-12)
    np.testing.assert_allclose(O.conv3x3(x, W, b, relu=True), np.maximum(ref, 0), atol=1e-12)


def test_conv_backward_matches_autograd():
    rng = np.random.default_rng(4)
    cin, cout, n = 4, 6, 7
    x, W, b = rng.standard_normal((cin, n, n)), rng.standard_normal((cout, cin, 3, 3)), rng.standard_normal(cout)
    dout = rng.standard_normal((cout, n, n))
    xt, Wt, bt = (torch.tensor(a, requires_grad=True) for a in (x, W, b))
    out = F.conv2d(F.pad(xt[None], (1, 1, 1, 1), mode="circular"), Wt, bt)[0]
    (out * torch.tensor(dout)).sum().backward()
    din, dW, db = O.conv3x3_bwd(x, W, dout)
    np.testing.assert_allclose(din, xt.grad.numpy(), atol=1e-11)
    np.testing.assert_allclose(dW, Wt.grad.numpy(), atol=1e-11)
    np.testing.assert_allclose(db, bt.grad.numpy(), atol=1e-11)


def test_pixel_shuffle_matches_library():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((64, 5, 3 * 1 + 2))
    ref = F.pixel_shuffle(torch.tensor(x)[None], 4)[0].numpy()
    np.testing.assert_array_equal(O.pixel_shuffle4(x), ref)
    np.testing.assert_array_equal(O.pixel_unshuffle4(ref), x)


def _params(rng, zero_last=False, scale=0.2):
    p = {k: scale * rng.standard_normal(s) for k, s in O.CNN_SHAPES}
    if zero_last:
        p["W3"][...] = 0.0
        p["b3"][...] = 0.0
    return p


def _stats():
    return dict(mu_in=np.linspace(-0.1, 0.1, 8), s_in=np.linspace(0.5, 1.5, 8), s_out=np.array([0.3, 0.5, 0.7, 0.9]))


def test_zero_last_layer_is_plain_prolongation():
    rng = np.random.default_rng(6)
    nc = 5
    dC, xs = rng.standard_normal((4, nc, nc)), rng.standard_normal((4, nc, nc))
    pred, _ = O.cnn_forward(_params(rng, zero_last=True), dC, xs, _stats())
    base = O.prolong_add(dC.reshape(-1), np.zeros(4 * (4 * nc) ** 2), 2, 4, nc, 4).reshape(4, 4 * nc, 4 * nc)
    np.testing.assert_array_equal(pred, base)


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    nc = 4
    dC, xs = rng.standard_normal((4, nc, nc)), rng.standard_normal((4, nc, nc))
    target = rng.standard_normal((4, 4 * nc, 4 * nc))
    params, stats = _params(rng), _stats()
    _, grads = O.cnn_loss_grad(params, dC, xs, target, stats)
    h = 1e-6
    for k in params:
        flat = params[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = O.cnn_loss_grad(params, dC, xs, target, stats)
            flat[idx] = old - h
            lm, _ = O.cnn_loss_grad(params, dC, xs, target, stats)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = grads[k].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (k, idx, fd, g)


def test_adam_matches_library_optimizer():
    rng = np.random.default_rng(8)
    params = {k: rng.standard_normal(s) for k, s in O.CNN_SHAPES[:2]}
    tp = [torch.tensor(params[k].copy(), requires_grad=True) for k in params]
    opt = torch.optim.Adam(tp, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    for step in range(5):
        grads = {k: rng.standard_normal(params[k].shape) for k in params}
        for t, k in zip(tp, params):
            t.grad = torch.tensor(grads[k])
        opt.step()
        params = O.adam_step(params, grads, state, lr=1e-3)
    for t, k in zip(tp, params):
        np.testing.assert_allclose(params[k], t.detach().numpy(), rtol=1e-12, atol=1e-14)
