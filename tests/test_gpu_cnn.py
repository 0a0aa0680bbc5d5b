"""GPU parity of the learned correction (residual CNN over Pi_F): forward pass
and parameter gradients against the FP64 oracle fed the same BF16-rounded
weights, the zero-initialised last layer, and one Adam step."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf
    return mgenkf


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _case(nc, B, seed, zero_last=False):
    rng = np.random.default_rng(seed)
    params = {k: 0.15 * rng.standard_normal(s) for k, s in O.CNN_SHAPES}
    if zero_last:
        params["W3"][...] = 0
        params["b3"][...] = 0
    stats = dict(mu_in=0.1 * rng.standard_normal(8), s_in=rng.uniform(0.5, 2.0, 8), s_out=rng.uniform(0.2, 1.0, 4))
    dC = rng.standard_normal((B, 4, nc, nc))
    xs = rng.standard_normal((B, 4, nc, nc))
    target = rng.standard_normal((B, 4, 4 * nc, 4 * nc))
    return params, stats, dC, xs, target


def _gpu(M, nc, B, params, stats):
    cnn = M.CNN(nc, B)
    cnn.set_params(params, stats)
    return cnn


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


# 130: two 128-pixel tiles per row (the second ragged) and a ragged last row
# block; 256: the learned-correction configuration (256^2 coarse, 1024^2 fine)
@pytest.mark.parametrize("nc,B", [(8, 2), (20, 1), (32, 3), (130, 1), (256, 1)])
def test_forward_matches_oracle(M, nc, B):
    import torch
    params, stats, dC, xs, _ = _case(nc, B, nc)
    cnn = _gpu(M, nc, B, params, stats)
    d_dC = torch.tensor(dC, dtype=torch.float32, device="cuda")
    d_xs = torch.tensor(xs, dtype=torch.float32, device="cuda")
    res = torch.zeros((B, 4, 4 * nc, 4 * nc), dtype=torch.float32, device="cuda")
    cnn.forward(d_dC, d_xs, B, res)
    torch.cuda.synchronize()
    pq = {k: _bf16(v) if k.startswith("W") else v for k, v in params.items()}
    for b in range(B):
        pred, _ = O.cnn_forward(pq, dC[b], xs[b], stats)
        base = O.prolong_add(dC[b].reshape(-1), np.zeros(4 * (4 * nc) ** 2), 2, 4, nc, 4).reshape(pred.shape)
        # BF16 activations (2^-9 rounding at each of three layers), FP32 accumulation
        assert _rel(res[b].cpu().double().numpy(), pred - base) < 2e-2
    cnn.close()


def _round_bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("nc", [20, 130, 256])
def test_forward_elementwise_against_bf16_rounding_oracle(M, nc):
    """Element-wise forward parity.  The GPU rounds the normalised input and
    the two hidden activations to BF16 and accumulates in FP32; the oracle's
    convolutions with the same roundings give the reference, and what remains
    is FP32 accumulation order plus activations that land on the other side of
    a BF16 rounding boundary.  Bound per output element: 2e-3 of the absolute
    value network |W3| * |a2| (+ |b3|) at that element, times s_out.  A wrong
    tap, row, tile or channel group moves an element by a sizeable fraction of
    that sum."""
    import torch
    params, stats, dC, xs, _ = _case(nc, 1, 500 + nc)
    cnn = _gpu(M, nc, 1, params, stats)
    res = torch.zeros((1, 4, 4 * nc, 4 * nc), dtype=torch.float32, device="cuda")
    cnn.forward(torch.tensor(dC, dtype=torch.float32, device="cuda"),
                torch.tensor(xs, dtype=torch.float32, device="cuda"), 1, res)
    torch.cuda.synchronize()
    got = res[0].cpu().double().numpy()
    pq = {k: _bf16(v) if k.startswith("W") else v for k, v in params.items()}
    a0 = _round_bf16((np.concatenate([dC[0], xs[0]]) - stats["mu_in"][:, None, None]) / stats["s_in"][:, None, None])
    a1 = _round_bf16(np.maximum(O.conv3x3(a0, pq["W1"], pq["b1"]), 0.0))
    a2 = _round_bf16(np.maximum(O.conv3x3(a1, pq["W2"], pq["b2"]), 0.0))
    z3 = O.conv3x3(a2, pq["W3"], pq["b3"])
    s_out = stats["s_out"][:, None, None]
    ref = O.pixel_shuffle4(z3) * s_out
    bound = O.pixel_shuffle4(O.conv3x3(np.abs(a2), np.abs(pq["W3"]), np.abs(pq["b3"]))) * s_out
    err = np.abs(got - ref)
    assert np.all(err <= 2e-3 * bound), (float(np.max(err / bound)), np.unravel_index(np.argmax(err / bound), err.shape))
    cnn.close()


def test_zero_last_layer_gives_zero_residual(M):
    import torch
    params, stats, dC, xs, _ = _case(8, 1, 3, zero_last=True)
    cnn = _gpu(M, 8, 1, params, stats)
    res = torch.full((1, 4, 32, 32), 7.0, dtype=torch.float32, device="cuda")
    cnn.forward(torch.tensor(dC, dtype=torch.float32, device="cuda"),
                torch.tensor(xs, dtype=torch.float32, device="cuda"), 1, res)
    torch.cuda.synchronize()
    assert float(res.abs().max()) == 0.0
    cnn.close()


@pytest.mark.parametrize("nc,B", [(8, 2), (20, 1), (256, 1)])
def test_gradients_match_oracle(M, nc, B):
    import torch
    params, stats, dC, xs, target = _case(nc, B, 100 + nc)
    cnn = _gpu(M, nc, B, params, stats)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    cnn.loss_grad(torch.tensor(dC, dtype=torch.float32, device="cuda"),
                  torch.tensor(xs, dtype=torch.float32, device="cuda"),
                  torch.tensor(target, dtype=torch.float32, device="cuda"), B, loss)
    torch.cuda.synchronize()
    _, g = cnn.get_params()
    gg = M.unflatten_cnn(g)
    pq = {k: _bf16(v) if k.startswith("W") else v for k, v in params.items()}
    tot_loss, tot = 0.0, {k: np.zeros_like(v) for k, v in params.items()}
    for b in range(B):
        l, gr = O.cnn_loss_grad(pq, dC[b], xs[b], target[b], stats)
        tot_loss += l / B
        for k in tot:
            tot[k] += gr[k] / B
    assert abs(float(loss.item()) - tot_loss) <= 1e-3 * tot_loss
    for k in tot:
        # BF16 operands of every product: 2e-2 relative, norm-wise per tensor
        assert _rel(gg[k], tot[k]) < 2e-2, (k, _rel(gg[k], tot[k]))
    # element-wise: every gradient entry within 2e-2 of the sum of the absolute
    # values of its terms (each term a product of BF16-rounded factors, three
    # layers of rounding, ReLU masks that flip where z is within rounding of 0),
    # and within 5e-2 of the tensor's largest entry (the first layers' sums
    # cancel to ~1% of their absolute sums, so the first bound alone would not
    # see a missing or misplaced block of the partial reduction there)
    absb = _abs_grad_bounds(pq, dC, xs, target, stats)
    for k in tot:
        err = np.abs(gg[k] - tot[k])
        assert np.all(err <= 2e-2 * absb[k] + 1e-12), (k, float(np.max(err / (absb[k] + 1e-300))))
        assert np.all(err <= 5e-2 * np.max(np.abs(tot[k]))), (k, float(np.max(err) / np.max(np.abs(tot[k]))))
    cnn.close()


def _abs_grad_bounds(pq, dC, xs, target, stats):
    """Per parameter entry, the sum over samples and pixels of the absolute
    values of the terms whose sum is its gradient: the oracle's backward pass
    of the same loss run on |activations|, |weights| and |output gradients|."""
    B = dC.shape[0]
    out = {k: np.zeros_like(v) for k, v in pq.items()}
    for b in range(B):
        pred, c = O.cnn_forward(pq, dC[b], xs[b], stats)
        s_out = stats["s_out"][:, None, None]
        r = (pred - target[b]) / s_out
        dz3 = O.pixel_unshuffle4(2.0 * r / r.size) / B
        W = {k: np.abs(v) for k, v in pq.items()}
        da2, dW3, db3 = O.conv3x3_bwd(np.abs(c["a2"]), W["W3"], np.abs(dz3))
        dz2 = da2 * (c["z2"] > -1e-2 * np.abs(c["z2"]).max())
        da1, dW2, db2 = O.conv3x3_bwd(np.abs(c["a1"]), W["W2"], dz2)
        dz1 = da1 * (c["z1"] > -1e-2 * np.abs(c["z1"]).max())
        _, dW1, db1 = O.conv3x3_bwd(np.abs(c["a0"]), W["W1"], dz1, want_din=False)
        for k, v in dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3).items():
            out[k] += v
    return out


def test_adam_step_matches_oracle(M):
    import torch
    params, stats, dC, xs, target = _case(8, 1, 9)
    cnn = _gpu(M, 8, 1, params, stats)
    cnn.loss_grad(torch.tensor(dC, dtype=torch.float32, device="cuda"),
                  torch.tensor(xs, dtype=torch.float32, device="cuda"),
                  torch.tensor(target, dtype=torch.float32, device="cuda"), 1)
    cnn.adam_step(1e-3)
    torch.cuda.synchronize()
    new, g = cnn.get_params()
    p0 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}
    ref = O.adam_step(p0, M.unflatten_cnn(g), {}, lr=1e-3)
    got = M.unflatten_cnn(new)
    for k in ref:
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-5, atol=1e-6)
    cnn.close()
