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


@pytest.mark.parametrize("nc,B", [(8, 2), (20, 1)])
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
    cnn.close()


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
