"""Training data and training loop of the learned prolongation correction.

The paper's conclusion names better projection operators between the two
grids as a way forward.  Here the correction applied to the fine run,
Pi_F(dC) (Algorithm 4 step 5), gets a learned residual: a small CNN
(``mgenkf.CNN``) maps the coarse analysis fields [dC, x^C*] to the part of the
fine correction that a full-resolution EnKF would apply and Pi_F(dC) misses.

Training pairs come from two runs advanced in lockstep on the same truth,
observations and observation perturbations:

* A: the MGEnKF (members on the coarse grid, ratio 4);
* B: an EnKF with the members on the fine grid (ratio 1).  Before each
  analysis B's fine run is set to A's fine forecast, so B's coarse correction
  (its grid is the fine grid) is K_full (y^o - H^F x^F,f_A): the correction a
  full-resolution EnKF applies to A's forecast.

Each analysis gives one pair: input (dC, x^C*) of A, target dC of B.
Everything runs through the C ABI; torch only holds the device buffers.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import mgenkf as M
from . import workloads as W


def generate_pairs(w: W.Workload, cycles: int, stream=None):
    """Run A (w, ratio 4) and B (ratio 1) for `cycles` analyses; returns a dict
    of device FP32 tensors dC (n x 4 x nc x nc), xs (same), target
    (n x 4 x nf x nf), and the RMSE of A's fine run per cycle."""
    import torch
    assert w.model == W.NS2D and w.ratio == 4
    wB = dataclasses.replace(w, ratio=1)
    inA, inB = W.make_inputs(w), W.make_inputs(wB)
    A = M.MGEnKF.from_workload(w, precision="mixed", stream=stream)
    B = M.MGEnKF.from_workload(wB, precision="mixed", stream=stream)
    A.set_state(inA["fine0"], inA["members0"])
    B.set_state(inA["fine0"], inB["members0"])
    nc, nf = w.nc, w.nf
    dev = "cuda"
    truth = torch.tensor(inA["truth0"], dtype=torch.float64, device=dev)
    fine64 = torch.empty(w.nxf, dtype=torch.float64, device=dev)
    eps = torch.empty(w.ne * w.ny, dtype=torch.float64, device=dev)
    c64 = torch.empty((4, nc, nc), dtype=torch.float64, device=dev)   # FP64 staging of one pair
    t64 = torch.empty((4, nf, nf), dtype=torch.float64, device=dev)
    dC = torch.empty((cycles, 4, nc, nc), dtype=torch.float32, device=dev)
    xs = torch.empty_like(dC)
    tgt = torch.empty((cycles, 4, nf, nf), dtype=torch.float32, device=dev)
    rm = np.empty(cycles)
    out = np.empty(4)
    for k in range(cycles):
        M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_FP64, truth, 1, nf, w.length, w.dt, w.nu, w.gamma,
                       w.prandtl, nsteps=w.steps_per_cycle, stream=stream)
        A.forecast(w.steps_per_cycle)
        B.forecast(w.steps_per_cycle)
        yo = W.sample_truth(w, truth.cpu().numpy(), inA["obs_idx"], inA["obs_var"]) + \
            W.observation_noise(w, k)
        A.analyse(yo)
        M.mgenkf_get_field(A.h, M.MGENKF_FIELD_EPS, eps, eps.numel())
        M.mgenkf_get_state(A.h, fine64, None)
        M.mgenkf_set_state(B.h, fine64, None)
        B.analyse(yo, eps)
        M.mgenkf_get_field(A.h, M.MGENKF_FIELD_DC, c64, c64.numel())
        dC[k].copy_(c64)
        M.mgenkf_get_field(A.h, M.MGENKF_FIELD_XSTAR, c64, c64.numel())
        xs[k].copy_(c64)
        M.mgenkf_get_field(B.h, M.MGENKF_FIELD_DC, t64, t64.numel())
        tgt[k].copy_(t64)
        A.prolong_correct()
        M.mgenkf_rmse(A.h, truth, out)
        rm[k] = out[2]
        sa, sb = A.sync(), B.sync()
        if sa or sb:
            raise RuntimeError(f"analysis {k}: device status {sa} (coarse-member run), {sb} (fine-member run)")
    A.close()
    B.close()
    return dict(dC=dC, xs=xs, target=tgt, rmse=rm)


def run_cycles(w: W.Workload, cycles: int, cnn=None, stream=None):
    """MGEnKF run of `cycles` analyses with plain prolongation (cnn None) or
    with the learned correction; returns the per-cycle RMSE of the fine run
    (4 variables) against an FP64 truth run."""
    import torch
    inp = W.make_inputs(w)
    A = M.MGEnKF.from_workload(w, precision="mixed", stream=stream)
    A.set_state(inp["fine0"], inp["members0"])
    if cnn is not None:
        A.set_prolong_cnn(cnn)
    truth = torch.tensor(inp["truth0"], dtype=torch.float64, device="cuda")
    rm = np.empty((cycles, 4))
    for k in range(cycles):
        M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_FP64, truth, 1, w.nf, w.length, w.dt, w.nu, w.gamma,
                       w.prandtl, nsteps=w.steps_per_cycle, stream=stream)
        yo = W.sample_truth(w, truth.cpu().numpy(), inp["obs_idx"], inp["obs_var"]) + \
            W.observation_noise(w, k)
        A.cycle(w.steps_per_cycle, yo, truth, rm[k])
        assert A.sync() == 0
    A.close()
    return rm


def _stats(pairs, idx):
    import torch
    x = torch.cat([pairs["dC"][idx], pairs["xs"][idx]], dim=1)          # n x 8 x nc x nc
    mu = x.mean(dim=(0, 2, 3)).double().cpu().numpy()
    s_in = x.std(dim=(0, 2, 3)).double().cpu().numpy()
    s_out = pairs["target"][idx].std(dim=(0, 2, 3)).double().cpu().numpy()
    s_in = np.where(s_in > 0, s_in, 1.0)
    s_out = np.where(s_out > 0, s_out, 1.0)
    return dict(mu_in=mu, s_in=s_in, s_out=s_out)


def init_params(seed=0):
    """He-normal W1, W2; zero W3 and biases, so the untrained network adds
    nothing to Pi_F(dC)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in M.CNN_SHAPES:
        if k in ("W1", "W2"):
            fan_in = shp[1] * 9
            p[k] = rng.standard_normal(shp) * math.sqrt(2.0 / fan_in)
        else:
            p[k] = np.zeros(shp)
    return p


def _mean_loss(cnn, pairs, idx, batch, loss_buf):
    tot, cnt = 0.0, 0
    for s in range(0, len(idx), batch):
        b = idx[s:s + batch]
        cnn.loss_grad(pairs["dC"][b].contiguous(), pairs["xs"][b].contiguous(),
                      pairs["target"][b].contiguous(), len(b), loss_buf)
        tot += float(loss_buf.item()) * len(b)
        cnt += len(b)
    return tot / max(cnt, 1)


def concat_pairs(*sets):
    import torch
    return {k: (torch.cat([s[k] for s in sets]) if k != "rmse" else np.concatenate([s[k] for s in sets]))
            for k in sets[0]}


def fit(pairs, epochs=20, batch=8, lr=1e-3, val_frac=0.2, seed=0, val_pairs=None):
    """Train on the pairs (all of them if val_pairs is given, else the first
    1 - val_frac); returns (cnn, stats, history) with the validation loss of
    the CNN per epoch and that of plain prolongation."""
    import torch
    if val_pairs is not None:
        n_tr = pairs["dC"].shape[0]
        pairs = concat_pairs(pairs, val_pairs)
        n = pairs["dC"].shape[0]
        nval = n - n_tr
    else:
        n = pairs["dC"].shape[0]
        nval = max(1, int(round(val_frac * n)))
    nc = pairs["dC"].shape[-1]
    tr = torch.arange(0, n - nval, device="cuda")
    va = torch.arange(n - nval, n, device="cuda")
    stats = _stats(pairs, tr)
    cnn = M.CNN(nc, batch)
    cnn.set_params(init_params(seed), stats)
    plain = M.CNN(nc, batch)
    plain.set_params({k: np.zeros(s) for k, s in M.CNN_SHAPES}, stats)
    loss_buf = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = dict(train=[], val=[], val_plain=_mean_loss(plain, pairs, va, batch, loss_buf))
    for ep in range(epochs):
        perm = tr[torch.randperm(len(tr), generator=g).to("cuda")]
        tl, cnt = 0.0, 0
        for s in range(0, len(perm) - batch + 1, batch):
            b = perm[s:s + batch]
            cnn.loss_grad(pairs["dC"][b].contiguous(), pairs["xs"][b].contiguous(),
                          pairs["target"][b].contiguous(), batch, loss_buf)
            cnn.adam_step(lr)
            tl += float(loss_buf.item())
            cnt += 1
        hist["train"].append(tl / max(cnt, 1))
        hist["val"].append(_mean_loss(cnn, pairs, va, batch, loss_buf))
    plain.close()
    return cnn, stats, hist
