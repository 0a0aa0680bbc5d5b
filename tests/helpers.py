"""Shared drivers of the parity tests: run the same seeded workload through
the CPU oracle and through the GPU library (each side computes its own truth
run and observations; only the seeded inputs of ``workloads`` are shared)."""
import numpy as np

import oracle as O
from paper_2012_10091_gb300 import workloads as W


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def oracle_run(w, cycles, gain_form=1, inp=None, eps_fn=None):
    """FP64 oracle MGEnKF; returns (oracle object, rmse per cycle)."""
    inp = inp or W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"],
                  inp["obs_idx"], inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma,
                  prandtl=w.prandtl, gain_form=gain_form)
    truth = inp["truth0"].copy()
    rm = []
    for k in range(cycles):
        truth = mg._advance(truth, w.nf, w.steps_per_cycle)
        mg.forecast(w.steps_per_cycle)
        yo = W.sample_truth(w, truth, inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
        assert mg.analyse(yo, None if eps_fn is None else eps_fn(k)) == 0
        mg.prolong_correct()
        rm.append(mg.rmse(truth))
    return mg, np.array(rm), truth


def gpu_run(w, cycles, gain_form=0, precision=None, inp=None, eps_fn=None):
    """GPU MGEnKF through the C ABI; returns (handle, rmse per cycle, truth)."""
    import torch

    from paper_2012_10091_gb300 import mgenkf as M
    inp = inp or W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, gain_form=gain_form, precision=precision)
    g.set_state(inp["fine0"], inp["members0"])
    model = M.MGENKF_BURGERS1D if w.model == W.BURGERS1D else M.MGENKF_NS2D
    truth = torch.tensor(inp["truth0"], dtype=torch.float64, device="cuda")
    rm = []
    for k in range(cycles):
        M.mgk_forecast(model, M.MGENKF_FP64, truth, 1, w.nf, w.length, w.dt, w.nu, w.gamma,
                       w.prandtl, nsteps=w.steps_per_cycle)
        yo = W.sample_truth(w, truth.cpu().numpy(), inp["obs_idx"], inp["obs_var"]) + \
            W.observation_noise(w, k)
        out = np.empty(w.V)
        if eps_fn is None:
            g.cycle(w.steps_per_cycle, yo, truth, out)
        else:
            g.forecast(w.steps_per_cycle)
            g.analyse(yo, eps_fn(k))
            g.prolong_correct()
            out = g.rmse(truth)
        assert g.sync() == 0
        rm.append(out)
    return g, np.array(rm), truth.cpu().numpy()
