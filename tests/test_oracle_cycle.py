"""Whole-cycle sanity pins of the oracle MGEnKF (Algorithm 4) on the small
Burgers workload: assimilation beats the free run, a finer coarse grid does
no worse, and r_C = 1 reduces to a plain EnKF correcting the fine run."""
import numpy as np

import oracle as O
from paper_2012_10091_gb300 import workloads as W


def run_oracle(w, cycles, assimilate=True):
    inp = W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"],
                  inp["obs_idx"], inp["obs_var"], w.sigma, w.seed, nu=w.nu)
    truth = inp["truth0"].copy()
    out = []
    for k in range(cycles):
        truth = O.burgers_rk3(truth, w.length / w.nf, w.nu, w.dt, w.steps_per_cycle)
        mg.forecast(w.steps_per_cycle)
        if assimilate:
            yo = W.sample_truth(w, truth, inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
            assert mg.analyse(yo) == 0
            mg.prolong_correct()
        out.append(mg.rmse(truth)[0])
    return np.array(out), mg


def test_assimilation_beats_free_run():
    w = W.burgers_small()
    da, _ = run_oracle(w, w.cycles)
    free, _ = run_oracle(w, w.cycles, assimilate=False)
    assert da[-25:].mean() < 0.5 * free[-25:].mean(), (da[-25:].mean(), free[-25:].mean())


def test_finer_coarse_grid_is_not_worse():
    errs = {}
    for r in (2, 8):
        w = W.burgers_custom(256, r, 32, 16, cycles=30, obs_kind="equispaced")
        da, _ = run_oracle(w, w.cycles)
        errs[r] = da[-15:].mean()
    assert errs[2] <= 1.05 * errs[8], errs


def test_ratio_one_is_plain_enkf_on_fine_run():
    w = W.burgers_custom(64, 1, 10, 6, cycles=1)
    inp = W.make_inputs(w)
    fine = O.burgers_rk3(inp["fine0"], w.length / w.nf, w.nu, w.dt, w.steps_per_cycle)
    mem = O.burgers_rk3(inp["members0"], w.length / w.nf, w.nu, w.dt, w.steps_per_cycle)
    yo = np.linspace(-1, 1, w.ny)
    eps = O.obs_perturbations(w.seed, 0, w.ne, w.ny, w.sigma)
    # r = 1: Pi_C = Pi_F = I and H^C = H^F (injection), so the corrected fine run
    # is the fine forecast plus the EnKF gain times its innovation.
    st, ma, dC = O.enkf_analyse(mem, fine, yo, eps, w.sigma, inp["obs_idx"], inp["obs_var"], 1, 1,
                                w.nf, 1, gain_form=0)
    assert st == 0
    A = (mem - mem.mean(0)).T / np.sqrt(w.ne - 1)
    H = np.zeros((w.ny, w.nf))
    H[np.arange(w.ny), inp["obs_idx"]] = 1
    K = A @ (H @ A).T @ np.linalg.inv((H @ A) @ (H @ A).T + w.sigma**2 * np.eye(w.ny))
    np.testing.assert_allclose(dC, K @ (yo - H @ fine), atol=1e-12)
    np.testing.assert_allclose(O.prolong_add(dC, fine, 1, 1, w.nf, 1), fine + dC, atol=0)
