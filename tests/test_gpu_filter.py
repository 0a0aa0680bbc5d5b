"""GPU parity of the centred sixth-order filter of the NS model (the paper's
Euler and NS runs use one, Secs. 5 and 6) against the CPU oracle through the C
ABI: whole MGEnKF cycles with the filter after every model step, both
precisions; the filter removes grid-scale content; invalid uses are refused."""
import numpy as np
import pytest

import oracle as O
from helpers import rel_err
from paper_2012_10091_gb300 import workloads as W

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


def _runs(M, w, cycles, sigma, precision):
    inp = W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                  inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl, gain_form=1,
                  filter_sigma=sigma)
    g = M.MGEnKF.from_workload(w, precision=precision)
    g.set_state(inp["fine0"], inp["members0"])
    g.set_filter(sigma)
    truth = inp["truth0"].copy()
    for k in range(cycles):
        truth = mg._advance(truth, w.nf, w.steps_per_cycle)
        yo = W.sample_truth(w, truth, inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
        mg.forecast(w.steps_per_cycle)
        assert mg.analyse(yo) == 0
        mg.prolong_correct()
        g.forecast(w.steps_per_cycle)
        g.analyse(yo)
        g.prolong_correct()
        assert g.sync() == 0
    return g, mg


@pytest.mark.parametrize("sigma", [0.2, 1.0])
def test_fp64_matches_oracle(M, sigma):
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="fp64", delta=0.08)
    g, mg = _runs(M, w, 2, sigma, "fp64")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    g.close()


def test_mixed_close_to_oracle(M):
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="mixed", delta=0.08)
    g, mg = _runs(M, w, 2, 0.5, "mixed")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-3
    assert rel_err(mem, mg.members) < 1e-3
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_removes_grid_scale_content(M, precision):
    w = W.ns2d_shear(nf=64, ratio=4, ne=8, n_probes=20, cycles=1, precision=precision, delta=0.08)
    inp = W.make_inputs(w)
    n = w.nf
    j = np.arange(n)
    cb = (-1.0) ** (j[:, None] + j[None, :])
    fine0 = inp["fine0"].reshape(4, n, n).copy()
    fine0[1] += 1e-3 * cb                      # a grid-scale (odd-even) mode in rho u
    content = {}
    for sigma in (0.0, 1.0):
        g = M.MGEnKF.from_workload(w, precision=precision)
        g.set_state(fine0.reshape(-1), inp["members0"])
        g.set_filter(sigma)
        g.forecast(1)
        assert g.sync() == 0
        fine, _ = g.get_state()
        content[sigma] = abs(float(np.sum(fine.reshape(4, n, n)[1] * cb))) / n ** 2
        g.close()
    assert content[0.0] > 5e-4                 # one RK3 step keeps most of it
    assert content[1.0] < 1e-3 * content[0.0]  # sigma = 1 removes it (transfer 1 - sin^6(pi/2) = 0)


def test_invalid_uses_are_refused(M):
    wb = W.burgers_small()
    gb = M.MGEnKF.from_workload(wb, precision="fp64")
    with pytest.raises(M.MGEnKFError):
        gb.set_filter(0.5)                     # the filter belongs to the NS model
    gb.close()
    ws = W.ns2d_batch(nprob=2, seed=3, coarse=(16, 24), members=(5, 8), n_obs=(16, 32))
    runs = []
    for w in ws:
        inp = W.make_inputs(w)
        g = M.MGEnKF.from_workload(w, precision="mixed")
        g.set_state(inp["fine0"], inp["members0"])
        runs.append(g)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(M.MGEnKFError):
            runs[0].set_filter(bad)
    runs[1].set_filter(0.3)
    with pytest.raises(M.MGEnKFError):
        M.Batch(runs)                          # not available in batches
    runs[1].set_filter(0.0)
    b = M.Batch(runs)
    b.close()
    for g in runs:
        g.close()
