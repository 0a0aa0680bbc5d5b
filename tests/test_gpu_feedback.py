"""GPU parity of the fine-to-coarse feedback (forecast ensemble re-centred on
the restricted fine forecast before each analysis) against the CPU oracle, and
its use inside a batch."""
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


def _runs(M, w, cycles, precision):
    inp = W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                  inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl, gain_form=1,
                  recentre=True)
    g = M.MGEnKF.from_workload(w, precision=precision)
    g.set_state(inp["fine0"], inp["members0"])
    g.set_recentre(True)
    truth = inp["truth0"].copy()
    for k in range(cycles):
        truth = mg._advance(truth, w.nf, w.steps_per_cycle)
        yo = W.sample_truth(w, truth, inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
        mg.forecast(w.steps_per_cycle)
        assert mg.analyse(yo) == 0
        mg.prolong_correct()
        g.cycle(w.steps_per_cycle, yo)
        assert g.sync() == 0
    return g, mg


@pytest.mark.parametrize("case", ["burgers", "ns2d"])
def test_fp64_matches_oracle(M, case):
    if case == "burgers":
        w, cycles = W.burgers_small(), 4
    else:
        w, cycles = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="fp64", delta=0.08), 2
    g, mg = _runs(M, w, cycles, "fp64")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    g.close()


def test_mixed_close_to_oracle(M):
    w = W.burgers_custom(1024, 4, 16, 32, steps_per_cycle=20, dt=1e-3, sigma=0.05, precision="mixed")
    g, mg = _runs(M, w, 3, "mixed")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-3
    assert rel_err(mem, mg.members) < 1e-3
    g.close()


def test_batch_applies_the_feedback(M):
    ws = W.ns2d_batch(nprob=3, seed=3, coarse=(16, 24), members=(5, 8), n_obs=(16, 32))
    inps = [W.make_inputs(w) for w in ws]
    yos = [[W.sample_truth(w, inp["truth0"], inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
            for k in range(2)] for w, inp in zip(ws, inps)]

    def runs():
        out = []
        for w, inp in zip(ws, inps):
            g = M.MGEnKF.from_workload(w, precision="mixed")
            g.set_state(inp["fine0"], inp["members0"])
            g.set_recentre(True)
            out.append(g)
        return out
    ref = []
    for j, g in enumerate(runs()):
        for k in range(2):
            g.cycle(10, yos[j][k])
        assert g.sync() == 0
        ref.append(g.get_state())
        g.close()
    b = M.Batch(runs())
    for k in range(2):
        b.cycle(10, np.concatenate([yos[j][k] for j in range(len(ws))]))
    assert b.sync() == 0
    for g, (f0, m0) in zip(b.runs, ref):
        f1, m1 = g.get_state()
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()
