"""GPU parity of the final fine-grid iteration (Algorithm 4 step 6: one relaxed
Jacobi sweep of the implicit last model step, alpha = 0.5) and of the
conservativity residual Gamma (Eq. Conservativity_rhov) against the CPU oracle,
through the C ABI, for both models and both precisions."""
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


def _runs(M, w, cycles, alpha, precision):
    """GPU and oracle runs of `cycles` analyses with the final fine iteration;
    the truth and observations come from the oracle's truth run."""
    inp = W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                  inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl, gain_form=1,
                  alpha=alpha)
    g = M.MGEnKF.from_workload(w, precision=precision)
    g.set_state(inp["fine0"], inp["members0"])
    g.set_regularisation(alpha)
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


@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_burgers_fp64_matches_oracle(M, alpha):
    w = W.burgers_small()
    g, mg = _runs(M, w, 4, alpha, "fp64")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    gam = g.gamma_residual()
    ref = mg.gamma_residual()
    assert rel_err(gam, ref) < 1e-6     # a difference quotient over one step: 1e-16 / (dt L) digits lost
    g.close()


def test_ns2d_fp64_matches_oracle(M):
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="fp64", delta=0.08)
    g, mg = _runs(M, w, 2, 0.5, "fp64")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    gam, ref = g.gamma_residual().reshape(4, -1), mg.gamma_residual().reshape(4, -1)
    for v in range(4):
        assert rel_err(gam[v], ref[v]) < 1e-5, v
    g.close()


@pytest.mark.parametrize("model", ["burgers", "ns2d"])
def test_mixed_close_to_oracle(M, model):
    if model == "burgers":
        w = W.burgers_custom(1024, 4, 16, 32, steps_per_cycle=20, dt=1e-3, sigma=0.05, precision="mixed")
    else:
        w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="mixed", delta=0.08)
    g, mg = _runs(M, w, 2, 0.5, "mixed")
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-3
    assert rel_err(mem, mg.members) < 1e-3
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_reduces_the_conservativity_residual(M, precision):
    """Same inputs, one cycle, alpha = 0 (recorded, no sweep) against 0.5."""
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=1, precision=precision, delta=0.08)
    norms = {}
    for alpha in (0.0, 0.5):
        g, _ = _runs(M, w, 1, alpha, precision)
        norms[alpha] = np.linalg.norm(g.gamma_residual().reshape(4, -1)[1:3])
        g.close()
    assert norms[0.5] < 0.6 * norms[0.0]


def test_recording_off_and_bad_alpha(M):
    w = W.burgers_small()
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, precision="fp64")
    g.set_state(inp["fine0"], inp["members0"])
    g.forecast(5)
    with pytest.raises(M.MGEnKFError):        # nothing recorded
        g.gamma_residual()
    for bad in (1.5, float("nan")):
        with pytest.raises(M.MGEnKFError):
            g.set_regularisation(bad)
    g.set_regularisation(0.0)
    g.forecast(5)
    assert np.all(np.isfinite(g.gamma_residual()))
    g.set_regularisation(-1.0)                 # off again
    with pytest.raises(M.MGEnKFError):
        g.gamma_residual()
    g.close()


def test_batches_refuse_regularised_handles(M):
    ws = W.ns2d_batch(nprob=2, seed=3, coarse=(16, 24), members=(5, 8), n_obs=(16, 32))
    runs = []
    for w in ws:
        inp = W.make_inputs(w)
        g = M.MGEnKF.from_workload(w, precision="mixed")
        g.set_state(inp["fine0"], inp["members0"])
        runs.append(g)
    runs[1].set_regularisation(0.5)
    with pytest.raises(M.MGEnKFError):
        M.Batch(runs)
    for g in runs:
        g.close()


@pytest.mark.parametrize("model", ["burgers", "ns2d"])
def test_normalised_gamma_matches_oracle(M, model):
    """Gamma* = Gamma / max |(x - x_prev)/dt| (the paper's normalisation of its
    conservativity maps), formed by the library (MGENKF_FIELD_GAMMA_NORM), and
    the rate field itself, FP64, against the oracle."""
    if model == "burgers":
        w = W.burgers_small()
    else:
        w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=2, precision="fp64", delta=0.08)
    g, mg = _runs(M, w, 2, 0.0, "fp64")
    rate = g.state_rate()
    assert rel_err(rate, (mg.fine - mg.fine_prev) / w.dt) < 1e-7   # difference quotient over one step
    got = g.gamma_normalised().reshape(w.V, -1)
    ref = O.gamma_normalised(mg.gamma_residual(), mg.fine, mg.fine_prev, w.dt, w.V).reshape(w.V, -1)
    for v in range(w.V):
        assert rel_err(got[v], ref[v]) < 1e-5, v
    g.close()
