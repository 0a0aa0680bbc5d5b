"""End-to-end GPU parity of the MGEnKF cycle (Algorithm 4) against the CPU
oracle: the small FP64 Burgers workload over all its cycles, and the large
mixed-precision workload at full size on its first cycle."""
import numpy as np
import pytest

from helpers import gpu_run, oracle_run, rel_err
from paper_2012_10091_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("gain_form", [0, 1])
def test_small_fp64_workload_all_cycles(gain_form):
    w = W.burgers_small()
    mg, rm_o, _ = oracle_run(w, w.cycles)
    g, rm_g, _ = gpu_run(w, w.cycles, gain_form=gain_form)
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    np.testing.assert_allclose(rm_g[:, 0], rm_o[:, 0], rtol=1e-9)
    assert rm_g[-25:, 0].mean() < 0.05
    g.close()


def test_large_mixed_workload_first_cycle_full_size():
    w = W.burgers_large()
    mg, rm_o, truth_o = oracle_run(w, 1)
    g, rm_g, truth_g = gpu_run(w, 1)
    assert rel_err(truth_g, truth_o) < 1e-12
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-3
    assert rel_err(mem, mg.members) < 1e-3
    assert abs(rm_g[0, 0] - rm_o[0, 0]) < 1e-3 * rm_o[0, 0] + 1e-4
    g.close()


def test_checkpoint_resume_is_bit_exact(tmp_path):
    w = W.burgers_custom(256, 4, 16, 10, cycles=6, obs_kind="random")
    inp = W.make_inputs(w)
    g1, _, _ = gpu_run(w, 6, inp=inp)
    a_fine, a_mem = g1.get_state()
    # run 3 cycles, save, load into a new handle, run the last 3
    import torch

    from paper_2012_10091_gb300 import mgenkf as M
    g2 = M.MGEnKF.from_workload(w)
    g2.set_state(inp["fine0"], inp["members0"])
    truth = torch.tensor(inp["truth0"], dtype=torch.float64, device="cuda")
    for k in range(6):
        M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, truth, 1, w.nf, w.length, w.dt, w.nu,
                       nsteps=w.steps_per_cycle)
        yo = W.sample_truth(w, truth.cpu().numpy(), inp["obs_idx"], inp["obs_var"]) + \
            W.observation_noise(w, k)
        if k == 3:
            path = str(tmp_path / "ck.bin")
            g2.save(path)
            g3 = M.MGEnKF.from_workload(w)
            g3.load(path)
            g2.close()
            g2 = g3
        g2.cycle(w.steps_per_cycle, yo)
        assert g2.sync() == 0
    b_fine, b_mem = g2.get_state()
    np.testing.assert_array_equal(a_fine, b_fine)
    np.testing.assert_array_equal(a_mem, b_mem)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cycle_with_host_truth_matches_separate_rmse(precision):
    # mgenkf_cycle copies a host truth beside the forecast (side stream) and
    # reads the RMSE after it: the same states and RMSE values as a cycle
    # without truth followed by mgenkf_rmse, over several cycles with a fresh
    # truth buffer each time.
    import torch
    from paper_2012_10091_gb300 import mgenkf as M
    w = W.burgers_custom(1024, 4, 16, 40, precision=precision)
    inp = W.make_inputs(w)
    ga = M.MGEnKF.from_workload(w, precision=precision)
    gb = M.MGEnKF.from_workload(w, precision=precision)
    for g in (ga, gb):
        g.set_state(inp["fine0"], inp["members0"])
    truth = torch.tensor(inp["truth0"], dtype=torch.float64, device="cuda")
    for k in range(4):
        M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, truth, 1, w.nf, w.length, w.dt, w.nu,
                       nsteps=w.steps_per_cycle)
        th = truth.cpu().numpy().copy()
        yo = W.sample_truth(w, th, inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
        ra = np.empty(w.V)
        ga.cycle(w.steps_per_cycle, yo, th, ra)
        gb.cycle(w.steps_per_cycle, yo)
        rb = gb.rmse(th)
        np.testing.assert_array_equal(ra, rb)
    for a, b in zip(ga.get_state(), gb.get_state()):
        np.testing.assert_array_equal(a, b)
    ga.close()
    gb.close()
