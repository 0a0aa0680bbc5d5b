"""GPU parity of the Dual EnKF parameter estimation on the Burgers inlet model
(Sec. 4; Algorithm 3 with its parameter rows inside Algorithm 4) against the
CPU oracle through the C ABI: the inlet model's free run, and whole cycles
(parameters, members, fine run) on a small case and on the paper's setting
(800 fine nodes, 100 members, ratio 4, 80 sensors)."""
import numpy as np
import pytest

import oracle as O
from helpers import rel_err

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


def _pair(M, nf, r, ne, obs, dt, q, seed=0):
    L, nu, sigma = 10.0, 1 / 200, 0.05
    rng = np.random.default_rng(seed)
    theta0 = np.stack([rng.normal(0.0, 0.05, ne), rng.normal(0.3, 0.05, ne)], axis=1)
    fine0 = np.ones(nf)
    mem0 = np.ones((ne, nf // r))
    mg = O.DualMGEnKF(nf, r, L, dt, nu, fine0, mem0, theta0, [0.0, 0.3], obs, sigma, 7, q)
    g = M.DualMGEnKF(nf, r, ne, obs, L, dt, nu, sigma, q, 7)
    g.set_state(fine0, mem0, theta0, [0.0, 0.3], 0.0)
    return g, mg, rng


def _run(g, mg, rng, spin, ncyc, nsteps, obs, dt):
    L, nu, sigma, nf = 10.0, 1 / 200, 0.05, mg.nf
    truth = O.burgers_inlet_rk3(np.ones(nf), L / nf, nu, dt, spin, 0.0, [0.2, 0.0])
    mg.free_run(spin)
    g.free_run(spin)
    t = spin * dt
    for _ in range(ncyc):
        truth = O.burgers_inlet_rk3(truth, L / nf, nu, dt, nsteps, t, [0.2, 0.0])
        t += nsteps * dt
        yo = truth[obs] + sigma * rng.standard_normal(obs.size)
        mg.cycle_step(nsteps, yo)
        g.cycle(nsteps, yo)


def test_free_run_matches_oracle(M):
    obs = np.arange(1, 21)
    g, mg, _ = _pair(M, 400, 4, 12, obs, 4e-4, 1e-6)
    mg.free_run(3000)
    g.free_run(3000)
    fine, mem, th, tf = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-12
    assert rel_err(mem, mg.members) < 1e-12
    np.testing.assert_array_equal(th, mg.theta)
    g.close()


@pytest.mark.parametrize("r", [1, 4, 8])
def test_cycles_match_oracle_small(M, r):
    obs = np.arange(1, 41)
    g, mg, rng = _pair(M, 400, r, 16, obs, 4e-4, 1e-5)
    _run(g, mg, rng, 2000, 6, 30, obs, 4e-4)
    fine, mem, th, tf = g.get_state()
    assert rel_err(th, mg.theta) < 1e-10
    assert rel_err(tf, mg.theta_fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    assert rel_err(fine, mg.fine) < 1e-10
    g.close()


def test_paper_setting_matches_oracle_and_estimates_the_amplitude(M):
    obs = np.arange(1, 81)
    g, mg, rng = _pair(M, 800, 4, 100, obs, 2e-4, 1e-6)
    _run(g, mg, rng, 50000, 40, 30, obs, 2e-4)
    fine, mem, th, tf = g.get_state()
    assert rel_err(th, mg.theta) < 1e-9
    assert rel_err(fine, mg.fine) < 1e-9
    assert abs(tf[0] - 0.2) < 0.03                 # the inlet amplitude moves from 0 to the true 0.2
    g.close()


def test_invalid_configurations_are_refused(M):
    obs = np.arange(1, 11)
    bad = [dict(n_fine=2048), dict(ratio=3), dict(ratio=32), dict(n_members=1), dict(obs_sigma=0.0),
           dict(theta_q=-1.0)]
    for b in bad:
        kw = dict(n_fine=400, ratio=4, n_members=8, obs_sigma=0.05, theta_q=1e-6)
        kw.update(b)
        with pytest.raises(M.MGEnKFError):
            M.DualMGEnKF(kw["n_fine"], kw["ratio"], kw["n_members"], obs, 10.0, 4e-4, 0.005, kw["obs_sigma"],
                         kw["theta_q"], 1)
    with pytest.raises(M.MGEnKFError):
        M.DualMGEnKF(400, 4, 8, np.array([5, 400]), 10.0, 4e-4, 0.005, 0.05, 1e-6, 1)   # sensor off the grid
