"""Pins of the oracle's fine-to-coarse feedback (the paper's conclusion names
projecting the fine run's information onto the ensemble as the next step):
the forecast ensemble is re-centred on the restricted fine forecast x^C*
before each analysis.  Pins: the re-centred mean is x^C*, the anomalies are
untouched, and - since H^C is linear - the analysed ensemble mean equals
x^C' + K mean(eps) with K computed here by dense linear algebra."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2012_10091_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_recentre_moves_the_mean_and_keeps_the_anomalies():
    rng = np.random.default_rng(0)
    ne, nx = 9, 50
    m = rng.standard_normal((ne, nx)) * 0.3 + 1.0
    xs = rng.standard_normal(nx)
    r = O.recentre(m, xs)
    np.testing.assert_allclose(r.mean(axis=0), xs, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r - r.mean(axis=0), m - m.mean(axis=0), rtol=0, atol=1e-14)


def test_analysed_mean_is_corrected_state_plus_gain_times_mean_perturbation():
    w = W.burgers_custom(256, 4, 12, 20, sigma=0.1, obs_kind="random")
    inp = W.make_inputs(w)
    mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                  inp["obs_var"], w.sigma, w.seed, nu=w.nu, gain_form=1, recentre=True)
    mg.forecast(w.steps_per_cycle)
    xs = O.restrict(mg.fine, 1, 1, w.nc, w.ratio)
    mf = O.recentre(mg.members, xs)                 # the forecast ensemble the analysis will see
    rng = np.random.default_rng(1)
    yo = W.sample_truth(w, inp["truth0"], inp["obs_idx"], inp["obs_var"]) + 0.1 * rng.standard_normal(w.ny)
    eps = 0.1 * rng.standard_normal((w.ne, w.ny))
    assert mg.analyse(yo, eps) == 0
    # dense gain of the re-centred forecast ensemble, exact R = sigma^2 I
    H = np.stack([O.obs_coarse(e, 1, 1, w.nc, w.ratio, inp["obs_idx"], inp["obs_var"])
                  for e in np.eye(w.nc)], axis=1)
    X = (mf - mf.mean(axis=0)).T / math.sqrt(w.ne - 1)
    Y = H @ X
    K = X @ Y.T @ np.linalg.inv(Y @ Y.T + w.sigma ** 2 * np.eye(w.ny))
    np.testing.assert_allclose(mg.xstar, xs, rtol=0, atol=1e-15)
    expect = xs + mg.dC + K @ eps.mean(axis=0)
    np.testing.assert_allclose(mg.members.mean(axis=0), expect, rtol=0, atol=1e-12)
    # and dC itself is K d* with d* = y^o - H x^C*
    np.testing.assert_allclose(mg.dC, K @ (yo - H @ xs), rtol=0, atol=1e-12)
