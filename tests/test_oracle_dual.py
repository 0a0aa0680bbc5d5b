"""Pins of the oracle's Dual EnKF parameter estimation on the Burgers inlet
model (Sec. 4; Algorithm 3 with its parameter rows inside Algorithm 4):
the inlet model keeps a uniform state exactly and converges at second order to
the closed-form time-harmonic solution of the linearised equation; the open
projections reproduce cubics up to the ends; the estimated inlet amplitude
reaches the true 0.2 at coarsening ratio 4 (the paper reports < 2%; checked
within 4% on a time average) and is overestimated at ratio 16, as the paper
reports (0.27)."""
import cmath
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_uniform_state_with_zero_amplitude_is_steady():
    u = O.burgers_inlet_rk3(np.ones(200), 0.05, 0.005, 2e-4, 500, 0.0, [0.0, 0.7])
    np.testing.assert_array_equal(u, np.ones(200))


def test_inlet_signal_converges_to_linearised_closed_form():
    # u = u0 + u', u'_t + u0 u'_x = nu u'_xx, u'(0, t) = th1 u0 sin(omega t + th2):
    # u' = th1 u0 Im exp(i(omega t + th2 - kappa x)), nu kappa^2 - i u0 kappa + i omega = 0, Im kappa < 0
    u0, om, nu, th1, th2, T = 1.0, 2 * math.pi, 1 / 200, 1e-4, 0.3, 3.0
    disc = cmath.sqrt(-u0 ** 2 - 4j * nu * om)
    kap = [k for k in ((1j * u0 + disc) / (2 * nu), (1j * u0 - disc) / (2 * nu)) if k.imag < 0][0]
    errs = []
    for n, dt in ((400, 4e-4), (800, 2e-4), (1600, 1e-4)):
        dx = 10.0 / n
        x = np.arange(n) * dx
        u = O.burgers_inlet_rk3(np.ones(n), dx, nu, dt, int(round(T / dt)), 0.0, [th1, th2])
        exact = u0 + th1 * u0 * np.imag(np.exp(1j * (om * T + th2 - kap * x)))
        m = (x >= 0.2) & (x <= 1.0)
        errs.append(np.abs(u[m] - exact[m]).max() / th1)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[2] < 2e-3


def test_open_prolongation_reproduces_cubics_to_the_ends():
    nc, r = 12, 4
    c = lambda s: 0.3 + 0.1 * s - 0.02 * s ** 2 + 0.003 * s ** 3
    f = O.open_prolong(c(np.arange(nc, dtype=float)), nc, r)
    np.testing.assert_allclose(f, c(np.arange(nc * r) / r), rtol=0, atol=1e-13)
    np.testing.assert_allclose(f[::r], c(np.arange(nc, dtype=float)), rtol=0, atol=1e-14)  # Pi_C Pi_F = I


def _estimate(r, ncyc, seed=0):
    nf, L, dt, nu, ne, sigma = 800, 10.0, 2e-4, 1 / 200, 100, 0.05
    rng = np.random.default_rng(seed)
    theta0 = np.stack([rng.normal(0.0, 0.05, ne), rng.normal(0.3, 0.05, ne)], axis=1)
    obs = np.arange(1, 81)                       # 80 sensors on (0, 1]
    truth = O.burgers_inlet_rk3(np.ones(nf), L / nf, nu, dt, 50000, 0.0, [0.2, 0.0])
    mg = O.DualMGEnKF(nf, r, L, dt, nu, np.ones(nf), np.ones((ne, nf // r)), theta0, [0.0, 0.3], obs,
                      sigma, 7, 1e-6)
    mg.free_run(50000)                           # the flow develops up to t = 10
    t, th1 = 10.0, []
    for _ in range(ncyc):
        truth = O.burgers_inlet_rk3(truth, L / nf, nu, dt, 30, t, [0.2, 0.0])
        t += 30 * dt
        th1.append(mg.cycle_step(30, truth[obs] + sigma * rng.standard_normal(obs.size))[:, 0].mean())
    return np.array(th1)


def test_amplitude_estimate_within_two_percent_at_ratio_4_and_high_at_16():
    th4 = _estimate(4, 300)
    # the paper reports < 2% at r = 4; here the mean over the last 100 cycles
    # must be within 4% (the random walk keeps a spread of about 0.006)
    assert abs(th4[-100:].mean() - 0.2) < 0.008
    th16 = _estimate(16, 300)
    assert th16[-100:].mean() > 0.24                       # paper: overestimated (0.27) at r = 16
