"""Pins of the oracle's Burgers model (Eq. burgers, periodic, flux-form central
differences + SSP-RK3): Fourier amplification factor, Cole-Hopf convergence
and conservation of the discrete mass."""
import math
import os

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("k", [1, 3, 7, 15])
def test_linear_flux_matches_amplification_factor(k):
    # u_t + c u_x = nu u_xx on a periodic grid: every Fourier mode is an
    # eigenvector of the central operator, so one RK3 step multiplies it by
    # G(z) = 1 + z + z^2/2 + z^3/6 with z = dt * (-i c sin(k dx)/dx - 4 nu sin^2(k dx/2)/dx^2).
    n, c, nu, dt, steps = 64, 1.3, 0.02, 2e-3, 1000
    dx = 2 * math.pi / n
    x = np.arange(n) * dx
    u0 = np.cos(k * x)
    got = O.burgers_rk3(u0, dx, nu, dt, steps, flux_kind=1, c=c)
    z = dt * (-1j * c * math.sin(k * dx) / dx - 4 * nu * math.sin(k * dx / 2) ** 2 / dx**2)
    G = 1 + z + z**2 / 2 + z**3 / 6
    exact = np.real(G**steps * np.exp(1j * k * x))
    assert np.max(np.abs(got - exact)) < 1e-13 * max(1.0, np.max(np.abs(exact))) * 10


def test_nonlinear_flux_conserves_mass():
    n, nu, dt = 128, 0.01, 1e-3
    dx = 2 * math.pi / n
    x = np.arange(n) * dx
    u0 = 0.7 + np.sin(x) + 0.3 * np.cos(3 * x)
    u = O.burgers_rk3(u0, dx, nu, dt, 500)
    assert abs(u.sum() - u0.sum()) < 1e-12 * np.abs(u0).sum()
    assert not np.allclose(u, u0)


def _cole_hopf(x, t, nu, nterms=200):
    # u0 = sin x: phi0 = exp(a cos x), a = 1/(2 nu) = I0(a) + 2 sum I_n(a) cos(n x);
    # phi solves the heat equation and u = -2 nu phi_x / phi (Cole-Hopf).
    from scipy.special import ive
    a = 1.0 / (2.0 * nu)
    nn = np.arange(1, nterms + 1)[:, None]
    In = ive(nn, a) * np.exp(-nu * nn**2 * t)
    num = 2.0 * np.sum(nn * In * np.sin(nn * x[None, :]), axis=0)
    den = ive(0, a) + 2.0 * np.sum(In * np.cos(nn * x[None, :]), axis=0)
    return 2.0 * nu * num / den


def test_second_order_convergence_to_cole_hopf():
    nu, T, dt = 0.05, 0.5, 2e-4
    errs = []
    for n in (64, 128, 256):
        dx = 2 * math.pi / n
        x = np.arange(n) * dx
        u = O.burgers_rk3(np.sin(x), dx, nu, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(u - _cole_hopf(x, T, nu))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 5e-4
    for p in orders:
        assert 1.8 < p < 2.2, (errs, orders)


def test_rhs_matches_hand_computed_three_point_case():
    # n = 3: every point's neighbours are the other two points
    u = np.array([1.0, 2.0, -1.0])
    dx, nu = 0.5, 0.1
    L = O.burgers_rhs(u, dx, nu)
    # point 0: F(+1) = 2, F(-1) = 0.5 -> -(2 - 0.5)/(1.0) = -1.5 ; diffusion 0.1*(2 - 2 - 1)/0.25 = -0.4
    assert L[0] == pytest.approx(-1.9, abs=1e-15)
    # point 1: F(+1) = 0.5 (u=-1), F(-1) = 0.5 (u=1) -> 0 ; diffusion 0.1*(-1 - 4 + 1)/0.25 = -1.6
    assert L[1] == pytest.approx(-1.6, abs=1e-15)


def test_thread_count_changes_no_result():
    # the OpenMP loops run over independent problems: one thread and several
    # give the same bits (the CPU baseline times both)
    rng = np.random.default_rng(3)
    n, dx = 96, 2 * math.pi / 96
    u0 = 0.5 + 0.3 * rng.standard_normal((7, n))
    try:
        O.set_threads(1)
        one = O.burgers_rk3(u0, dx, 0.02, 1e-3, 50)
        O.set_threads(4)
        four = O.burgers_rk3(u0, dx, 0.02, 1e-3, 50)
    finally:
        O.set_threads(os.cpu_count() or 1)
    assert np.array_equal(one, four)
