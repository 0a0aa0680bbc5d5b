"""Pins of the oracle's 2-D compressible NS model (Eqs. Mass, Momentum, Energy,
periodic, central inviscid fluxes, face-centred viscous/heat fluxes, SSP-RK3):
conservation, uniform-state and symmetry invariants, and the exact discrete
evolution of small-amplitude acoustic and shear modes."""
import math

import numpy as np
import pytest

import oracle as O

GAMMA, PR = 1.4, 0.72


def _state(rho, u, v, p):
    E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def _random_smooth_state(n, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(n) * (1.0 / n)
    X, Y = np.meshgrid(x, x)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * X + rng.uniform(0, 6)) * np.cos(2 * np.pi * Y)
    u = 0.3 * np.sin(2 * np.pi * Y + rng.uniform(0, 6)) + 0.01 * rng.standard_normal((n, n))
    v = 0.2 * np.cos(2 * np.pi * X) + 0.01 * rng.standard_normal((n, n))
    p = 8.0 + 0.2 * np.cos(2 * np.pi * (X + Y))
    return _state(rho, u, v, p)


def test_totals_are_conserved():
    n = 24
    q0 = _random_smooth_state(n, 0)
    q = O.ns2d_rk3(q0, 1.0 / n, GAMMA, 1e-2, PR, 5e-4, 30)
    for k in range(4):
        assert abs(q[k].sum() - q0[k].sum()) < 1e-12 * np.abs(q0[k]).sum(), k
    assert np.max(np.abs(q - q0)) > 1e-4


def test_uniform_state_is_steady():
    n = 8
    one = np.ones((n, n))
    q0 = _state(1.3 * one, 0.4 * one, -0.2 * one, 7.0 * one)
    L = O.ns2d_rhs(q0, 1.0 / n, GAMMA, 1e-2, PR)
    assert np.max(np.abs(L)) < 1e-12


def test_transpose_symmetry():
    n = 16
    q0 = _random_smooth_state(n, 1)
    qt = np.stack([q0[0].T, q0[2].T, q0[1].T, q0[3].T])
    a = O.ns2d_rk3(q0, 1.0 / n, GAMMA, 1e-2, PR, 5e-4, 10)
    b = O.ns2d_rk3(qt, 1.0 / n, GAMMA, 1e-2, PR, 5e-4, 10)
    bt = np.stack([b[0].T, b[2].T, b[1].T, b[3].T])
    np.testing.assert_allclose(a, bt, rtol=0, atol=1e-13)


def test_acoustic_mode_follows_discrete_dispersion():
    # inviscid linear acoustics about rho=1, u=0, p=p0: the central operator
    # maps a right-running wave cos(kx) to the pair with eigenvalue
    # -i c sin(kh)/h, so RK3 multiplies it by G(z), z = -i dt c sin(kh)/h.
    n, k, eps = 32, 2 * np.pi * 3, 1e-7
    h = 1.0 / n
    p0 = 1.0 / (GAMMA * 0.3**2)
    c = math.sqrt(GAMMA * p0)
    x = np.arange(n) * h
    X, _ = np.meshgrid(x, x)
    dt, steps = 2e-4, 200
    q0 = _state(1.0 + eps * np.cos(k * X), c * eps * np.cos(k * X), 0 * X, p0 + c * c * eps * np.cos(k * X))
    q = O.ns2d_rk3(q0, h, GAMMA, 0.0, PR, dt, steps)
    z = -1j * dt * c * math.sin(k * h) / h
    G = 1 + z + z * z / 2 + z**3 / 6
    expect = 1.0 + eps * np.real(G**steps * np.exp(1j * k * X))
    assert np.max(np.abs(q[0] - expect)) < 1e-4 * eps


def test_shear_mode_decays_with_compact_laplacian():
    # v = eps sin(kx), u = 0: to first order d v/dt = mu * D2 v with the compact
    # second difference (eigenvalue -4 sin^2(kh/2)/h^2), other terms O(eps^2).
    n, k, eps, mu = 32, 2 * np.pi * 2, 1e-6, 0.05
    h = 1.0 / n
    x = np.arange(n) * h
    X, _ = np.meshgrid(x, x)
    dt, steps = 1e-4, 300
    q0 = _state(1.0 + 0 * X, 0 * X, eps * np.sin(k * X), 8.0 + 0 * X)
    q = O.ns2d_rk3(q0, h, GAMMA, mu, PR, dt, steps)
    z = -dt * mu * 4 * math.sin(k * h / 2) ** 2 / h**2
    G = 1 + z + z * z / 2 + z**3 / 6
    np.testing.assert_allclose(q[2] / q[0], eps * G**steps * np.sin(k * X), rtol=0, atol=1e-9 * eps)
