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


# ---------------------------------------------------------------------------
# Dissipative terms (Eqs. Momentum and Energy: the viscous stresses with their
# 4/3 and -2/3 normal-stress factors and cross terms, the heat flux kappa grad T
# with kappa = mu gamma / ((gamma - 1) Pr), and the viscous work tau . u).
# Symbols of the discrete operators on a Fourier mode exp(i(a x + b y)), with
# s = sin(a h), c = sin(b h):
#   central first difference          -> i s / h
#   compact second difference (faces) -> -4 sin^2(a h / 2) / h^2
#   averaged tangential difference of a face flux, differenced across the
#   cell                              -> (i s / h)(i c / h) = -s c / h^2
# ---------------------------------------------------------------------------
P0 = 1.0 / (GAMMA * 0.3**2)


def _linear_symbol(a, b, h, mu):
    """4 x 4 matrix A with L(q_rest + eps q) = eps A q + O(eps^2) for the
    conserved perturbation q = (rho', (rho u)', (rho v)', E') of a Fourier
    mode, about rho = 1, u = v = 0, p = P0, written from the equations:
      mass:   -d_x(rho u) - d_y(rho v)
      x-mom:  -d_x p + d_x tau_xx + d_y tau_xy,  tau_xx = mu(4/3 u_x - 2/3 v_y),
              tau_xy = mu(u_y + v_x)
      y-mom:  -d_y p + d_x tau_xy + d_y tau_yy,  tau_yy = mu(4/3 v_y - 2/3 u_x)
      energy: -d_x((E + p)u) - d_y((E + p)v) + d . (tau u) + kappa lap T,
    linearised: u = (rho u)', p' = (gamma - 1) E', T' = p' - P0 rho',
    (E + p) = gamma P0 / (gamma - 1) at rest, tau . u is second order."""
    ix, iy = 1j * math.sin(a * h) / h, 1j * math.sin(b * h) / h
    dxx, dyy = -4 * math.sin(a * h / 2) ** 2 / h**2, -4 * math.sin(b * h / 2) ** 2 / h**2
    cross = ix * iy
    kappa = mu * GAMMA / ((GAMMA - 1) * PR)
    lap = dxx + dyy
    H0 = GAMMA * P0 / (GAMMA - 1)
    return np.array([
        [0, -ix, -iy, 0],
        [0, mu * (4 / 3 * dxx + dyy), mu * (-2 / 3 + 1) * cross, -(GAMMA - 1) * ix],
        [0, mu * (1 - 2 / 3) * cross, mu * (dxx + 4 / 3 * dyy), -(GAMMA - 1) * iy],
        [-kappa * P0 * lap, -H0 * ix, -H0 * iy, kappa * (GAMMA - 1) * lap],
    ], dtype=complex)


@pytest.mark.parametrize("ka,kb", [(3, 0), (3, 2), (1, 5)])
@pytest.mark.parametrize("var", [0, 1, 2, 3])
def test_linearised_operator_matches_discrete_symbol(ka, kb, var):
    # A (symmetric) central difference in eps removes the O(eps^2) terms, so
    # the oracle's right-hand side must reproduce A q_hat to O(eps^2).
    n, mu, eps = 16, 0.05, 1e-4
    h = 1.0 / n
    a, b = 2 * np.pi * ka, 2 * np.pi * kb
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    phase = np.exp(1j * (a * X + b * Y))
    rest = np.stack([np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), P0 / (GAMMA - 1) * np.ones((n, n))])
    qhat = np.zeros(4)
    qhat[var] = 1.0
    for part in (np.real, np.imag):
        dq = np.stack([qhat[k] * part(phase) for k in range(4)])
        Lp = O.ns2d_rhs(rest + eps * dq, h, GAMMA, mu, PR)
        Lm = O.ns2d_rhs(rest - eps * dq, h, GAMMA, mu, PR)
        got = (Lp - Lm) / (2 * eps)
        A = _linear_symbol(a, b, h, mu)
        expect = np.stack([part(A[k, var] * phase) for k in range(4)])
        scale = max(1.0, np.max(np.abs(A[:, var])))
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-6 * scale)


def test_linearised_symbol_separates_the_stress_factors():
    # the check above would fail for a 4/3 -> 1 or -2/3 -> 0 misreading: the
    # entries it changes are far above the tolerance used there
    h, mu = 1.0 / 16, 0.05
    a, b = 2 * np.pi * 3, 2 * np.pi * 2
    A = _linear_symbol(a, b, h, mu)
    dxx = -4 * math.sin(a * h / 2) ** 2 / h**2
    cross = -math.sin(a * h) * math.sin(b * h) / h**2
    assert abs(mu * dxx / 3) > 1e3 * 1e-6 * np.max(np.abs(A[:, 1]))
    assert abs(mu * 2 / 3 * cross) > 1e3 * 1e-6 * np.max(np.abs(A[:, 2]))


def test_heat_flux_of_density_wave_at_constant_pressure():
    # rho = 1 + 0.2 cos(a x), u = v = 0, p = P0: every inviscid and viscous term
    # vanishes exactly and the energy equation is kappa times the compact
    # second difference of T = P0 / rho (exact, not linearised)
    n, mu = 16, 0.03
    h = 1.0 / n
    x = np.arange(n) * h
    X, _ = np.meshgrid(x, x)
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * 3 * X)
    q = _state(rho, 0 * X, 0 * X, P0 + 0 * X)
    L = O.ns2d_rhs(q, h, GAMMA, mu, PR)
    T = P0 / rho
    kappa = mu * GAMMA / ((GAMMA - 1) * PR)
    lapT = (np.roll(T, -1, axis=1) - 2 * T + np.roll(T, 1, axis=1)) / h**2
    np.testing.assert_allclose(L[:3], 0 * L[:3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(L[3], kappa * lapT, rtol=1e-12, atol=1e-12 * np.max(np.abs(kappa * lapT)))


@pytest.mark.parametrize("axis", [0, 1])
def test_viscous_work_of_transverse_shear(axis):
    # v = f(x), u = 0 (or u = f(y), v = 0), rho = 1, p = P0: the inviscid terms
    # and the heat flux vanish, the only stress is tau_xy = mu (f_{i+1} - f_i)/h
    # on the faces normal to the shear gradient, the face velocity is the
    # average of the two nodes, so the energy equation is exactly
    #   (tau_xy f_face)_{i+1/2} - (...)_{i-1/2}) / h
    #   = mu (f_{i+1}^2 - 2 f_i^2 + f_{i-1}^2) / (2 h^2)
    # and the transverse momentum equation mu (f_{i+1} - 2 f_i + f_{i-1}) / h^2.
    n, mu = 16, 0.04
    h = 1.0 / n
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    rng = np.random.default_rng(7)
    f1 = 0.3 * np.sin(2 * np.pi * 2 * x + 0.4) + 0.05 * rng.standard_normal(n)
    if axis == 0:
        f = np.broadcast_to(f1[None, :], (n, n))
        q = _state(1 + 0 * X, 0 * X, f, P0 + 0 * X)
        d2 = lambda g: (np.roll(g, -1, axis=1) - 2 * g + np.roll(g, 1, axis=1)) / h**2
        mom = 2
    else:
        f = np.broadcast_to(f1[:, None], (n, n))
        q = _state(1 + 0 * X, f, 0 * X, P0 + 0 * X)
        d2 = lambda g: (np.roll(g, -1, axis=0) - 2 * g + np.roll(g, 1, axis=0)) / h**2
        mom = 1
    L = O.ns2d_rhs(q, h, GAMMA, mu, PR)
    atol = 1e-12 * np.max(np.abs(mu * d2(f)))
    np.testing.assert_allclose(L[0], 0 * f, rtol=0, atol=1e-12)
    np.testing.assert_allclose(L[3 - mom], 0 * f, rtol=0, atol=atol)
    np.testing.assert_allclose(L[mom], mu * d2(f), rtol=0, atol=atol)
    np.testing.assert_allclose(L[3], mu * d2(f * f) / 2, rtol=0, atol=atol)


def test_viscous_work_of_longitudinal_stretch():
    # u = f(x), v = 0, rho = 1, p = P0: tau_xx = 4/3 mu (f_{i+1} - f_i)/h on the
    # x-faces, tau_xy = tau_yy = 0 (the tangential derivatives of a y-independent
    # field vanish); T = P0 is uniform.  The energy equation is the central
    # difference of the inviscid flux (E + p) u plus the work term
    #   4/3 mu (f_{i+1}^2 - 2 f_i^2 + f_{i-1}^2) / (2 h^2),
    # the x-momentum equation -d_x(f^2) + 4/3 mu times the compact second
    # difference of f.
    n, mu = 16, 0.04
    h = 1.0 / n
    x = np.arange(n) * h
    X, _ = np.meshgrid(x, x)
    f = 0.2 * np.sin(2 * np.pi * X + 0.3) + 0.1 * np.cos(2 * np.pi * 3 * X)
    q = _state(1 + 0 * X, f, 0 * X, P0 + 0 * X)
    L = O.ns2d_rhs(q, h, GAMMA, mu, PR)
    E = q[3]
    cd = lambda g: (np.roll(g, -1, axis=1) - np.roll(g, 1, axis=1)) / (2 * h)
    d2 = lambda g: (np.roll(g, -1, axis=1) - 2 * g + np.roll(g, 1, axis=1)) / h**2
    scale = np.max(np.abs(cd((E + P0) * f)))
    np.testing.assert_allclose(L[0], -cd(f), rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(L[1], -cd(f * f) + 4 / 3 * mu * d2(f), rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(L[2], 0 * f, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(L[3], -cd((E + P0) * f) + 4 / 3 * mu * d2(f * f) / 2, rtol=0, atol=1e-12 * scale)
