"""Pins of the oracle's final fine-grid iteration (Algorithm 4 step 6: one
relaxed matrix-splitting sweep, alpha = 0.5, Sec. 3 tailoring) and of the
conservativity residual Gamma (Eq. Conservativity_rhov).

The sweep is read as one relaxed Jacobi iteration on the implicit-Euler form
of the last model step, x - dt L(x) = x_prev, started from the analysis state.
The pins do not retype that formula: an implicit solution built by a dense
solve must be a fixed point, pure diffusion of a Fourier mode must be damped
by the closed-form factor, the diagonal the sweep divides by must be the
diagonal of the right-hand side's Jacobian (by finite differences), and the
residual must shrink."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _burgers_matrix(n, dx, nu, flux_kind, c):
    # L of the linear scheme, column by column
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = O.burgers_rhs(e, dx, nu, flux_kind, c)
    return L


def test_burgers_alpha_zero_is_identity():
    rng = np.random.default_rng(0)
    x, xp = rng.standard_normal(32), rng.standard_normal(32)
    np.testing.assert_array_equal(O.burgers_sweep(x, xp, 0.1, 0.01, 1e-3, 0.0), x)


def test_burgers_implicit_solution_is_a_fixed_point():
    n, dx, nu, dt, c = 24, 2 * math.pi / 24, 0.05, 0.02, 0.7
    L = _burgers_matrix(n, dx, nu, 1, c)
    rng = np.random.default_rng(1)
    xp = rng.standard_normal(n)
    x = np.linalg.solve(np.eye(n) - dt * L, xp)        # x - dt L x = x_prev
    assert np.max(np.abs(O.burgers_gamma(x, xp, dx, nu, dt, 1, c))) < 1e-11
    np.testing.assert_allclose(O.burgers_sweep(x, xp, dx, nu, dt, 0.5, 1, c), x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_burgers_diffusion_mode_closed_form(k):
    # pure diffusion (linear flux, c = 0), x_prev = 0, x = sin(k x_j):
    # Gamma = x / dt + (4 nu / dx^2) sin^2(k dx / 2) x, so one sweep multiplies
    # x by 1 - alpha (1 + 4 s sin^2) / (1 + 2 s), s = nu dt / dx^2
    n, nu, dt, alpha = 32, 0.02, 0.5, 0.5
    dx = 2 * math.pi / n
    xj = np.arange(n) * dx
    x = np.sin(k * xj)
    s = nu * dt / dx ** 2
    th = k * dx / 2
    factor = 1 - alpha * (1 + 4 * s * math.sin(th) ** 2) / (1 + 2 * s)
    out = O.burgers_sweep(x, np.zeros(n), dx, nu, dt, alpha, 1, 0.0)
    np.testing.assert_allclose(out, factor * x, rtol=0, atol=1e-13)


def test_burgers_divisor_is_the_jacobian_diagonal():
    # the sweep divides the residual by D = diag(d Psi / dx); recover D from
    # the sweep and compare with 1 - dt dL_i/dx_i by central finite differences
    n, nu, dt = 40, 0.03, 2e-3
    dx = 2 * math.pi / n
    rng = np.random.default_rng(2)
    x = np.sin(np.arange(n) * dx) + 0.1 * rng.standard_normal(n)
    xp = x + 0.05 * rng.standard_normal(n)
    g = O.burgers_gamma(x, xp, dx, nu, dt)
    D_sweep = 0.5 * (-dt * g) / (O.burgers_sweep(x, xp, dx, nu, dt, 0.5) - x)
    eps = 1e-6
    for i in range(0, n, 7):
        e = np.zeros(n)
        e[i] = eps
        dLii = (O.burgers_rhs(x + e, dx, nu)[i] - O.burgers_rhs(x - e, dx, nu)[i]) / (2 * eps)
        assert abs(D_sweep[i] - (1 - dt * dLii)) < 1e-6 * D_sweep[i]


def test_burgers_sweep_reduces_the_residual():
    # an analysis-like jump on a forecast state: smooth profile advanced one
    # step plus a smooth correction
    n, nu, dt = 256, 0.01, 1e-3
    dx = 2 * math.pi / n
    xj = np.arange(n) * dx
    xp = np.sin(xj) + 0.3 * np.sin(3 * xj + 0.4)
    x = O.burgers_rk3(xp, dx, nu, dt, 1) + 0.05 * np.exp(-((xj - 2.0) / 0.4) ** 2)
    g0 = np.linalg.norm(O.burgers_gamma(x, xp, dx, nu, dt))
    g1 = np.linalg.norm(O.burgers_gamma(O.burgers_sweep(x, xp, dx, nu, dt, 0.5), xp, dx, nu, dt))
    assert g1 < 0.6 * g0


GAMMA, MU, PR = 1.4, 1e-3, 0.72


def _ns_state(n, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    u = 0.3 * np.sin(2 * np.pi * Y) + amp * rng.standard_normal((n, n))
    v = 0.2 * np.cos(2 * np.pi * X) + amp * rng.standard_normal((n, n))
    p = 8.0 + 0.2 * np.cos(2 * np.pi * (X + Y))
    E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E]).reshape(-1)


def test_ns2d_alpha_zero_is_identity_and_rest_state_is_fixed():
    n = 12
    q = _ns_state(n, 0)
    qp = _ns_state(n, 1)
    np.testing.assert_array_equal(O.ns2d_sweep(q, qp, 1.0 / n, GAMMA, MU, PR, 1e-3, 0.0), q)
    # a uniform state is steady: with q_prev = q the residual vanishes
    rest = np.concatenate([np.full(n * n, 1.2), np.zeros(2 * n * n), np.full(n * n, 20.0)])
    assert np.max(np.abs(O.ns2d_gamma(rest, rest, 1.0 / n, GAMMA, MU, PR, 1e-3))) < 1e-10
    np.testing.assert_allclose(O.ns2d_sweep(rest, rest, 1.0 / n, GAMMA, MU, PR, 1e-3, 0.5), rest,
                               rtol=0, atol=1e-12)


def test_ns2d_divisor_is_the_jacobian_diagonal():
    n, dt = 12, 1e-3
    h = 1.0 / n
    q = _ns_state(n, 3)
    qp = q + 1e-3 * _ns_state(n, 4)
    g = O.ns2d_gamma(q, qp, h, GAMMA, MU, PR, dt)
    D_sweep = 0.5 * (-dt * g) / (O.ns2d_sweep(q, qp, h, GAMMA, MU, PR, dt, 0.5) - q)
    plane = n * n
    eps = 1e-6
    for v in range(4):
        for p in (0, 37, 101):
            idx = v * plane + p
            e = np.zeros_like(q)
            e[idx] = eps * max(1.0, abs(q[idx]))
            dL = (O.ns2d_rhs(q + e, h, GAMMA, MU, PR)[idx] - O.ns2d_rhs(q - e, h, GAMMA, MU, PR)[idx]) / (2 * e[idx])
            assert abs(D_sweep[idx] - (1 - dt * dL)) < 1e-6 * D_sweep[idx], (v, p)


def test_ns2d_sweep_reduces_the_residual():
    n, dt = 24, 2e-3
    h = 1.0 / n
    qp = _ns_state(n, 5, amp=0.0)
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    bump = 0.02 * np.exp(-((X - 0.5) ** 2 + (Y - 0.4) ** 2) / 0.02)
    q = O.ns2d_rk3(qp, h, GAMMA, MU, PR, dt, 1)
    q[n * n:2 * n * n] += bump.reshape(-1)       # an analysis jump in rho u
    q[2 * n * n:3 * n * n] -= bump.reshape(-1)   # and in rho v
    g0 = O.ns2d_gamma(q, qp, h, GAMMA, MU, PR, dt).reshape(4, -1)
    g1 = O.ns2d_gamma(O.ns2d_sweep(q, qp, h, GAMMA, MU, PR, dt, 0.5), qp, h, GAMMA, MU, PR, dt).reshape(4, -1)
    for v in (1, 2):     # the momentum components carry the jump
        assert np.linalg.norm(g1[v]) < 0.6 * np.linalg.norm(g0[v])
    assert np.linalg.norm(g1) < 0.6 * np.linalg.norm(g0)
