"""Pins of the oracle's centred sixth-order filter of the NS model (the paper
uses one in its Euler and Navier-Stokes runs, Secs. 5 and 6, citing Bogey and
Bailly; reading: the 7-point centred stencil with transfer function
1 - sigma sin^6(k h / 2), along x then y).  Pins: every 2-D Fourier mode is
damped by the product of the two 1-D transfer functions (closed form), the
totals of the conserved variables are kept, constants pass unchanged and the
grid-scale (odd-even) mode is removed at sigma = 1."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


@pytest.mark.parametrize("kx,ky,sigma", [(1, 0, 1.0), (3, 5, 0.7), (7, 2, 0.2), (15, 16, 1.0), (16, 16, 0.5)])
def test_fourier_mode_damping(kx, ky, sigma):
    n = 32
    h = 1.0 / n
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    q = np.zeros((4, n, n))
    for c, ph in enumerate((0.0, 0.4, 1.1, 2.0)):
        q[c] = np.cos(2 * math.pi * (kx * X + ky * Y) + ph)
    got = O.ns2d_filter6(q, sigma)
    gx = 1 - sigma * math.sin(math.pi * kx * h) ** 6
    gy = 1 - sigma * math.sin(math.pi * ky * h) ** 6
    np.testing.assert_allclose(got, q * gx * gy, rtol=0, atol=1e-14)


def test_totals_kept_constants_unchanged_grid_mode_removed():
    rng = np.random.default_rng(4)
    n = 24
    q = 1.0 + rng.standard_normal((2, 4, n, n))
    f = O.ns2d_filter6(q, 0.6)
    np.testing.assert_allclose(f.sum(axis=(2, 3)), q.sum(axis=(2, 3)), rtol=1e-13)
    assert not np.allclose(f, q)
    c = np.full((4, n, n), 3.25)
    np.testing.assert_array_equal(O.ns2d_filter6(c, 1.0), c)
    j = np.arange(n)
    odd_even = np.broadcast_to((-1.0) ** (j[:, None] + j[None, :]), (4, n, n))
    np.testing.assert_allclose(O.ns2d_filter6(odd_even + 2.0, 1.0), np.full((4, n, n), 2.0), rtol=0, atol=1e-14)


def test_low_modes_change_at_sixth_order():
    # halving the wavenumber divides the damping 1 - G by about 2^6
    # ((sin(2a) / sin(a))^6 = 64 cos^6 a)
    n = 256
    h = 1.0 / n
    X = np.arange(n) * h
    d = []
    for k in (4, 2):
        q = np.zeros((4, n, n))
        q[0] = np.cos(2 * math.pi * k * X)[None, :]
        d.append(np.max(np.abs(O.ns2d_filter6(q, 1.0) - q)))
    a = math.pi * 2 * h
    assert abs(d[0] / d[1] - 64 * math.cos(a) ** 6) < 1e-6 * 64
