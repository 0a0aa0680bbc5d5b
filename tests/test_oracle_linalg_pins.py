"""Pins of small oracle routines that the larger pins use only indirectly:
the textbook Cholesky, the normalised conservativity indicator Gamma* and the
open-grid observation rows of the Dual EnKF."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_cholesky_factor_reproduces_the_matrix(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n + 3))
    A = B @ B.T + 0.5 * np.eye(n)
    st, a = O.cholesky(A)
    assert st == 0
    L = np.tril(a)
    # brute force: L L^T = A, and the factor of a library routine
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-13, atol=1e-13 * np.abs(A).max())
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)
    assert np.all(np.diag(L) > 0)


def test_cholesky_reports_the_failing_pivot():
    # leading 2 x 2 block SPD, the third pivot 4 - 1 - 4 = -1 < 0
    A = np.array([[1.0, 1.0, 0.0],
                  [1.0, 2.0, 2.0],
                  [0.0, 2.0, 4.0 - 1.0]])
    st, _ = O.cholesky(A)
    assert st == 3
    st, _ = O.cholesky(-np.eye(4))
    assert st == 1


def test_gamma_normalised_divides_by_the_largest_rate_per_variable():
    # x - x_prev = c_v dt p with max |p| = 1 on plane v: C_v = c_v and
    # Gamma* = Gamma / c_v; a plane that does not change keeps Gamma
    rng = np.random.default_rng(3)
    V, npts, dt = 3, 200, 0.01
    p = rng.uniform(-1, 1, (V, npts))
    p[:, 17] = 1.0
    c = np.array([2.0, 0.5, 0.0])
    xprev = rng.standard_normal((V, npts))
    x = xprev + c[:, None] * dt * p
    g = rng.standard_normal((V, npts))
    got = O.gamma_normalised(g, x, xprev, dt, V).reshape(V, npts)
    np.testing.assert_allclose(got[0], g[0] / 2.0, rtol=1e-12)
    np.testing.assert_allclose(got[1], g[1] / 0.5, rtol=1e-12)
    np.testing.assert_array_equal(got[2], g[2])


def test_open_observation_rows_are_the_prolongation_rows():
    # H^C on the open grid = the Pi_F row at each observed fine node
    nc, r = 25, 4
    dC = np.random.default_rng(4).standard_normal(nc)
    fine = O.open_prolong(dC, nc, r)
    obs = np.array([0, 1, 3, 4, 50, 97, nc * r - 1])
    j0, w = O.open_obs_rows(obs, nc, r)
    y = np.array([w[q] @ dC[j0[q]:j0[q] + 4] for q in range(len(obs))])
    np.testing.assert_allclose(y, fine[obs], rtol=1e-14, atol=1e-15)
    # coincident nodes are injection
    np.testing.assert_allclose(fine[::r], dC, rtol=1e-14, atol=1e-15)
