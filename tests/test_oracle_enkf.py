"""Pins of the oracle's EnKF analysis (Sec. 2.1.2, Algorithm 1, Algorithm 3
state part) and of the multigrid correction (Algorithm 4 step 5): brute force
against dense matrices built with numpy, the Kalman-filter limit, and the
limits of huge and vanishing observation noise."""
import math

import numpy as np
import pytest

import oracle as O


def _cubic_weights(s):
    # closed form of the 4-point Lagrange weights on nodes -1, 0, 1, 2
    return np.array([-s * (s - 1) * (s - 2) / 6, (s + 1) * (s - 1) * (s - 2) / 2,
                     -(s + 1) * s * (s - 2) / 2, (s + 1) * s * (s - 1) / 6])


def _dense_H(nc, r, idx):
    H = np.zeros((len(idx), nc))
    for j, f in enumerate(idx):
        J, s = f // r, (f % r) / r
        for t, w in enumerate(_cubic_weights(s)):
            H[j, (J - 1 + t) % nc] += w
    return H


def _problem(nc, r, ne, ny, seed, sigma=0.3):
    rng = np.random.default_rng(seed)
    members = rng.standard_normal((ne, nc)) * 0.5 + np.sin(np.arange(nc))
    xstar = rng.standard_normal(nc)
    idx = np.sort(rng.choice(nc * r, size=ny, replace=False)).astype(np.int32)
    var = np.zeros(ny, np.int32)
    yo = rng.standard_normal(ny)
    eps = sigma * rng.standard_normal((ne, ny))
    return members, xstar, idx, var, yo, eps, sigma


def _brute_force(members, xstar, idx, yo, eps, sigma, nc, r, R=None):
    ne = members.shape[0]
    H = _dense_H(nc, r, idx)
    xbar = members.mean(0)
    A = (members - xbar).T / math.sqrt(ne - 1)           # X, nx x ne
    P = A @ A.T                                          # P^e = X X^T
    if R is None:
        R = sigma**2 * np.eye(len(idx))
    K = P @ H.T @ np.linalg.inv(H @ P @ H.T + R)
    ma = members + (K @ (yo[:, None] + eps.T - H @ members.T)).T
    dC = K @ (yo - H @ xstar)
    return ma, dC, K


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("nc,r,ne,ny", [(12, 1, 6, 5), (16, 4, 9, 7), (10, 3, 16, 13)])
def test_analysis_matches_brute_force(form, nc, r, ne, ny):
    m, xs, idx, var, yo, eps, sigma = _problem(nc, r, ne, ny, seed=nc + ne)
    st, ma, dC = O.enkf_analyse(m, xs, yo, eps, sigma, idx, var, 1, 1, nc, r, gain_form=form)
    assert st == 0
    ma_bf, dC_bf, _ = _brute_force(m, xs, idx, yo, eps, sigma, nc, r)
    np.testing.assert_allclose(ma, ma_bf, rtol=0, atol=1e-12)
    np.testing.assert_allclose(dC, dC_bf, rtol=0, atol=1e-12)


def test_sample_observation_covariance_form_matches_brute_force():
    nc, r, ne, ny = 14, 2, 12, 5          # ny <= 2 (ne - 1): E E^T + Y Y^T is SPD
    m, xs, idx, var, yo, eps, sigma = _problem(nc, r, ne, ny, seed=5)
    E = (eps - eps.mean(0)).T / math.sqrt(ne - 1)
    st, ma, dC = O.enkf_analyse(m, xs, yo, eps, sigma, idx, var, 1, 1, nc, r, gain_form=2)
    assert st == 0
    ma_bf, dC_bf, _ = _brute_force(m, xs, idx, yo, eps, sigma, nc, r, R=E @ E.T)
    np.testing.assert_allclose(ma, ma_bf, atol=1e-11)
    np.testing.assert_allclose(dC, dC_bf, atol=1e-11)


def test_gain_matches_brute_force_general_H():
    rng = np.random.default_rng(7)
    nx, ne, ny = 13, 7, 5
    X = rng.standard_normal((nx, ne))
    H = rng.standard_normal((ny, nx))
    Y = H @ X
    R = np.diag(rng.uniform(0.1, 1.0, ny))
    st, K = O.enkf_gain(X, Y, R)
    assert st == 0
    P = X @ X.T
    np.testing.assert_allclose(K, P @ H.T @ np.linalg.inv(H @ P @ H.T + R), atol=1e-12)


def test_singular_innovation_matrix_is_reported():
    nc, r, ne, ny = 16, 1, 4, 10          # rank(Y Y^T) <= 3 < 10 and R = 0
    m, xs, idx, var, yo, eps, _ = _problem(nc, r, ne, ny, seed=9)
    st, ma, dC = O.enkf_analyse(m, xs, yo, 0 * eps, 0.0, idx, var, 1, 1, nc, r, gain_form=0)
    assert st == 1
    np.testing.assert_array_equal(ma, m)


def test_huge_noise_gives_no_correction_and_tiny_noise_fits_observations():
    nc, r, ne, ny = 20, 2, 12, 5          # ny <= ne - 1
    m, xs, idx, var, yo, eps, _ = _problem(nc, r, ne, ny, seed=11)
    st, _, dC = O.enkf_analyse(m, xs, yo, 0 * eps, 1e8, idx, var, 1, 1, nc, r, gain_form=1)
    assert st == 0 and np.max(np.abs(dC)) < 1e-12
    st, _, dC = O.enkf_analyse(m, xs, yo, 1e-9 * eps, 1e-9, idx, var, 1, 1, nc, r, gain_form=0)
    assert st == 0
    hx = O.obs_coarse(xs + dC, 1, 1, nc, r, idx, var)
    np.testing.assert_allclose(hx, yo, atol=1e-6)


def test_ensemble_mean_converges_to_kalman_filter():
    # Linear-Gaussian case (Sec. 2.1.1): with Q = 0 and a prior ensemble drawn
    # from N(m0, P0), the EnKF increment tends to the KF increment
    # K (y - H m0), K = P0 H^T (H P0 H^T + R)^-1, with error ~ 1/sqrt(Ne).
    n, ny, sigma = 8, 3, 0.5
    rng = np.random.default_rng(0)
    Lp = rng.standard_normal((n, n)) * 0.4
    P0 = Lp @ Lp.T + 0.2 * np.eye(n)
    m0 = rng.standard_normal(n)
    idx = np.array([1, 4, 6], np.int32)
    var = np.zeros(ny, np.int32)
    H = np.zeros((ny, n))
    H[np.arange(ny), idx] = 1.0
    yo = rng.standard_normal(ny)
    K = P0 @ H.T @ np.linalg.inv(H @ P0 @ H.T + sigma**2 * np.eye(ny))
    kf_inc = K @ (yo - H @ m0)
    Pa = (np.eye(n) - K @ H) @ P0
    sizes, errs, cov_errs = [500, 2000, 8000, 32000], [], []
    chol = np.linalg.cholesky(P0)
    for ne in sizes:
        e2, c2 = [], []
        for s in range(20):
            g = np.random.default_rng([ne, s])
            ens = m0 + (chol @ g.standard_normal((n, ne))).T
            eps = sigma * g.standard_normal((ne, ny))
            st, ma, dC = O.enkf_analyse(ens, m0, yo, eps, sigma, idx, var, 1, 1, n, 1, gain_form=0)
            assert st == 0
            e2.append(np.sum((dC - kf_inc) ** 2))
            c2.append(np.sum((np.cov(ma.T) - Pa) ** 2))
        errs.append(math.sqrt(np.mean(e2)))
        cov_errs.append(math.sqrt(np.mean(c2)))
    slope = np.polyfit(np.log(sizes), np.log(errs), 1)[0]
    cslope = np.polyfit(np.log(sizes), np.log(cov_errs), 1)[0]
    assert -0.6 < slope < -0.4, (errs, slope)
    assert -0.6 < cslope < -0.4, (cov_errs, cslope)
    assert errs[-1] < 0.02 * np.linalg.norm(kf_inc)
