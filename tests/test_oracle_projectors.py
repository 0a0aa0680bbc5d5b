"""Pins of the oracle's projectors Pi_C / Pi_F (4th-order Lagrange, end of
Sec. 2.2) and of the coarse observation operator H^C = H^F Pi_F."""
import math

import numpy as np
import pytest

import oracle as O

NODES = [-1.0, 0.0, 1.0, 2.0]


@pytest.mark.parametrize("s", [0.0, 0.25, 0.5, 0.75, 0.3])
def test_lagrange_weights_reproduce_cubics(s):
    w = O.lagrange_weights(NODES, s)
    assert abs(w.sum() - 1.0) < 1e-15
    rng = np.random.default_rng(1)
    for _ in range(5):
        c = rng.standard_normal(4)
        p = lambda t: c[0] + c[1] * t + c[2] * t * t + c[3] * t**3
        assert abs(np.dot(w, [p(t) for t in NODES]) - p(s)) < 1e-13


@pytest.mark.parametrize("dim,V,nc,r", [(1, 1, 16, 4), (1, 1, 7, 3), (2, 4, 8, 4), (2, 1, 5, 2),
                                        (1, 1, 9, 1)])
def test_restrict_of_prolong_is_identity(dim, V, nc, r):
    rng = np.random.default_rng(2)
    dc = rng.standard_normal(V * nc**dim)
    fine = O.prolong_add(dc, np.zeros(V * (nc * r) ** dim), dim, V, nc, r)
    np.testing.assert_array_equal(O.restrict(fine, dim, V, nc, r), dc)


def test_prolong_exact_on_cubic_away_from_wrap_1d():
    nc, r = 32, 4
    J = np.arange(nc, dtype=float)
    p = lambda t: 0.3 - 0.2 * t + 0.05 * t * t - 0.001 * t**3
    fine = O.prolong_add(p(J), np.zeros(nc * r), 1, 1, nc, r)
    f = np.arange(nc * r)
    Jf = f // r
    ok = (Jf >= 1) & (Jf <= nc - 3)
    np.testing.assert_allclose(fine[ok], p(f[ok] / r), rtol=0, atol=1e-12)


def test_prolong_exact_on_bicubic_away_from_wrap_2d():
    nc, r = 12, 2
    J = np.arange(nc, dtype=float)
    px = lambda t: 1.0 + 0.1 * t - 0.02 * t**3
    py = lambda t: -0.5 + 0.03 * t * t + 0.004 * t**3
    dc = np.outer(py(J), px(J)).reshape(-1)
    fine = O.prolong_add(dc, np.zeros((nc * r) ** 2), 2, 1, nc, r).reshape(nc * r, nc * r)
    f = np.arange(nc * r)
    ok = ((f // r) >= 1) & ((f // r) <= nc - 3)
    expect = np.outer(py(f / r), px(f / r))
    np.testing.assert_allclose(fine[np.ix_(ok, ok)], expect[np.ix_(ok, ok)], atol=1e-12)


def test_prolong_fourier_mode_error_is_fourth_order():
    errs = []
    for nc in (16, 32, 64):
        r = 4
        xc = np.arange(nc) * 2 * math.pi / nc
        xf = np.arange(nc * r) * 2 * math.pi / (nc * r)
        fine = O.prolong_add(np.sin(3 * xc), np.zeros(nc * r), 1, 1, nc, r)
        errs.append(np.max(np.abs(fine - np.sin(3 * xf))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for p in orders:
        assert 3.7 < p < 4.3, (errs, orders)


def test_obs_coarse_is_prolongation_row():
    rng = np.random.default_rng(3)
    for dim, V, nc, r in [(1, 1, 16, 4), (2, 4, 6, 3)]:
        xc = rng.standard_normal(V * nc**dim)
        nfp = (nc * r) ** dim
        idx = rng.integers(0, nfp, size=11).astype(np.int32)
        var = rng.integers(0, V, size=11).astype(np.int32)
        y = O.obs_coarse(xc, dim, V, nc, r, idx, var)
        fine = O.prolong_add(xc, np.zeros(V * nfp), dim, V, nc, r)
        np.testing.assert_allclose(y, fine[var * nfp + idx], rtol=0, atol=1e-14)
    # coincident nodes: H^C is injection
    xc = rng.standard_normal(16)
    y = O.obs_coarse(xc, 1, 1, 16, 4, np.arange(0, 64, 4, dtype=np.int32), np.zeros(16, np.int32))
    np.testing.assert_array_equal(y, xc)
