"""Pins of the oracle's relative RMSE (Eq. L2norm_u): closed forms that a
dropped square, a swapped denominator or a mixed-up variable plane would fail."""
import math

import numpy as np

import oracle as O


def test_identical_fields_give_zero():
    t = np.random.default_rng(0).standard_normal((3, 257))
    np.testing.assert_array_equal(O.rmse(t, t, 3), np.zeros(3))


def test_uniform_relative_error_per_variable():
    # x = (1 + c_v) t on plane v: the relative RMSE of plane v is |c_v|,
    # whatever t is; one c per plane pins the plane layout
    rng = np.random.default_rng(1)
    t = rng.standard_normal((4, 1000)) + 2.0
    c = np.array([0.1, -0.02, 0.3, 1e-4])
    x = (1.0 + c[:, None]) * t
    np.testing.assert_allclose(O.rmse(x, t, 4), np.abs(c), rtol=1e-12)


def test_constant_offset_on_a_sine():
    # t_j = sin(2 pi j / N): sum t^2 = N / 2, so an offset delta gives
    # sqrt(N delta^2 / (N / 2)) = sqrt(2) |delta|
    n, delta = 4096, 0.0125
    t = np.sin(2 * math.pi * np.arange(n) / n)
    np.testing.assert_allclose(O.rmse(t + delta, t, 1), [math.sqrt(2) * delta], rtol=1e-12)


def test_denominator_is_the_truth():
    # not symmetric: x = 2 t gives 1, t = 2 x gives 1/2
    t = np.random.default_rng(2).standard_normal(513)
    np.testing.assert_allclose(O.rmse(2 * t, t, 1), [1.0], rtol=1e-13)
    np.testing.assert_allclose(O.rmse(t, 2 * t, 1), [0.5], rtol=1e-13)
