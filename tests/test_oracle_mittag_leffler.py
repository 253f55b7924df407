"""Pins for the oracle's Mittag-Leffler function (the exact solution of the paper's
1-D experiment, Sec. 7) against closed forms of the special orders, and the L1
scheme's order-alpha convergence to it (Sec. 7: error O(h^2 + tau^alpha))."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import l1, separable
from oracle.mittag_leffler import mittag_leffler


def _bound(alpha, z):
    # rounding of the series: a few ulps of the sum of |terms| = E_alpha(|z|)
    return 8 * np.finfo(float).eps * mittag_leffler(alpha, np.abs(z))


def test_order_one_is_the_exponential():
    z = np.linspace(-4.0, 4.0, 33)
    assert np.all(np.abs(mittag_leffler(1.0, z) - np.exp(z)) <= _bound(1.0, z))


def test_order_two_is_cos_and_cosh():
    x = np.linspace(0.0, 4.0, 17)
    assert np.all(np.abs(mittag_leffler(2.0, -x) - np.cos(np.sqrt(x))) <= _bound(2.0, x))
    assert np.all(np.abs(mittag_leffler(2.0, x) - np.cosh(np.sqrt(x))) <= _bound(2.0, x))


def test_order_one_half_is_the_scaled_complementary_error_function():
    # E_{1/2}(-x) = exp(x^2) erfc(x), E_{1/2}(x) = exp(x^2) erfc(-x)
    x = np.linspace(0.0, 2.0, 21)
    assert np.all(np.abs(mittag_leffler(0.5, -x) - sp.erfcx(x)) <= _bound(0.5, x))
    assert np.all(np.abs(mittag_leffler(0.5, x) - np.exp(x * x) * sp.erfc(-x)) <= _bound(0.5, x))


def test_value_at_zero_and_argument_range():
    assert mittag_leffler(0.3, 0.0) == 1.0
    with pytest.raises(ValueError):
        mittag_leffler(0.5, -5.0)
    with pytest.raises(ValueError):
        mittag_leffler(0.0, -1.0)


@pytest.mark.parametrize("alpha", [0.1, 0.4, 0.7])
def test_completely_monotone_decay(alpha):
    # E_alpha(-x), 0 < alpha <= 1, decreases from 1 and stays positive on x >= 0
    x = np.linspace(0.0, min(4.0, 0.99 * 8.0 ** alpha), 81)
    v = mittag_leffler(alpha, -x)
    assert v[0] == 1.0 and np.all(np.diff(v) < 0) and np.all(v > 0)


@pytest.mark.parametrize("alpha", [0.4, 0.7])
def test_l1_solution_converges_at_order_alpha(alpha):
    # Sec. 7 first experiment on (0,1): g = sin(pi x), f = 0, T = pi^(-2/alpha), exact
    # u = E_alpha(-pi^2 t^alpha) sin(pi x).  With h negligible the error is O(tau^alpha);
    # the observed order approaches alpha from below (alpha = 0.7: already 0.70).
    T = math.pi ** (-2.0 / alpha)
    n = 4095
    errs = []
    for M in (256, 512, 1024, 2048):
        c = l1.l1_scale(alpha, T, M)
        F = c * l1.l1_weights(alpha, M)[1:]          # the c d_m g term, g = 1 on the mode
        w = separable.time_factor(1, n, M, T, alpha, F)
        t = T * np.arange(1, M + 1) / M
        errs.append(np.abs(w - mittag_leffler(alpha, -math.pi ** 2 * t ** alpha)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(0.85 * alpha <= r <= 1.02 * alpha for r in rates), rates
    assert rates[0] <= rates[1] + 1e-3 <= rates[2] + 2e-3
