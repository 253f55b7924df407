"""Pins for the oracle's L1 weights, Toeplitz column and inverse column.

Each test checks the oracle against something it does not compute itself:
high-precision arithmetic, closed forms of the Caputo derivative, the
alpha -> 0 / alpha -> 1 limits, or a dense matrix product.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import l1, toeplitz
from paper_1608_05400_gb300 import inputs


def test_weights_match_high_precision_difference():
    # d_k = k^beta - (k-1)^beta evaluated in 60-digit arithmetic (Sec. 2, below Eq. L1_scheme2)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for alpha in (0.1, 0.5, 0.9):
        M = 70000
        d = l1.l1_weights(alpha, M)
        beta = mpmath.mpf(1) - mpmath.mpf(alpha)
        for k in (1, 2, 3, 10, 1000, 65536, 70000):
            ref = mpmath.power(k, beta) - mpmath.power(k - 1, beta)
            assert abs(d[k] - float(ref)) <= 4e-16 * float(ref), (alpha, k)
        assert d[0] == 0.0


def test_column_high_precision_second_difference():
    # r_i = c (d_i - d_{i-1}); the second difference is the ill-conditioned part
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    alpha, T, M = 0.2, 1.0, 65536
    r = l1.toeplitz_column(alpha, T, M)
    c = l1.l1_scale(alpha, T, M)
    beta = mpmath.mpf(1) - mpmath.mpf(alpha)
    for i in (2, 3, 17, 4096, 65536):
        ref = c * float(mpmath.power(i, beta) - 2 * mpmath.power(i - 1, beta) + mpmath.power(i - 2, beta))
        # absolute error against d_i (the scale of the operands), Sec. 5 Eq. Toeplitz_matrix
        assert abs(r[i - 1] - ref) <= 2e-15 * c * abs(float(mpmath.power(i, beta) - mpmath.power(i - 1, beta)))


@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.5, 0.8, 0.95])
@pytest.mark.parametrize("M", [1, 2, 7, 64, 1000])
def test_l1_exact_on_linear_functions(alpha, M):
    # The L1 scheme interpolates u piecewise linearly (Sec. 2 Eq. L1_scheme1), so for
    # u = t it reproduces D^alpha t = t^{1-alpha} / Gamma(2-alpha) exactly.
    T = 1.7
    t = inputs.time_nodes(M, T)
    Tm = l1.toeplitz_matrix(alpha, T, M)
    exact = inputs.caputo_of_profile("t1", alpha, t)
    # rounding bound: a few ulps of sum_j |T_mj| t_j (the terms cancel to O(1))
    np.testing.assert_allclose(Tm @ t, exact, rtol=0, atol=4e-16 * (np.abs(Tm) @ t).max())


def test_term_by_term_form_with_initial_value():
    # Eq. L1_scheme2 with u_0 != 0: D_M u = T_M u - c d_m u_0, checked for u = 3 + t
    alpha, T, M = 0.35, 1.0, 40
    t = inputs.time_nodes(M, T)
    u = 3.0 + t
    out = l1.l1_derivative(u, 3.0, alpha, T)
    np.testing.assert_allclose(out, inputs.caputo_of_profile("t1", alpha, t), rtol=1e-12)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_l1_order_two_minus_alpha_on_t_squared(alpha):
    # L1 truncation error for smooth u = t^2 is O(tau^{2-alpha}) (standard L1 result)
    errs = []
    for M in (64, 128, 256, 512):
        t = inputs.time_nodes(M, 1.0)
        Tm = l1.toeplitz_matrix(alpha, 1.0, M)
        errs.append(np.abs(Tm @ (t * t) - inputs.caputo_of_profile("t2", alpha, t)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(q - (2 - alpha)) < 0.08 for q in rates), rates


def test_alpha_one_is_backward_euler():
    # alpha -> 1: d_1 = 1, d_k = 0 (k >= 2), c = 1/tau: T_M is the backward difference
    M, T = 16, 2.0
    r = l1.toeplitz_column(1.0, T, M)
    tau = T / M
    ref = np.zeros(M)
    ref[0], ref[1] = 1 / tau, -1 / tau
    np.testing.assert_allclose(r, ref, rtol=1e-15, atol=1e-15)


def test_alpha_zero_limit_is_identity_scaled():
    # alpha -> 0: d_k -> 1, so r_1 = c and r_i = O(alpha) for i >= 2
    alpha, M = 1e-9, 32
    r = l1.toeplitz_column(alpha, 1.0, M)
    assert abs(r[0] - 1.0) < 1e-7
    assert np.abs(r[1:]).max() < 1e-8


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.9])
@pytest.mark.parametrize("sigma", [0.0, 8.0, 2.0 * 2 * 256.0 ** 2])
def test_inverse_column_definition_and_sign(alpha, sigma):
    M = 256
    r = l1.toeplitz_column(alpha, 1.0, M)
    k = toeplitz.inverse_column(alpha, 1.0, M, sigma)
    # dense product with the library Toeplitz constructor: (T + sigma I) k = e_1
    A = sla.toeplitz(r, np.zeros(M)) + sigma * np.eye(M)
    e1 = np.zeros(M)
    e1[0] = 1.0
    np.testing.assert_allclose(A @ k, e1, atol=1e-14 * np.abs(A).sum(1).max() * np.abs(k).max())
    # T_M + sigma I is an M-matrix (positive diagonal, r_i < 0 off it): inverse is nonnegative
    assert (r[1:] < 0).all()
    assert (k > 0).all()


def test_inverse_column_alpha_one_closed_form():
    # backward Euler: (c + sigma) k_1 = 1, (c + sigma) k_m = c k_{m-1}
    M, T, sigma = 50, 1.0, 3.0
    c = M / T
    k = toeplitz.inverse_column(1.0, T, M, sigma)
    ref = (1.0 / (c + sigma)) * (c / (c + sigma)) ** np.arange(M)
    np.testing.assert_allclose(k, ref, rtol=1e-13)


def test_causal_apply_matches_numpy_convolve():
    rng = np.random.default_rng(3)
    col = rng.standard_normal(33)
    b = rng.standard_normal((4, 33))
    y = toeplitz.causal_apply(col, b)
    for p in range(4):
        np.testing.assert_allclose(y[p], np.convolve(col, b[p])[:33], rtol=1e-13, atol=1e-13)
