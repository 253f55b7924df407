"""Pins for the oracle's discrete solution (time stepping, dense solve, separable form)."""
import math

import numpy as np
import pytest

from oracle import direct, l1, separable
from paper_1608_05400_gb300 import inputs


@pytest.mark.parametrize("d,n,M", [(1, 3, 4), (1, 7, 16), (2, 3, 8), (2, 7, 4), (1, 1, 8), (2, 1, 4)])
@pytest.mark.parametrize("with_ic", [False, True])
def test_time_stepping_equals_dense_solve(d, n, M, with_ic):
    # Sec. 5: A = T_M (x) I_N + A_h is block lower triangular; stepping in time and the
    # all-at-once dense solve are two routes to the same vector.
    alpha, T = 0.37, 0.8
    N = n ** d
    f = inputs.random_field(N, M, seed=11 + n + M)
    g = inputs.random_field(N, 1, seed=5)[:, 0] if with_ic else None
    u1 = direct.time_stepping(d, n, M, T, alpha, f, g)
    u2 = direct.dense_solve(d, n, M, T, alpha, f, g)
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-13 * np.abs(u2).max())


def test_dense_solve_satisfies_pointwise_scheme():
    # Residual of Eqs. (discrete_model_IVP_1)-(discrete_model_IVP_3) written out per
    # point with the term-by-term L1 form, independent of the Kronecker assembly.
    d, n, M, T, alpha = 1, 5, 6, 1.0, 0.6
    f = inputs.random_field(n, M, seed=2)
    g = inputs.random_field(n, 1, seed=3)[:, 0]
    u = direct.dense_solve(d, n, M, T, alpha, f, g)
    h = 1.0 / (n + 1)
    for i in range(n):
        Du = l1.l1_derivative(u[i], g[i], alpha, T)
        left = u[i - 1] if i > 0 else 0.0
        right = u[i + 1] if i < n - 1 else 0.0
        lap = (left - 2 * u[i] + right) / h ** 2
        np.testing.assert_allclose(Du - lap, f[i], rtol=1e-11, atol=1e-11)


def test_laplacian_sine_eigenvector():
    for d, n in ((1, 31), (2, 15)):
        ph = inputs.phi(d, n)
        lam = separable.eigenvalue(d, n)
        np.testing.assert_allclose(direct.laplacian(d, n) @ ph, lam * ph, rtol=1e-12, atol=1e-9)
        # lambda_h -> d pi^2 as h -> 0
        assert abs(lam - d * math.pi ** 2) < d * math.pi ** 4 / (n + 1) ** 2


@pytest.mark.parametrize("d,n,M,kind", [(1, 31, 64, "t2"), (2, 15, 32, "talpha"), (2, 7, 16, "t2")])
def test_separable_equals_time_stepping(d, n, M, kind):
    prob = inputs.Problem(d, n, M, 1.0, 0.5, kind)
    f = prob.rhs()
    u1 = direct.time_stepping(d, n, M, 1.0, 0.5, f)
    u2 = separable.solution(d, n, M, 1.0, 0.5, prob.rhs_profile(), inputs.phi(d, n))
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-13 * np.abs(u2).max())


def _sep_error(d, n, M, alpha, kind):
    prob = inputs.Problem(d, n, M, 1.0, alpha, kind)
    w = separable.time_factor(d, n, M, 1.0, alpha, prob.rhs_profile())
    return np.abs(w - inputs.time_profile(kind, alpha, inputs.time_nodes(M, 1.0))).max()


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_observed_order_in_tau_smooth(alpha):
    # u = t^2 sin: error O(tau^{2-alpha}) once h is negligible (n large)
    n = 2 ** 16 - 1
    e = [_sep_error(1, n, M, alpha, "t2") for M in (32, 64, 128, 256)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(3)]
    assert all(abs(q - (2 - alpha)) < 0.12 for q in rates), rates


@pytest.mark.parametrize("alpha", [0.4, 0.6])
def test_observed_order_in_tau_nonsmooth(alpha):
    # u = t^alpha sin: error O(tau^alpha) (Sec. 7: O(h^2 + tau^delta) for typical
    # solutions).  As Sec. 7 notes for small delta, the rate approaches alpha only on
    # fine temporal meshes: the observed rate rises monotonically towards alpha.
    n = 2 ** 16 - 1
    e = [_sep_error(1, n, M, alpha, "talpha") for M in (512, 1024, 2048, 4096)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(3)]
    assert all(rates[i] < rates[i + 1] for i in range(2)), rates
    assert alpha - 0.15 < rates[-1] < alpha + 0.02, rates


def test_observed_order_in_h():
    # spatial error O(h^2) with tau negligible: only lambda_h vs pi^2 enters
    M, alpha = 64, 0.5
    prob_ref = inputs.Problem(1, 2 ** 20 - 1, M, 1.0, alpha, "t2")
    w_ref = separable.time_factor(1, prob_ref.n, M, 1.0, alpha, prob_ref.rhs_profile())
    e = []
    for n in (15, 31, 63, 127):
        w = separable.time_factor(1, n, M, 1.0, alpha, prob_ref.rhs_profile())
        e.append(np.abs(w - w_ref).max())
    rates = [math.log2(e[i] / e[i + 1]) for i in range(3)]
    assert all(abs(q - 2.0) < 0.05 for q in rates), rates


def test_time_stepping_partial_steps():
    d, n, M = 1, 7, 12
    f = inputs.random_field(n, M, seed=9)
    full = direct.time_stepping(d, n, M, 1.0, 0.5, f)
    part = direct.time_stepping(d, n, M, 1.0, 0.5, f, steps=5)
    np.testing.assert_array_equal(part[:, :5], full[:, :5])
    assert not part[:, 5:].any()


@pytest.mark.parametrize("M,alpha", [(64, 0.5), (1000, 0.2), (4096, 0.85)])
def test_separable_substitution_equals_dense(M, alpha):
    # the O(M)-memory forward substitution used for long lines against the dense solve
    F = inputs.random_field(1, M, seed=M)[0]
    w1 = separable.time_factor_dense(1, 63, M, 0.9, alpha, F)
    w2 = separable.time_factor_substitution(1, 63, M, 0.9, alpha, F)
    np.testing.assert_allclose(w2, w1, rtol=0, atol=1e-13 * np.abs(w1).max())


@pytest.mark.parametrize("alpha", [0.2, 0.7])
def test_separable_substitution_linear_in_time_exact(alpha):
    # T_M t = t^{1-alpha} / Gamma(2-alpha) exactly (the L1 sums telescope), so
    # F = t^{1-alpha}/Gamma(2-alpha) + lambda_h t has the discrete solution w = t:
    # a pin at long M that does not go through the dense matrix
    d, n, M, T = 1, 4095, 16384, 1.0
    t = inputs.time_nodes(M, T)
    F = t ** (1 - alpha) / math.gamma(2 - alpha) + separable.eigenvalue(d, n) * t
    w = separable.time_factor_substitution(d, n, M, T, alpha, F)
    assert np.abs(w - t).max() <= 1e-11
    # beyond the dense limit time_factor is this substitution
    np.testing.assert_array_equal(separable.time_factor(d, n, M, T, alpha, F), w)
