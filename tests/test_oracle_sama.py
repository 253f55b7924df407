"""Pins for the semi-algebraic mode analysis (Sec. 4) in oracle/sama.py.

The symbols are checked against the two-grid cycle built as plain matrices on a
small periodic space-time grid (brute force: the 2h-harmonic pair must be an
invariant subspace on which the brute-force operator equals the symbol); the
elliptic limit, where 1-D red-black relaxation with full weighting and linear
interpolation solves exactly; the structure that makes the exact spectral radius
independent of M; and the factors the paper prints in Table lambdas_m, both the
predicted ones and the measured W-cycle ones they are compared with.
"""
import functools
import math
import os

import numpy as np
import pytest

from oracle import l1, sama

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(autouse=True)
def _one_blas_thread():
    # the eigenproblems are small (at most 128 x 128): a threaded BLAS only adds
    # synchronisation, about nine times the single-thread time on an 8-core host
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        yield
        return
    with threadpool_limits(1):
        yield


@functools.lru_cache(maxsize=None)
def _predicted(log2lam, M):
    return sama.two_grid_factor(2.0 ** log2lam, int(M), 0.4, mode="dense")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def _circulant(n, centre, side):
    A = np.zeros((n, n))
    for j in range(n):
        A[j, j] = centre
        A[j, (j - 1) % n] += side
        A[j, (j + 1) % n] += side
    return A


def _periodic_cycle(lam, M, delta, n):
    """Error propagation of the red-black waveform step, the coarse-grid correction
    and the Jacobi step on n periodic points x M time steps, h = 1, built from the
    cycle's definitions (Sec. 3 smoother, Algorithm 1 transfers), not from symbols."""
    tau = sama.tau_of(lam, 1.0, delta)
    Tm = l1.toeplitz_matrix(delta, M * tau, M)
    IM, In = np.eye(M), np.eye(n)
    A = np.kron(_circulant(n, 2.0, -1.0), IM) + np.kron(In, Tm)
    Dinv = np.linalg.inv(np.kron(In, Tm + 2.0 * IM))
    even = np.diag([1.0 if j % 2 == 0 else 0.0 for j in range(n)])
    eye = np.eye(n * M)
    red = eye - np.kron(even, IM) @ Dinv @ A
    black = eye - np.kron(In - even, IM) @ Dinv @ A
    jac = eye - Dinv @ A
    nc = n // 2
    R = np.zeros((nc, n))
    P = np.zeros((n, nc))
    for J in range(nc):
        R[J, 2 * J] = 0.5
        R[J, (2 * J - 1) % n] = 0.25
        R[J, (2 * J + 1) % n] = 0.25
        P[2 * J, J] = 1.0
        P[2 * J + 1, J] = 0.5
        P[2 * J + 1, (J + 1) % nc] = 0.5
    Ac = np.kron(_circulant(nc, 0.5, -0.25), IM) + np.kron(np.eye(nc), Tm)
    C = eye - np.kron(P, IM) @ np.linalg.solve(Ac, np.kron(R, IM) @ A)
    return red, black, C, jac


def _basis(theta, n, M):
    v = np.exp(1j * theta * np.arange(n)) / math.sqrt(n)
    return np.kron(v[:, None], np.eye(M))


def _symbol_errors(lam, delta=0.4, M=6, n=16):
    """(largest departure from invariance of the harmonic pairs, largest difference
    between the brute-force operators there and the symbols)."""
    red, black, C, jac = _periodic_cycle(lam, M, delta, n)
    S = black @ red
    inv = err = 0.0
    for k in range(1, n // 4 + 1):
        t0, t1 = sama.harmonics(2 * math.pi * k / n)
        Q = np.hstack([_basis(t0, n, M), _basis(t1, n, M)])
        want_red, want_black = sama.red_black_symbols(lam, M, delta, t0)
        for full, want in ((red, want_red), (black, want_black),
                           (C, sama.coarse_grid_symbol(lam, M, delta, t0)),
                           (C @ S, sama.two_grid_symbol(lam, M, delta, t0, 1, 0)),
                           (S @ C @ S, sama.two_grid_symbol(lam, M, delta, t0, 1, 1))):
            B = Q.conj().T @ full @ Q
            inv = max(inv, np.abs(full @ Q - Q @ B).max())
            err = max(err, np.abs(B - want).max() / max(1.0, np.abs(want).max()))
        for t in (t0, t1):
            Qa = _basis(t, n, M)
            B = Qa.conj().T @ jac @ Qa
            err = max(err, np.abs(B - sama.jacobi_symbol(lam, M, delta, t)).max())
    return inv, err


@pytest.mark.parametrize("lam", [0.25, 4.0])
def test_symbols_equal_the_periodic_two_grid_cycle(lam):
    # the harmonic pairs are invariant and the operators there are the symbols
    inv, err = _symbol_errors(lam)
    assert inv <= 1e-12 and err <= 1e-12, (inv, err)


def _red_black_wrong_sign(lam, M, delta, theta0):
    s_red, s_black = _RED_BLACK(lam, M, delta, theta0)
    M2 = s_black.shape[0] // 2
    s_black = s_black.copy()
    s_black[:M2, M2:] *= -1.0
    return s_red, s_black


_RED_BLACK = sama.red_black_symbols


@pytest.mark.parametrize("name,mutant", [
    ("laplacian_symbol", lambda t: 4.0 * math.sin(t / 2.0)),               # square dropped
    ("transfer_symbol", lambda t: 0.5 * (1.0 - math.cos(t))),             # wrong sign
    ("coarse_laplacian_symbol", lambda t: 4.0 * math.sin(t / 2.0) ** 2),  # fine stencil
    ("red_black_symbols", _red_black_wrong_sign),                         # coupling sign
])
def test_planted_mistakes_are_caught(monkeypatch, name, mutant):
    monkeypatch.setattr(sama, name, mutant)
    assert _symbol_errors(0.25)[1] > 1e-3


def test_elliptic_limit_is_an_exact_two_grid_solver():
    # lambda = inf drops the time operator: red-black relaxation, full weighting
    # and linear interpolation with the 2h stencil then solve 1-D exactly
    for t in sama.low_frequencies(8):
        assert np.abs(sama.two_grid_symbol(math.inf, 4, 0.4, t)).max() <= 1e-12
    assert sama.two_grid_factor(2.0 ** 30, 8, 0.4, K=16, mode="dense") <= 1e-8
    assert sama.two_grid_factor(2.0 ** 30, 8, 0.4, K=16) <= 1e-8


def test_exact_radius_is_the_first_time_step():
    # every block of T(theta) is lower-triangular Toeplitz, so reordered by time step
    # T is block lower triangular with one repeated 2 x 2 diagonal block
    lam, delta, M = 0.5, 0.4, 16
    for t in sama.low_frequencies(6):
        T = sama.two_grid_symbol(lam, M, delta, t)
        for a in range(2):
            for b in range(2):
                blk = T[a * M:(a + 1) * M, b * M:(b + 1) * M]
                assert np.abs(np.triu(blk, 1)).max() <= 1e-15
                for k in range(M):
                    diag = np.diagonal(blk, -k)
                    assert np.abs(diag - diag[0]).max() <= 1e-13
        one = sama.two_grid_symbol(lam, 1, delta, t)
        assert abs(sama.spectral_radius(T, 2, "exact") - sama.spectral_radius(one, 2, "dense")) <= 1e-14
    assert sama.two_grid_factor(lam, 64, delta, K=16, mode="exact") == \
        sama.two_grid_factor(lam, 1, delta, K=16, mode="dense")


def test_dense_radius_grows_with_M_from_the_exact_one():
    lam, delta = 2.0 ** -4, 0.4
    exact = sama.two_grid_factor(lam, 32, delta, K=32, mode="exact")
    dense = [sama.two_grid_factor(lam, M, delta, K=32, mode="dense") for M in (1, 32, 64, 128)]
    assert abs(dense[0] - exact) <= 1e-14
    assert exact < dense[1] < dense[2] < dense[3]


PREDICTED = [r for r in _table("sama_rho_table.txt") if r[1] <= 128]


@pytest.mark.parametrize("row", PREDICTED, ids=lambda r: f"l{int(r[0])}-M{int(r[1])}")
def test_prediction_matches_paper_table(row):
    # Table lambdas_m, rows without brackets.  Where the factor has settled in M
    # (log2 lambda >= -2) the dense value agrees to a few per cent; below, it is
    # set by how rounding scatters the M-fold eigenvalues, so the bound is wider.
    log2lam, M, rho = row
    got = _predicted(log2lam, M)
    rel = 0.05 if log2lam >= -2 else 0.25
    assert abs(got - rho) <= rel * rho + 0.0006, (log2lam, M, got, rho)


def test_exact_radius_bounds_every_printed_prediction_from_below():
    # the exact spectral radius does not depend on M and lies below every printed
    # value (printed to three decimals)
    for log2lam, M, rho in _table("sama_rho_table.txt"):
        exact = sama.two_grid_factor(2.0 ** log2lam, int(M), 0.4, mode="exact")
        assert exact <= rho + 0.0005, (log2lam, M, exact, rho)


@pytest.mark.parametrize("M", [32, 64])
def test_prediction_matches_measured_w_cycle_factors(M):
    # Table lambdas_m: the prediction agrees with the bracketed measured factors
    # of the multilevel W-cycle wherever those have settled (log2 lambda >= -2)
    for log2lam, Mr, rho_h in _table("sama_lambda_table.txt"):
        if int(Mr) != M or log2lam < -2:
            continue
        got = _predicted(log2lam, M)
        assert abs(got - rho_h) <= 0.12 * rho_h + 0.003, (log2lam, M, got, rho_h)


def test_factors_stay_below_two_tenths_for_all_orders():
    # Sec. 4.2 (Fig. delta_lambda_star): one smoothing step, tau / h^2 from 2^-12 to
    # 2^12, the predicted factors stay below 0.2 for every fractional order
    # (taken here with M = 32 and h = 1/256)
    h = 1.0 / 256
    for delta in (0.1, 0.3, 0.5, 0.7, 0.9):
        for e in range(-12, 13, 4):
            lam = sama.lam_of(2.0 ** e * h * h, h, delta)
            assert sama.two_grid_factor(lam, 32, delta, K=16, mode="dense") < 0.2, (delta, e)
            assert sama.two_grid_factor(lam, 32, delta, K=16) < 0.2, (delta, e)


def test_smoothing_factor_of_waveform_jacobi():
    # exact: the first time step, |Nhat / (1/lambda + 2)| at the worst high
    # frequency theta h = pi, i.e. 2 lambda / (1 + 2 lambda); dense agrees at M = 1
    for lam in (0.01, 1.0, 100.0):
        mu = sama.smoothing_factor(lam, 32, 0.4, K=8, mode="exact")
        assert abs(mu - 2 * lam / (1 + 2 * lam)) <= 1e-14
        assert sama.smoothing_factor(lam, 1, 0.4, K=8) == pytest.approx(mu, abs=1e-14)


def test_lambda_and_tau_are_inverse():
    for delta in (0.2, 0.4, 0.9):
        tau = sama.tau_of(2.0 ** -3, 1.0 / 64, delta)
        assert sama.lam_of(tau, 1.0 / 64, delta) == pytest.approx(2.0 ** -3, rel=1e-13)


def test_command_line_table(capsys):
    sama._main(["--M", "8,16", "--log2lam=0:2:2", "--K", "8"])
    out = capsys.readouterr().out.splitlines()
    assert out[0].split() == ["log2_lambda", "M=8", "M=16"]
    assert [int(line.split()[0]) for line in out[1:]] == [0, 2]


def test_pre_and_post_smoothing_give_the_same_factor():
    # T(1,0) = C S and T(0,1) = S C: AB and BA have the same eigenvalues
    for lam in (2.0 ** -4, 1.0, 2.0 ** 4):
        for t in sama.low_frequencies(6):
            a = np.linalg.eigvals(sama.two_grid_symbol(lam, 1, 0.4, t, 1, 0))
            b = np.linalg.eigvals(sama.two_grid_symbol(lam, 1, 0.4, t, 0, 1))
            assert np.allclose(np.sort_complex(a), np.sort_complex(b), rtol=0, atol=1e-12)
        assert abs(sama.two_grid_factor(lam, 8, 0.4, 1, 0, K=8, mode="exact")
                   - sama.two_grid_factor(lam, 8, 0.4, 0, 1, K=8, mode="exact")) <= 1e-14


def test_exact_factor_is_that_of_the_shifted_elliptic_problem():
    # the first time step sees -Delta_h + r_1 I: at delta = 1 (backward Euler) r_1 h^2 =
    # 1/lambda, so the factor is that of the 1-D two-grid cycle for h^-2 [-1 2+s -1],
    # s = 1/lambda; its time-free limit lambda = inf gives 0, and for s > 0 the cycle
    # is no longer exact
    assert sama.two_grid_factor(math.inf, 1, 1.0, K=16, mode="exact") <= 1e-12
    vals = [sama.two_grid_factor(2.0 ** e, 1, 1.0, K=32, mode="exact") for e in (8, 4, 0)]
    assert 0 < vals[0] < vals[1] < vals[2] < 0.2
    # the value at M = 1 does not depend on delta (only r_1 = c d_1 = c enters)
    for lam in (0.25, 4.0):
        a = sama.two_grid_factor(lam, 1, 0.3, K=16, mode="exact")
        b = sama.two_grid_factor(lam, 1, 0.9, K=16, mode="exact")
        assert abs(a - b) <= 1e-15
