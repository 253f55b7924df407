"""Pins for the oracle's WRMG cycle (Algorithm 1) and its components."""
import math
import os

import numpy as np
import pytest

from oracle import direct, mgwr
from paper_1608_05400_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("d,n", [(1, 15), (2, 7)])
@pytest.mark.parametrize("colour", [mgwr.RED, mgwr.BLACK])
def test_sweep_zeroes_defect_on_its_colour(d, n, colour):
    # Eq. (red-black)/(red-black_2d): each visited point satisfies its own equation
    # exactly with the current neighbours, so the defect vanishes there.
    M = 24
    W = mgwr.WRMG(d, n, M, 1.0, 0.45)
    N = n ** d
    u = inputs.random_field(N, M, seed=1)
    f = inputs.random_field(N, M, seed=2)
    W.sweep(W.finest, u, f, colour)
    r = W.defect(W.finest, u, f)
    mask = mgwr.colour_mask(d, n, colour)
    assert np.abs(r[mask]).max() < 1e-10 * np.abs(f).max() * W.levels[-1].sigma
    assert np.abs(r[~mask]).max() > 1e-3


def test_colours_follow_paper_numbering():
    # text: 1-based even n first -> 0-based odd i; 2-D: n+l even -> 0-based i+j even
    np.testing.assert_array_equal(mgwr.colour_mask(1, 7, mgwr.RED), [0, 1, 0, 1, 0, 1, 0])
    np.testing.assert_array_equal(mgwr.colour_mask(1, 7, mgwr.RED, "table"), [1, 0, 1, 0, 1, 0, 1])
    for order in mgwr.ORDERS:
        m2 = mgwr.colour_mask(2, 3, mgwr.RED, order).reshape(3, 3)
        np.testing.assert_array_equal(m2, [[1, 0, 1], [0, 1, 0], [1, 0, 1]])


def test_full_weighting_of_sine_closed_form():
    # (1/4)(sin(pi(x-h)) + 2 sin(pi x) + sin(pi(x+h))) = cos^2(pi h/2) sin(pi x)
    for d, n in ((1, 31), (2, 15)):
        h = 1.0 / (n + 1)
        fine = np.outer(inputs.phi(d, n), [1.0, -2.0])
        coarse = mgwr.restrict_fw(fine, d, n)
        ref = np.outer(inputs.phi(d, (n - 1) // 2), [1.0, -2.0]) * math.cos(math.pi * h / 2) ** (2 * d)
        np.testing.assert_allclose(coarse, ref, rtol=1e-13, atol=1e-14)


def test_prolongation_is_library_interpolation():
    rng = np.random.default_rng(0)
    nc = 7
    n = 2 * nc + 1
    xc = inputs.interior_nodes(nc)
    xf = inputs.interior_nodes(n)
    E = rng.standard_normal((nc, nc, 3))  # (j, i, m)
    e = mgwr.prolong_linear(E.reshape(nc * nc, 3), 2, nc).reshape(n, n, 3)
    xp = np.concatenate([[0.0], xc, [1.0]])
    for m in range(3):
        # interpolate along x (i) then y (j) with zero boundary values
        Ex = np.stack([np.interp(xf, xp, np.concatenate([[0], E[j, :, m], [0]])) for j in range(nc)])
        ref = np.stack([np.interp(xf, xp, np.concatenate([[0], Ex[:, i], [0]])) for i in range(n)], axis=1)
        np.testing.assert_allclose(e[:, :, m], ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [1, 2])
def test_restriction_is_scaled_transpose_of_interpolation(d):
    # standard pair: I_h^{2h} = 2^{-d} (I_{2h}^h)^T
    nc = 3
    n = 2 * nc + 1
    P = np.stack([mgwr.prolong_linear(np.eye(nc ** d)[:, [k]], d, nc)[:, 0] for k in range(nc ** d)], axis=1)
    R = np.stack([mgwr.restrict_fw(np.eye(n ** d)[:, [k]], d, n)[:, 0] for k in range(n ** d)], axis=1)
    np.testing.assert_allclose(R, P.T / 2 ** d, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d,n,M,cyc", [(1, 31, 32, (0, 1, 1)), (1, 15, 16, (1, 1, 2)),
                                       (2, 15, 16, (1, 1, 1)), (2, 7, 8, (1, 0, 2))])
def test_wrmg_converges_to_direct_solution(d, n, M, cyc):
    nu1, nu2, gamma = cyc
    alpha, T = 0.5, 1.0
    f = inputs.random_field(n ** d, M, seed=7)
    W = mgwr.WRMG(d, n, M, T, alpha)
    u, hist = W.solve(f, nu1, nu2, gamma, tol=1e-13, max_cycles=60)
    ref = direct.time_stepping(d, n, M, T, alpha, f)
    assert hist[-1] <= 1e-13
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_steady_limit_1d_red_black_two_grid_is_exact():
    # Sec. 6 Remark: in the steady limit the 1-D red-black multigrid is an exact solver.
    # A huge final time makes T_M negligible next to A_h.  After the black half-sweep
    # the defect vanishes at the fine-only points, full weighting then gives the exact
    # coarse defect and linear interpolation the exact fine error, so one V(1,0)
    # cycle solves to rounding; a cycle without pre-smoothing does not.
    d, n, M = 1, 63, 8
    W = mgwr.WRMG(d, n, M, 1e30, 0.5)
    f = inputs.random_field(n, M, seed=4)
    _, hist = W.solve(f, 1, 0, 1, tol=0.0, max_cycles=1)
    assert hist[1] < 1e-11
    _, hist01 = W.solve(f, 0, 1, 1, tol=0.0, max_cycles=1)
    assert hist01[1] > 1e-3


def _asymptotic_factor(W, nu1, nu2, gamma, cycles=14, seed=0):
    """Random initial guess, zero right-hand side; factor of the last cycles (Sec. 4.2)."""
    L = W.finest
    N = W.levels[L].n ** W.d
    u = inputs.random_field(N, W.M, seed=seed)
    f = np.zeros_like(u)
    norms = []
    for _ in range(cycles):
        u = W.cycle(L, u, f, nu1, nu2, gamma)
        s = np.abs(u).max()
        norms.append(s)
        u /= s  # keep the iterate away from underflow
    tail = norms[-4:]
    return float(np.exp(np.mean(np.log(tail))))


def test_w_cycle_asymptotic_factors_match_paper_table():
    # Table lambdas_m, bracketed rows: measured W-cycle factors, delta = 0.4, 256 x M grid,
    # one smoothing step, random initial guess, zero right-hand side.  For
    # log2(lambda) >= -2 the factor settles within a few cycles and must agree.  For
    # smaller lambda the cycle operator is far from normal (block lower-triangular
    # Toeplitz in time) and the observed factor keeps drifting down for tens of
    # cycles, so only an upper bound is asserted there.
    delta = 0.4
    n = 255
    h = 1.0 / (n + 1)
    for log2lam, M, rho_h in _table("sama_lambda_table.txt"):
        M = int(M)
        lam = 2.0 ** log2lam
        tau = (lam * h * h / math.gamma(2 - delta)) ** (1 / delta)
        W = mgwr.WRMG(1, n, M, M * tau, delta)
        rho = _asymptotic_factor(W, 1, 0, 2, cycles=20)
        if log2lam >= -2:
            assert abs(rho - rho_h) <= 0.12 * rho_h + 0.003, (log2lam, M, rho, rho_h)
        else:
            assert rho_h * 0.8 <= rho <= 2.5 * rho_h, (log2lam, M, rho, rho_h)


def test_v11_2d_iterations_match_paper_table():
    # Table table_it_2d: V(1,1), reduce the initial residual by 1e-10.  The paper's
    # problem on (0,2)^2 maps to (0,1)^2 by x -> x/2, t -> t 4^{-1/delta}; the
    # iteration count is invariant under that rescaling.
    for delta, grid, M, its, factor in _table("table_it_2d.txt"):
        if grid != 32:
            continue
        n, M = int(grid) - 1, int(M)
        T = 4.0 ** (-1.0 / delta) if delta < 1 else 0.25
        prob = inputs.Problem(2, n, M, T, min(delta, 1.0), "t2")
        W = mgwr.WRMG(2, n, M, T, delta)
        u, hist = W.solve(prob.rhs(), 1, 1, 1, tol=1e-10, max_cycles=40)
        k = len(hist) - 1
        mean = hist[-1] ** (1.0 / k)
        assert abs(k - its) <= 2, (delta, k, its)
        assert abs(mean - factor) <= 0.04, (delta, mean, factor)


def _paper_1d_problem(delta, n, M):
    # Table table_it_1d's problem: f = 0, g = sin x on [0, pi]; mapped to (0,1) by
    # x -> x/pi, t -> t pi^{-2/delta}.  Initial iterate u^0 = g (Sec. 3, below Eq. GS_ODEs).
    from oracle import l1
    T = math.pi ** (-2.0 / delta)
    g = inputs.phi(1, n)
    dk = l1.l1_weights(delta, M)
    c = l1.l1_scale(delta, T, M)
    f = c * np.outer(g, dk[1:])  # f = 0 plus the u_0 term of Eq. L1_scheme2
    return T, f, np.repeat(g[:, None], M, axis=1)


def test_v01_1d_iterations_match_paper_table():
    # Table table_it_1d (V(0,1), 7-8 cycles, mean factor 0.03-0.05) is reproduced with
    # the "table" colour order; Sec. 7 also states V(0,1) beats V(1,0) clearly.
    for delta, grid, M, its, factor in _table("table_it_1d.txt"):
        if grid != 128:
            continue
        n, M = int(grid) - 1, int(M)
        T, f, u0 = _paper_1d_problem(delta, n, M)
        W = mgwr.WRMG(1, n, M, T, delta, order="table")
        u, hist = W.solve(f, 0, 1, 1, tol=1e-10, max_cycles=40, u0=u0)
        k = len(hist) - 1
        mean = hist[-1] ** (1.0 / k)
        assert abs(k - its) <= 1, (delta, k, its)
        assert abs(mean - factor) <= 0.02, (delta, mean, factor)
        _, h10 = W.solve(f, 1, 0, 1, tol=1e-10, max_cycles=40, u0=u0)
        assert len(h10) - 1 > k + 5


def test_v01_1d_text_order_is_slower_than_table():
    # The literal text order (even mesh index first) converges, to the same discrete
    # solution, but needs about twice the V(0,1) cycles of Table table_it_1d.
    delta, n, M = 0.4, 127, 128
    T, f, u0 = _paper_1d_problem(delta, n, M)
    res = {}
    for order in mgwr.ORDERS:
        W = mgwr.WRMG(1, n, M, T, delta, order=order)
        res[order] = W.solve(f, 0, 1, 1, tol=1e-10, max_cycles=60, u0=u0)
        assert res[order][1][-1] <= 1e-10
    assert len(res["text"][1]) > len(res["table"][1]) + 4
    ref = res["table"][0]
    np.testing.assert_allclose(res["text"][0], ref, rtol=0, atol=1e-8 * np.abs(ref).max())
