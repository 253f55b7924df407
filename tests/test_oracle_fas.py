"""Pins for the waveform relaxation FAS oracle (Sec. 7, nonlinear problem) in
oracle/fas.py.

The discrete operator is checked against the continuous one (second order for the
flux difference, first order with the sign of a forward difference for the upwind
convection); the line solve against the equations it solves; FAS with a linear
operator against the linear oracle's cycle (the two schemes coincide there); the
FAS solution against an independent time-marching Newton solver; and the cycle
counts of Table table_nonlinear.
"""
import math
import os

import numpy as np
import pytest

from oracle import direct, fas, mgwr
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


def _smooth_profile(n):
    # u(x) = A sin(pi x) on the interior nodes, with its first two derivatives
    A = 0.7
    x = np.arange(1, n + 1) / (n + 1)
    return (A * np.sin(math.pi * x), A * math.pi * np.cos(math.pi * x),
            -A * math.pi ** 2 * np.sin(math.pi * x))


@pytest.mark.parametrize("c", [0.0, 1.0, -1.0])
def test_spatial_term_converges_to_the_continuous_operator(c):
    # -(d/dx((1 + u^2) u_x) + c u_x) = -((1 + u^2) u_xx + 2 u u_x^2 + c u_x).  The flux
    # difference with arithmetic-mean coefficients is second order.  Upwind convection
    # (forward difference for c >= 0, backward for c < 0) is first order and adds
    # numerical diffusion: the spatial term's leading error is -(|c| h / 2) u_xx for
    # either sign of c; a downwind difference would give the opposite sign.
    errs = []
    for n in (63, 127, 255, 511):
        h = 1.0 / (n + 1)
        u, ux, uxx = _smooth_profile(n)
        exact = -((1 + u * u) * uxx + 2 * u * ux * ux + c * ux)
        got = fas.spatial_term(u[:, None], h, c, fas.porous_D)[:, 0]
        e = got - exact
        if c == 0.0:
            errs.append(np.abs(e).max())
        else:
            # (got - exact) / h -> -|c| u_xx / 2 (sign fixed by the upwind direction)
            lead = -abs(c) * uxx / 2
            errs.append(np.abs(e / h - lead).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # c = 0: the error itself falls at order 2; c != 0: after removing the O(h) term
    # the remainder divided by h falls at order 1
    assert all(r > 1.9 if c == 0.0 else r > 0.9 for r in rates), rates


def test_linear_operator_is_the_linear_model():
    # D = 1, c = 0: N_h(u) = T_M u + A_h u with the 3-point Laplacian (Sec. 2)
    n, M = 15, 8
    rng = np.random.default_rng(7)
    u = rng.standard_normal((n, M))
    W = mgwr.WRMG(1, n, M, 1.0, 0.6)
    got = fas.operator(u, W.Tm, 1.0 / (n + 1), 0.0, fas.constant_D)
    want = u @ W.Tm.T + W.levels[-1].A @ u
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("c", [1.0, 0.0, -2.0])
def test_sweep_zeroes_the_defect_of_its_colour(c):
    n, M = 31, 24
    W = fas.WRFAS(n, M, 1.0, 0.5, c=c, order="table")
    rng = np.random.default_rng(11)
    u = 0.3 * rng.standard_normal((n, M))
    f = rng.standard_normal((n, M))
    L = W.finest
    for colour in (mgwr.RED, mgwr.BLACK):
        before = u.copy()
        W.sweep(L, u, f, colour)
        mask = mgwr.colour_mask(1, n, colour, "table")
        r = W.defect(L, u, f)
        scale = np.abs(W.N(L, u)).max() + np.abs(f).max()
        assert np.abs(r[mask]).max() <= 1e-13 * scale
        assert np.array_equal(u[~mask], before[~mask])


@pytest.mark.parametrize("order", ["text", "table"])
@pytest.mark.parametrize("nu", [(0, 1), (1, 1), (2, 0)])
def test_fas_with_a_linear_operator_is_the_linear_cycle(order, nu):
    # for a linear N_h the FAS coarse problem from ubar with right-hand side
    # N_2h(ubar) + R r is the correction scheme's coarse problem shifted by ubar, so
    # every cycle of WRFAS (D = 1, c = 0) equals the linear oracle's cycle
    n, M, T, delta = 31, 16, 1.0, 0.35
    F = fas.WRFAS(n, M, T, delta, c=0.0, D=fas.constant_D, dD=fas.constant_dD, order=order)
    W = mgwr.WRMG(1, n, M, T, delta, order=order)
    f = inputs.random_field(n, M, seed=5)
    uF = uW = np.zeros((n, M))
    for _ in range(3):
        uF = F.cycle(F.finest, uF, f, *nu)
        uW = W.cycle(W.finest, uW, f, *nu)
        assert np.abs(uF - uW).max() <= 1e-12 * np.abs(uW).max()
    # and the W-cycle
    uF = F.cycle(F.finest, uF, f, 1, 1, 2)
    uW = W.cycle(W.finest, uW, f, 1, 1, 2)
    assert np.abs(uF - uW).max() <= 1e-12 * np.abs(uW).max()


def test_time_stepping_with_a_linear_operator_is_the_linear_solution():
    n, M, T, delta = 31, 20, 0.5, 0.6
    f = inputs.random_field(n, M, seed=9)
    got = fas.time_stepping(n, M, T, delta, f, c=0.0, D=fas.constant_D, dD=fas.constant_dD)
    want = direct.time_stepping(1, n, M, T, delta, f)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("delta,c,kind", [(0.4, 1.0, "ones"), (0.8, -1.0, "ones"),
                                          (0.2, 2.0, "random"), (1.0, 1.0, "random")])
def test_fas_converges_to_the_time_marching_solution(delta, c, kind):
    # the relaxation and the time-marching Newton solver reach the same discrete solution
    n, M, T = 31, 32, 1.0
    f = np.ones((n, M)) if kind == "ones" else inputs.random_field(n, M, seed=3, scale=4.0)
    W = fas.WRFAS(n, M, T, delta, c=c, order="table")
    u, hist = W.solve(f, 0, 1, tol=1e-13, max_cycles=40)
    assert hist[-1] <= 1e-13
    ref = fas.time_stepping(n, M, T, delta, f, c=c)
    assert np.abs(W.defect(W.finest, ref, f)).max() <= 1e-12 * np.abs(f).max()
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(ref).max() > 0.05  # the nonlinearity D(u) - 1 = u^2 is not negligible


NONLINEAR = [r for r in _table("table_nonlinear.txt") if r[1] <= 128]


@pytest.mark.parametrize("row", NONLINEAR, ids=lambda r: f"d{r[0]}-{int(r[1])}")
def test_paper_table_nonlinear(row):
    # Table table_nonlinear: D(u) = 1 + u^2, c = 1, f = 1 on (0,1) x (0,1], N x N grid,
    # V(0,1) from u = 0 until the max-norm defect falls by 1e-10.  Cycle counts agree
    # to one; the printed factors are those the cycle settles to (its last reduction)
    delta, N, cycles, factor = row
    N = int(N)
    W = fas.WRFAS(N - 1, N, 1.0, delta, c=1.0, order="table")
    u, hist = W.solve(np.ones((N - 1, N)), 0, 1, tol=1e-10, max_cycles=30)
    k = len(hist) - 1
    assert hist[-1] <= 1e-10
    assert abs(k - cycles) <= 1, (delta, N, k, cycles)
    assert abs(hist[-1] / hist[-2] - factor) <= 0.02, (delta, N, hist[-1] / hist[-2], factor)


@pytest.mark.parametrize("c", [1.0, -1.0])
def test_line_solve_equals_the_preconditioned_whole_line_iteration(c):
    # an independent solver of the same line equations, T_M v + phi(v) = f with phi the
    # pointwise flux and upwind terms (neighbours fixed): the fixed point of
    # v <- v - (T_M + sigma I)^{-1} (T_M v + phi(v) - f), sigma = 2/h^2 + |c|/h, whose
    # every step is two causal convolutions (no march in time); it converges in a few
    # steps because phi' stays within a few per cent of sigma
    n, M, delta = 63, 64, 0.4
    W = fas.WRFAS(n, M, 1.0, delta, c=c, order="table")
    f = np.ones((n, M))
    u = W.cycle(W.finest, np.zeros((n, M)), f, 0, 1)  # a realistic iterate
    h = W.h(W.finest)
    rows = mgwr.colour_mask(1, n, mgwr.RED, "table")
    ref = u.copy()
    fas.line_solve(ref, f, rows, W.Tm, h, c, fas.porous_D, fas.porous_dD)
    K = np.linalg.inv(W.Tm + (2.0 / h ** 2 + abs(c) / h) * np.eye(M))
    for i in np.flatnonzero(rows):
        v = u[i].copy()
        for k in range(30):
            line = u.copy()
            line[i] = v
            G = fas.operator(line, W.Tm, h, c, fas.porous_D)[i] - f[i]
            dv = K @ G
            v = v - dv
            if np.abs(dv).max() <= 1e-15 * np.abs(v).max():
                break
        assert k < 12, k
        assert np.abs(v - ref[i]).max() <= 1e-13 * np.abs(ref[i]).max()
