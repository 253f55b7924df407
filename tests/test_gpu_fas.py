"""GPU parity of the nonlinear problem of Sec. 7 (mgwr_fas_*) against the CPU oracle
(oracle/fas.py): one level's nonlinear half-sweep and defect, whole FAS cycles one by
one, solves against the oracle's time-marching Newton solution, the cycle counts of
Table table_nonlinear, the linear special case against the linear solver, edge sizes
and a non-finite right-hand side.

Tolerances (FP64 throughout): the history sums and Newton steps round in another
order than the oracle's (32-lane partial sums on the GPU), so one component agrees to
1e-12 of the field's scale and three cycles to 1e-11; a solve stopped at a 1e-10
defect reduction is within 2e-11 of the discrete solution in the oracle, checked here
to 1e-9."""
import os

import numpy as np
import pytest

from oracle import fas
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

ORDER = {"text": G.MGWR_ORDER_TEXT, "table": G.MGWR_ORDER_TABLE}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("c,order", [(1.0, "table"), (-2.0, "text"), (0.0, "table")])
def test_half_sweep_matches_oracle(c, order):
    n, M, T, delta = 31, 24, 1.0, 0.5
    W = fas.WRFAS(n, M, T, delta, c=c, order=order)
    u = inputs.random_field(n, M, seed=21, scale=0.3)
    f = inputs.random_field(n, M, seed=22)
    uo = u.copy()
    with G.FAS(n, M, T, delta, c) as g:
        g.set_order(ORDER[order])
        L = g.num_levels() - 1
        assert L == W.finest
        g.field_set(L, G.MGWR_U, u)
        g.field_set(L, G.MGWR_F, f)
        for colour in (G.MGWR_RED, G.MGWR_BLACK):
            g.smooth(L, colour)
            W.sweep(W.finest, uo, f, colour)
            assert rel(g.field_get(L, G.MGWR_U), uo) <= 1e-12


@pytest.mark.parametrize("c", [1.0, -1.0])
def test_defect_matches_oracle(c):
    n, M, T, delta = 63, 40, 0.7, 0.3
    W = fas.WRFAS(n, M, T, delta, c=c)
    u = inputs.random_field(n, M, seed=31, scale=0.5)
    f = inputs.random_field(n, M, seed=32)
    with G.FAS(n, M, T, delta, c) as g:
        L = g.num_levels() - 1
        g.field_set(L, G.MGWR_U, u)
        g.field_set(L, G.MGWR_F, f)
        nrm = g.defect(L)
        r = g.field_get(L, G.MGWR_R)
    ro = W.defect(W.finest, u, f)
    scale = np.abs(W.N(W.finest, u)).max() + np.abs(f).max()
    assert np.abs(r - ro).max() <= 1e-13 * scale
    assert nrm == np.abs(r).max()


@pytest.mark.parametrize("nu,gamma", [((0, 1), 1), ((1, 1), 1), ((1, 1), 2)])
@pytest.mark.parametrize("kind", ["ones", "random"])
def test_cycles_match_oracle(nu, gamma, kind):
    n, M, T, delta, c = 31, 32, 1.0, 0.4, 1.0
    f = np.ones((n, M)) if kind == "ones" else inputs.random_field(n, M, seed=41, scale=4.0)
    W = fas.WRFAS(n, M, T, delta, c=c, order="table")
    uo = np.zeros((n, M))
    with G.FAS(n, M, T, delta, c) as g:
        g.set_order(G.MGWR_ORDER_TABLE)
        g.set_rhs(f)
        for _ in range(3):
            g.cycle(gamma, *nu)
            uo = W.cycle(W.finest, uo, f, nu[0], nu[1], gamma)
            assert rel(g.solution(), uo) <= 1e-11
        nrm = g.residual()
    assert abs(nrm - np.abs(W.defect(W.finest, uo, f)).max()) <= 1e-9 * np.abs(f).max()


@pytest.mark.parametrize("n,M,delta,c,kind", [
    (31, 32, 0.4, 1.0, "ones"), (63, 64, 0.7, 1.0, "ones"), (127, 128, 0.1, 1.0, "ones"),
    (255, 256, 1.0, 1.0, "ones"), (63, 50, 0.8, -1.0, "random"), (15, 7, 0.5, 2.0, "random")])
def test_solve_matches_time_marching_solution(n, M, delta, c, kind):
    T = 1.0
    f = np.ones((n, M)) if kind == "ones" else inputs.random_field(n, M, seed=51, scale=4.0)
    with G.FAS(n, M, T, delta, c) as g:
        g.set_order(G.MGWR_ORDER_TABLE)
        g.set_rhs(f)
        st = g.solve(1, 0, 1, tol=1e-10, max_cycles=40)
        u = g.solution()
    assert st.relres <= 1e-10
    ref = fas.time_stepping(n, M, T, delta, f, c=c)
    assert rel(u, ref) <= 1e-9


@pytest.mark.parametrize("row", _table("table_nonlinear.txt"), ids=lambda r: f"d{r[0]}-{int(r[1])}")
def test_paper_table_nonlinear(row):
    # Table table_nonlinear: D(u) = 1 + u^2, c = 1, f = 1 on (0,1) x (0,1], V(0,1) from
    # u = 0 until the max-norm defect falls by 1e-10: cycle counts within one
    delta, N, cycles, _factor = row
    N = int(N)
    with G.FAS(N - 1, N, 1.0, delta, 1.0) as g:
        g.set_order(G.MGWR_ORDER_TABLE)
        g.set_rhs(np.ones((N - 1, N)))
        st = g.solve(1, 0, 1, tol=1e-10, max_cycles=30)
    assert st.relres <= 1e-10
    assert abs(st.cycles - cycles) <= 1, (delta, N, st.cycles, cycles)


def test_linear_coefficient_matches_the_linear_solver():
    # D = 1 and c = 0: the discrete problem is the linear model of Sec. 2, solved by
    # both paths to the same discrete solution
    n, M, T, delta = 127, 64, 0.5, 0.6
    f = inputs.random_field(n, M, seed=61)
    with G.FAS(n, M, T, delta, 0.0, G.MGWR_FAS_D_CONSTANT) as g:
        g.set_rhs(f)
        st = g.solve(1, 1, 1, tol=1e-11, max_cycles=40)
        u = g.solution()
    assert st.relres <= 1e-11
    with G.Solver(1, n, M, T, delta) as s:
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-11, max_cycles=40)
        v = s.solution()
    assert rel(u, v) <= 1e-9


@pytest.mark.parametrize("n,M", [(1, 1), (1, 16), (3, 5)])
def test_edge_sizes(n, M):
    T, delta, c = 1.0, 0.4, 1.0
    f = inputs.random_field(n, M, seed=71)
    with G.FAS(n, M, T, delta, c) as g:
        g.set_rhs(f)
        st = g.solve(1, 0, 1, tol=1e-12, max_cycles=30)
        u = g.solution()
    assert st.relres <= 1e-12
    assert rel(u, fas.time_stepping(n, M, T, delta, f, c=c)) <= 1e-10
    if n == 1:
        assert st.cycles == 1  # the one-point grid is solved exactly


def test_non_finite_rhs_is_reported():
    # the smoother's Newton loop is bounded; a NaN right-hand side ends as a status
    n, M = 15, 8
    f = np.ones((n, M))
    f[3, 2] = np.nan
    with G.FAS(n, M, 1.0, 0.5, 1.0) as g:
        g.set_rhs(f)
        with pytest.raises(G.MGWRError) as e:
            g.solve(1, 0, 1, tol=1e-10, max_cycles=5)
        assert e.value.status == G.MGWR_E_NUMERIC
        # the handle stays usable
        g.set_rhs(np.ones((n, M)))
        assert g.solve(1, 0, 1, tol=1e-10, max_cycles=30).relres <= 1e-10


def test_reset_and_stream_repeat_a_solve():
    import torch
    n, M = 63, 64
    f = np.ones((n, M))
    with G.FAS(n, M, 1.0, 0.4, 1.0) as g:
        g.set_order(G.MGWR_ORDER_TABLE)
        g.set_rhs(f)
        a = g.solve(1, 0, 1, tol=1e-10, max_cycles=30)
        ua = g.solution()
        stream = torch.cuda.Stream()
        g.set_stream(stream.cuda_stream)
        g.reset()
        b = g.solve(1, 0, 1, tol=1e-10, max_cycles=30)
        ub = g.solution()
        g.set_stream(None)
    assert a.cycles == b.cycles
    assert np.array_equal(ua, ub)  # the same kernels on the same data


SMOOTHERS = {"march": G.MGWR_FAS_SMOOTHER_MARCH, "fixed": G.MGWR_FAS_SMOOTHER_FIXED}


@pytest.mark.parametrize("smoother", sorted(SMOOTHERS))
@pytest.mark.parametrize("n,M,c,order", [(31, 128, 1.0, "table"), (63, 256, -2.0, "text"),
                                         (15, 1024, 0.0, "table"), (127, 128, 2.0, "text")])
def test_half_sweep_of_both_smoothers_matches_oracle(smoother, n, M, c, order):
    # the time march (Newton per step) and the whole-line fixed point (one FFT
    # convolution with the inverse column of T_M + sigma I per iteration) both
    # solve each line of the colour to rounding: against the oracle's march
    T, delta = 1.0, 0.45
    W = fas.WRFAS(n, M, T, delta, c=c, order=order)
    u = inputs.random_field(n, M, seed=23, scale=0.3)
    f = inputs.random_field(n, M, seed=24)
    uo = u.copy()
    with G.FAS(n, M, T, delta, c) as g:
        g.set_order(ORDER[order])
        g.set_smoother(SMOOTHERS[smoother])
        L = g.num_levels() - 1
        g.field_set(L, G.MGWR_U, u)
        g.field_set(L, G.MGWR_F, f)
        for colour in (G.MGWR_RED, G.MGWR_BLACK):
            g.smooth(L, colour)
            W.sweep(W.finest, uo, f, colour)
            assert rel(g.field_get(L, G.MGWR_U), uo) <= 1e-12
        iters = g.line_iterations()
    assert (iters > 0) == (smoother == "fixed")


@pytest.mark.parametrize("nu,gamma", [((0, 1), 1), ((1, 1), 2)])
def test_fixed_point_cycles_match_oracle(nu, gamma):
    n, M, T, delta, c = 63, 128, 1.0, 0.4, 1.0
    f = inputs.random_field(n, M, seed=42, scale=4.0)
    W = fas.WRFAS(n, M, T, delta, c=c, order="table")
    uo = np.zeros((n, M))
    with G.FAS(n, M, T, delta, c) as g:
        g.set_order(G.MGWR_ORDER_TABLE)
        g.set_smoother(G.MGWR_FAS_SMOOTHER_FIXED)
        g.set_rhs(f)
        for _ in range(3):
            g.cycle(gamma, *nu)
            uo = W.cycle(W.finest, uo, f, nu[0], nu[1], gamma)
            assert rel(g.solution(), uo) <= 1e-11


def test_smoother_choice_is_checked_and_both_solve_alike():
    with G.FAS(31, 24, 1.0, 0.5, 1.0) as g:  # M not a power of two >= 128: the march only
        with pytest.raises(G.MGWRError):
            g.set_smoother(G.MGWR_FAS_SMOOTHER_FIXED)
        g.set_smoother(G.MGWR_FAS_SMOOTHER_MARCH)
        with pytest.raises(G.MGWRError):
            g.set_smoother(7)
    n, M = 127, 128
    out = []
    for sm in (G.MGWR_FAS_SMOOTHER_MARCH, G.MGWR_FAS_SMOOTHER_FIXED):
        with G.FAS(n, M, 1.0, 0.4, 1.0) as g:
            g.set_order(G.MGWR_ORDER_TABLE)
            g.set_smoother(sm)
            g.set_rhs(np.ones((n, M)))
            st = g.solve(1, 0, 1, tol=1e-10, max_cycles=30)
            out.append((g.solution(), st.cycles))
    assert out[0][1] == out[1][1]
    assert rel(out[1][0], out[0][0]) <= 1e-11


def test_fixed_point_non_finite_rhs_is_reported():
    n, M = 31, 128
    f = np.ones((n, M))
    f[5, 7] = np.nan
    with G.FAS(n, M, 1.0, 0.5, 1.0) as g:
        g.set_smoother(G.MGWR_FAS_SMOOTHER_FIXED)
        g.set_rhs(f)
        with pytest.raises(G.MGWRError) as e:
            g.solve(1, 0, 1, tol=1e-10, max_cycles=3)
        assert e.value.status == G.MGWR_E_NUMERIC
        g.set_rhs(np.ones((n, M)))
        assert g.solve(1, 0, 1, tol=1e-10, max_cycles=30).relres <= 1e-10
