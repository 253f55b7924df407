"""GPU parity for long time lines (M > 4096), where every time-line product is
a partitioned convolution over blocks of 4096 steps: setup, each component
through the C ABI against the CPU oracle, whole solves against the exact
discrete solution, and the 1-D 4095-point, M = 65536 workload at full size.

References.  Sweep: (T_M + sigma I)^{-1} b as the causal product of b with the
oracle's inverse column (forward substitution, Sec. 5 smoothing procedure),
evaluated by direct sums.  Defect: f - T_M u - A_h u with the oracle's Toeplitz
column, direct sums and sparse Laplacian.  Solves: the time-stepping oracle on
small grids, the separable solution (forward substitution in time) at full
size.  Tolerances as for the short lines (FP64 1e-12 of the field's scale,
FP32 2e-5): the block sums add one more FFT-length factor at most.
"""
import numpy as np
import pytest

from oracle import direct, l1, mgwr as omg, separable, toeplitz
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
ALPHA, T = 0.35, 1.0


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _solver(d, n, M, hier, order=G.MGWR_ORDER_TEXT, alpha=ALPHA):
    s = G.Solver(d, n, M, T, alpha)
    if hier == G.MGWR_H32:
        s.set_precision(G.MGWR_MIXED)
    s.set_order(order)
    return s


def _inverse_column(d, nl, M, alpha=ALPHA):
    return toeplitz.inverse_column(alpha, T, M, 2.0 * d * (nl + 1) ** 2)


@pytest.mark.parametrize("M", [8192, 65536])
def test_setup_columns_long(M):
    with G.Solver(1, 7, M, T, 0.2) as s:
        r = s.toeplitz_column()
        ref = l1.toeplitz_column(0.2, T, M)
        assert np.abs(r - ref).max() <= 1e-14 * abs(ref[0])
        for l in range(s.num_levels()):
            k = s.inverse_column(l)
            assert rel(k, _inverse_column(1, s.level_n(l), M, 0.2)) <= 1e-12, l


SWEEP_CASES = [(1, 7, 8192), (2, 3, 8192), (1, 3, 16384)]


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", SWEEP_CASES)
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_sweep_long(hier, d, n, M, order):
    with _solver(d, n, M, hier, order) as s:
        for l in range(1, s.num_levels()):
            nl = s.level_n(l)
            N = nl ** d
            k = _inverse_column(d, nl, M)
            u = inputs.random_field(N, M, seed=10 + l)
            f = inputs.random_field(N, M, seed=20 + l)
            s.field_set(hier, l, G.MGWR_U, u)
            s.field_set(hier, l, G.MGWR_F, f)
            ref = u.copy()
            for colour in (G.MGWR_RED, G.MGWR_BLACK):
                s.smooth(hier, l, colour)
                mask = omg.colour_mask(d, nl, colour, "text" if order == G.MGWR_ORDER_TEXT else "table")
                b = f + (nl + 1) ** 2 * omg.neighbour_sum(ref, d, nl)
                ref[mask] = toeplitz.causal_apply(k, b[mask])
                got = s.field_get(hier, l, G.MGWR_U)
                tol = TOL64 if hier == G.MGWR_H64 else TOL32
                assert rel(got, ref) <= tol, (l, colour, rel(got, ref))


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", SWEEP_CASES)
def test_defect_long(hier, d, n, M):
    rcol = l1.toeplitz_column(ALPHA, T, M)
    with _solver(d, n, M, hier) as s:
        for l in range(s.num_levels()):
            nl = s.level_n(l)
            N = nl ** d
            sigma = 2.0 * d * (nl + 1) ** 2
            u = inputs.random_field(N, M, seed=30 + l)
            f = inputs.random_field(N, M, seed=40 + l, scale=sigma)
            s.field_set(hier, l, G.MGWR_U, u)
            s.field_set(hier, l, G.MGWR_F, f)
            nrm = s.defect(hier, l)
            got = s.field_get(hier, l, G.MGWR_R)
            ref = f - toeplitz.causal_apply(rcol, u) - direct.laplacian(d, nl) @ u
            scale = np.abs(f).max() + sigma * 2 * np.abs(u).max()
            tol = TOL64 if hier == G.MGWR_H64 else TOL32
            assert np.abs(got - ref).max() <= tol * scale, (l, np.abs(got - ref).max() / scale)
            if hier == G.MGWR_H64:
                assert nrm == np.abs(got).max()


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_defect_after_smoothing_step_long(hier, order):
    # the black change recorded by the partitioned sweep feeds the defect without
    # a convolution; compared with the defect of the reference step
    d, n, M = 1, 7, 8192
    rcol = l1.toeplitz_column(ALPHA, T, M)
    with _solver(d, n, M, hier, order) as s:
        l = s.num_levels() - 1
        N = n ** d
        sigma = 2.0 * d * (n + 1) ** 2
        k = _inverse_column(d, n, M)
        u = inputs.random_field(N, M, seed=81)
        f = inputs.random_field(N, M, seed=91, scale=sigma)
        s.field_set(hier, l, G.MGWR_U, u)
        s.field_set(hier, l, G.MGWR_F, f)
        s.smooth_defect(hier, l)
        ref = u.copy()
        name = "text" if order == G.MGWR_ORDER_TEXT else "table"
        for colour in (G.MGWR_RED, G.MGWR_BLACK):
            mask = omg.colour_mask(d, n, colour, name)
            b = f + (n + 1) ** 2 * omg.neighbour_sum(ref, d, n)
            ref[mask] = toeplitz.causal_apply(k, b[mask])
        ref_r = f - toeplitz.causal_apply(rcol, ref) - direct.laplacian(d, n) @ ref
        got = s.field_get(hier, l, G.MGWR_R)
        scale = np.abs(f).max() + sigma * 2 * np.abs(ref).max()
        tol = TOL64 if hier == G.MGWR_H64 else TOL32
        assert np.abs(got - ref_r).max() <= tol * scale


@pytest.mark.parametrize("M", [8192, 16384])
def test_coarsest_solve_long(M):
    with _solver(1, 3, M, G.MGWR_H64) as s:
        f = inputs.random_field(1, M, seed=3)
        s.field_set(G.MGWR_H64, 0, G.MGWR_F, f)
        s.coarsest(G.MGWR_H64)
        ref = toeplitz.causal_apply(_inverse_column(1, 1, M), f)
        assert rel(s.field_get(G.MGWR_H64, 0, G.MGWR_U), ref) <= TOL64


def test_solve_long_random_rhs_matches_time_stepping():
    d, n, M = 1, 7, 8192
    f = inputs.random_field(n, M, seed=12)
    with G.Solver(d, n, M, T, ALPHA) as s:
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-12, max_cycles=40, allow_noconv=True)
        u = s.solution()
    assert st.relres <= 2e-12
    assert rel(u, direct.time_stepping(d, n, M, T, ALPHA, f)) <= 1e-11


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M", [(1, 31, 16384), (2, 15, 8192)])
def test_solve_long_separable(precision, d, n, M):
    prob = inputs.Problem(d, n, M, T, 0.2, "talpha")
    with G.Solver(d, n, M, T, 0.2) as s:
        s.set_precision(precision)
        s.set_rhs(prob.rhs())
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u = s.solution()
    ref = separable.solution(d, n, M, T, 0.2, prob.rhs_profile(), inputs.phi(d, n))
    assert st.relres <= 1e-10
    assert rel(u, ref) <= (1e-9 if precision == G.MGWR_FP64 else 1e-8)


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED_DD])
def test_full_size_long_memory_1d(precision):
    # 1-D, 4095 interior points, M = 65536, alpha = 0.2, u = t^alpha sin(pi x):
    # the whole field against the separable exact discrete solution
    d, n, M, alpha = 1, 4095, 65536, 0.2
    prob = inputs.Problem(d, n, M, T, alpha, "talpha")
    with G.Solver(d, n, M, T, alpha) as s:
        s.set_precision(precision)
        s.set_rhs(prob.rhs())
        st = s.solve(1, 1, 1, tol=1e-8, max_cycles=40)
        u = s.solution()
    w = separable.time_factor(d, n, M, T, alpha, prob.rhs_profile())
    ref = np.outer(inputs.phi(d, n), w)
    assert st.relres <= 1e-8
    assert rel(u, ref) <= 1e-7
