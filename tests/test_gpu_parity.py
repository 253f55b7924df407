"""GPU parity: every CUDA component, called through the C ABI, against the CPU
oracle on the same seeded inputs.

Tolerances.  FP64 kernels evaluate the time-line products by FFT (Sec. 5); the
oracle uses dense triangular solves and direct sums.  Both round in FP64, so
their difference is a few ulps of the operands' scale times log2(2M): the
tests use 1e-12 relative to the field's max (about 50x that bound).  FP32
kernels: 2e-5 relative (FP32 unit roundoff 6e-8 times the same growth).  Full
solves: 1e-11 relative to max |u| once the defect stagnates at its rounding
floor (about 1e-12 relative for these grids: eps * 2d/h^2 * |u| / |f|).
"""
import numpy as np
import pytest

from oracle import direct, l1, mgwr as omg, separable, toeplitz
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def order_name(order):
    return "text" if order == G.MGWR_ORDER_TEXT else "table"


# ---------------------------------------------------------------------------------
# setup: coefficients, inverse columns
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.1, 0.5, 0.9, 1.0])
@pytest.mark.parametrize("M", [4, 64, 1024, 4096])
def test_toeplitz_column(alpha, M):
    with G.Solver(1, 7, M, 1.3, alpha) as s:
        r = s.toeplitz_column()
    ref = l1.toeplitz_column(alpha, 1.3, M)
    assert np.abs(r - ref).max() <= 1e-14 * abs(ref[0])
    # elementwise: both sides are within a few ulps of c*d_i, the scale of the two
    # weights whose difference r_i is (the oracle subtracts, the GPU sums a series)
    c = l1.l1_scale(alpha, 1.3, M)
    dk = l1.l1_weights(alpha, M)
    assert np.all(np.abs(r - ref) <= 2e-15 * c * np.maximum(dk[1:], dk[:-1]))


@pytest.mark.parametrize("d,n,M,alpha", [(1, 63, 64, 0.5), (2, 31, 1024, 0.3), (2, 7, 4096, 0.8), (1, 3, 4, 0.5)])
def test_inverse_columns(d, n, M, alpha):
    with G.Solver(d, n, M, 1.0, alpha) as s:
        for l in range(s.num_levels()):
            nl = s.level_n(l)
            sigma = 2.0 * d * (nl + 1) ** 2
            k = s.inverse_column(l)
            ref = toeplitz.inverse_column(alpha, 1.0, M, sigma)
            assert rel(k, ref) <= 1e-13, (l, rel(k, ref))


# ---------------------------------------------------------------------------------
# components at one level, FP64 and FP32
# ---------------------------------------------------------------------------------

CASES = [(1, 63, 64), (1, 15, 8), (1, 7, 16), (1, 31, 32), (2, 15, 64), (2, 7, 128), (2, 31, 256),
         (2, 3, 4), (1, 3, 4096), (2, 3, 2048)]


def _setup(d, n, M, alpha=0.45, T=1.0, hier=G.MGWR_H64, order=G.MGWR_ORDER_TEXT):
    s = G.Solver(d, n, M, T, alpha)
    if hier == G.MGWR_H32:
        s.set_precision(G.MGWR_MIXED)
    s.set_order(order)
    W = omg.WRMG(d, n, M, T, alpha, order=order_name(order))
    return s, W


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", CASES)
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_sweep(hier, d, n, M, order):
    s, W = _setup(d, n, M, hier=hier, order=order)
    with s:
        for l in range(1, s.num_levels()):
            N = s.level_n(l) ** d
            u = inputs.random_field(N, M, seed=10 + l)
            f = inputs.random_field(N, M, seed=20 + l)
            s.field_set(hier, l, G.MGWR_U, u)
            s.field_set(hier, l, G.MGWR_F, f)
            ref = u.copy()
            for colour in (G.MGWR_RED, G.MGWR_BLACK):
                s.smooth(hier, l, colour)
                W.sweep(l, ref, f, colour)
                got = s.field_get(hier, l, G.MGWR_U)
                tol = TOL64 if hier == G.MGWR_H64 else TOL32
                assert rel(got, ref) <= tol, (l, colour, rel(got, ref))


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", CASES)
def test_defect(hier, d, n, M):
    s, W = _setup(d, n, M, hier=hier)
    with s:
        for l in range(s.num_levels()):
            N = s.level_n(l) ** d
            u = inputs.random_field(N, M, seed=30 + l)
            f = inputs.random_field(N, M, seed=40 + l, scale=W.levels[l].sigma)
            s.field_set(hier, l, G.MGWR_U, u)
            s.field_set(hier, l, G.MGWR_F, f)
            nrm = s.defect(hier, l)
            got = s.field_get(hier, l, G.MGWR_R)
            ref = W.defect(l, u, f)
            scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(u).max()
            tol = TOL64 if hier == G.MGWR_H64 else TOL32
            assert np.abs(got - ref).max() <= tol * scale
            assert abs(nrm - np.abs(got).max()) <= 1e-15 * max(nrm, 1.0) or hier == G.MGWR_H32


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 31, 256), (2, 15, 8), (1, 7, 4096)])
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_defect_after_smoothing_step_without_convolution(hier, d, n, M, order):
    # one red-black step, then the defect from the black changes, against the oracle's
    # two half-sweeps followed by its direct-sum defect
    s, W = _setup(d, n, M, hier=hier, order=order)
    with s:
        for l in range(1, s.num_levels()):
            N = s.level_n(l) ** d
            u = inputs.random_field(N, M, seed=80 + l)
            f = inputs.random_field(N, M, seed=90 + l, scale=W.levels[l].sigma)
            s.field_set(hier, l, G.MGWR_U, u)
            s.field_set(hier, l, G.MGWR_F, f)
            nrm = s.smooth_defect(hier, l)
            ref_u = u.copy()
            W.smooth(l, ref_u, f, 1)
            ref_r = W.defect(l, ref_u, f)
            got = s.field_get(hier, l, G.MGWR_R)
            scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(ref_u).max()
            tol = TOL64 if hier == G.MGWR_H64 else TOL32
            assert np.abs(got - ref_r).max() <= tol * scale, (l, np.abs(got - ref_r).max() / scale)
            assert rel(s.field_get(hier, l, G.MGWR_U), ref_u) <= tol
            if hier == G.MGWR_H64:
                assert nrm == np.abs(got).max()


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 31, 32), (2, 15, 4)])
def test_restrict_and_prolong(hier, d, n, M):
    s, W = _setup(d, n, M, hier=hier)
    with s:
        for l in range(1, s.num_levels()):
            nl, nc = s.level_n(l), s.level_n(l - 1)
            r = inputs.random_field(nl ** d, M, seed=50 + l)
            e = inputs.random_field(nc ** d, M, seed=60 + l)
            u = inputs.random_field(nl ** d, M, seed=70 + l)
            s.field_set(hier, l, G.MGWR_R, r)
            s.field_set(hier, l - 1, G.MGWR_U, e)
            s.restrict(hier, l)
            tol = 1e-15 if hier == G.MGWR_H64 else 1e-6
            assert rel(s.field_get(hier, l - 1, G.MGWR_F), omg.restrict_fw(r, d, nl)) <= tol
            assert not s.field_get(hier, l - 1, G.MGWR_U).any()  # restriction clears e
            s.field_set(hier, l - 1, G.MGWR_U, e)
            s.field_set(hier, l, G.MGWR_U, u)
            s.prolong(hier, l)
            ref = u + omg.prolong_linear(e, d, nc)
            assert rel(s.field_get(hier, l, G.MGWR_U), ref) <= tol


@pytest.mark.parametrize("d,M", [(1, 64), (2, 256), (1, 4)])
def test_coarsest_solve(d, M):
    s, W = _setup(d, 15, M)
    with s:
        f = inputs.random_field(1, M, seed=3)
        s.field_set(G.MGWR_H64, 0, G.MGWR_F, f)
        s.coarsest(G.MGWR_H64)
        assert rel(s.field_get(G.MGWR_H64, 0, G.MGWR_U), W.coarsest_solve(f)) <= TOL64


# ---------------------------------------------------------------------------------
# whole cycles and solves
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,M,cyc", [(1, 63, 64, (1, 1, 1)), (1, 31, 32, (0, 1, 1)), (2, 31, 64, (1, 1, 1)),
                                       (2, 15, 16, (1, 0, 2)), (2, 7, 8, (2, 1, 2))])
def test_cycles_match_oracle_iterates(d, n, M, cyc):
    nu1, nu2, gamma = cyc
    s, W = _setup(d, n, M, alpha=0.6)
    with s:
        L = s.num_levels() - 1
        f = inputs.random_field(n ** d, M, seed=5)
        u = np.zeros_like(f)
        s.field_set(G.MGWR_H64, L, G.MGWR_F, f)
        s.field_set(G.MGWR_H64, L, G.MGWR_U, u)
        for k in range(4):
            s.cycle(G.MGWR_H64, gamma, nu1, nu2)
            u = W.cycle(L, u, f, nu1, nu2, gamma)
            got = s.field_get(G.MGWR_H64, L, G.MGWR_U)
            assert rel(got, u) <= 1e-11, (k, rel(got, u))


@pytest.mark.parametrize("kind", ["t2", "talpha"])
def test_solve_1d_config_matches_oracle_solution(kind):
    # 1-D plain MGWR: 63 interior points, M = 64, alpha = 0.5, u = t^2 sin(pi x)
    prob = inputs.Problem(1, 63, 64, 1.0, 0.5, kind)
    f = prob.rhs()
    with G.Solver(1, 63, 64, 1.0, 0.5) as s:
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-13, max_cycles=30, allow_noconv=True)
        u = s.solution()
        relres = s.residual()
    ref = direct.time_stepping(1, 63, 64, 1.0, 0.5, f)
    assert st.relres <= 2e-12 and relres == st.relres
    assert rel(u, ref) <= 1e-11


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_solve_2d_subcase_matches_oracle_solution(alpha):
    # 2-D subcase 63 x 63, M = 128, of the 255 x 255, M = 1024 configuration
    prob = inputs.Problem(2, 63, 128, 1.0, alpha, "t2")
    f = prob.rhs()
    with G.Solver(2, 63, 128, 1.0, alpha) as s:
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-13, max_cycles=30, allow_noconv=True)
        u = s.solution()
    ref = direct.time_stepping(2, 63, 128, 1.0, alpha, f)
    assert st.relres <= 2e-12
    assert rel(u, ref) <= 1e-11


def test_solve_with_initial_condition_matches_oracle():
    d, n, M, alpha = 1, 31, 32, 0.4
    g = inputs.phi(d, n) + 0.3 * inputs.random_field(n, 1, seed=8)[:, 0]
    f = inputs.random_field(n, M, seed=9)
    with G.Solver(d, n, M, 1.0, alpha) as s:
        s.set_rhs(f, g)
        s.solve(1, 0, 1, tol=1e-13, max_cycles=60, allow_noconv=True)
        u = s.solution()
    ref = direct.time_stepping(d, n, M, 1.0, alpha, f, g)
    assert rel(u, ref) <= 1e-11


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_full_size_2d_config_against_separable_solution(alpha):
    # 255 x 255 interior grid, M = 1024: the exact discrete solution is separable
    d, n, M = 2, 255, 1024
    prob = inputs.Problem(d, n, M, 1.0, alpha, "t2")
    with G.Solver(d, n, M, 1.0, alpha) as s:
        s.set_rhs(prob.rhs())
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u = s.solution()
    ref = separable.solution(d, n, M, 1.0, alpha, prob.rhs_profile(), inputs.phi(d, n))
    assert st.relres <= 1e-10
    assert 8 <= st.cycles <= 16
    assert rel(u, ref) <= 1e-9


def test_mixed_precision_solve_matches_oracle():
    d, n, M, alpha = 2, 63, 128, 0.5
    prob = inputs.Problem(d, n, M, 1.0, alpha, "talpha")
    f = prob.rhs()
    with G.Solver(d, n, M, 1.0, alpha) as s:
        s.set_precision(G.MGWR_MIXED)
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u = s.solution()
    ref = direct.time_stepping(d, n, M, 1.0, alpha, f)
    assert st.relres <= 1e-10
    assert rel(u, ref) <= 1e-8


@pytest.mark.parametrize("d,n,M,kind", [(2, 63, 128, "talpha"), (1, 255, 1024, "t2"), (2, 31, 4096, "t2")])
def test_mixed_double_float_solve_matches_oracle(d, n, M, kind):
    # FP32 cycles, double-float defect and update: same converged solution; the
    # IEEE-double defect of the result agrees with the double-float stopping test
    prob = inputs.Problem(d, n, M, 1.0, 0.5, kind)
    f = prob.rhs()
    with G.Solver(d, n, M, 1.0, 0.5) as s:
        s.set_precision(G.MGWR_MIXED_DD)
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u = s.solution()
        r64 = s.residual()
    ref = separable.solution(d, n, M, 1.0, 0.5, prob.rhs_profile(), inputs.phi(d, n))
    assert st.relres <= 1e-10 and r64 <= 2e-10
    assert rel(u, ref) <= 1e-8


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("cyc", [(1, 1, 1), (0, 1, 1), (1, 0, 2)])
def test_graph_replayed_solve_equals_direct_launches(precision, cyc):
    nu1, nu2, gamma = cyc
    d, n, M = 2, 31, 64
    f = inputs.Problem(d, n, M, 1.0, 0.4, "t2").rhs()
    out = []
    for graphs in (True, False):
        with G.Solver(d, n, M, 1.0, 0.4) as s:
            s.set_precision(precision)
            s.set_graphs(graphs)
            s.set_rhs(f)
            st = s.solve(gamma, nu1, nu2, tol=1e-10, max_cycles=40)
            out.append((s.solution(), st.cycles, st.relres))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_colour_order_switch_on_one_handle():
    # the black-change field keeps values from the other colour after a switch;
    # defects computed from it must still ignore red lines and the boundary
    d, n, M = 1, 63, 64
    f = inputs.Problem(d, n, M, 1.0, 0.5, "t2").rhs()
    ref = direct.time_stepping(d, n, M, 1.0, 0.5, f)
    with G.Solver(d, n, M, 1.0, 0.5) as s:
        for order in (G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE, G.MGWR_ORDER_TEXT):
            s.set_order(order)
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-12, max_cycles=40, allow_noconv=True)
            assert st.relres <= 2e-12
            assert rel(s.solution(), ref) <= 1e-11


def test_paper_table_1d_iterations_on_gpu():
    # Table table_it_1d, V(0,1), delta = 0.4, 128 x 128 grid: 7 cycles (table order)
    import math
    delta, n, M = 0.4, 127, 128
    T = math.pi ** (-2.0 / delta)
    g = inputs.phi(1, n)
    with G.Solver(1, n, M, T, delta) as s:
        s.set_order(G.MGWR_ORDER_TABLE)
        s.set_rhs(np.zeros((n, M)), g)
        st = s.solve(1, 0, 1, tol=1e-10, max_cycles=40)
    assert abs(st.cycles - 7) <= 1


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD])
def test_solve_from_zero_skips_nothing_it_needs(precision):
    # from u = 0 the initial defect is f itself and is not convolved; the solve must
    # be the one that starts from an explicitly set zero iterate: bitwise, except
    # in MGWR_MIXED, whose explicit start computes f - A 0 with the double-float
    # convolution and so holds the same carried defect in another double-float
    # pair (the same value to 2^-48)
    d, n, M = 2, 31, 128
    f = inputs.Problem(d, n, M, 1.0, 0.6, "talpha").rhs()
    out = []
    for explicit in (False, True):
        with G.Solver(d, n, M, 1.0, 0.6) as s:
            s.set_precision(precision)
            s.set_rhs(f)
            if explicit:
                s.set_initial(np.zeros_like(f))
            st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
            out.append((s.solution(), st.cycles, st.outer, st.relres))
    if precision == G.MGWR_MIXED:
        assert rel(out[0][0], out[1][0]) <= 1e-12
    else:
        np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1:3] == out[1][1:3]
    # the double-float defect reports its norm from the leading FP32 word, so r_0
    # from the explicit zero iterate differs from max |f| in the 8th digit; the
    # stop of MGWR_MIXED to 1e-10 is decided on its double-float-convolution
    # defect, good to about 2^-44 of |T_M u| (f's scale) in either run
    anchor = 2.0 ** -40 if precision == G.MGWR_MIXED else 0.0
    assert abs(out[0][3] - out[1][3]) <= 1e-6 * out[1][3] + anchor
    assert rel(out[0][0], direct.time_stepping(d, n, M, 1.0, 0.6, f)) <= (1e-11 if precision == G.MGWR_FP64 else 1e-8)
