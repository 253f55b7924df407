"""GPU parity of MGWR_DD, the refinement whose inner cycles run in double-float
arithmetic (the outer defect of the double-float iterate in double-float): the
double-float hierarchy's sweep and defect against the CPU oracle (FP64 direct
sums), whole solves against the oracle's discrete solution, graph replay,
batches, long lines, and its convergence on the fine 1-D grid where FP32 inner
cycles stall (h = 1/4096).

Tolerances: double-float carries about 48 bits; the FFT convolutions keep
about 2^-44 of the operands' scale per value (the lazily renormalised
butterfly sums), so components are checked to 1e-11 of the field's scale and
converged solutions to 1e-10 relative."""
import numpy as np
import pytest

from oracle import direct, mgwr as omg, separable
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

TOLDD = 1e-11


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _dd_solver(d, n, M, T=1.0, alpha=0.45, order=G.MGWR_ORDER_TEXT):
    s = G.Solver(d, n, M, T, alpha)
    s.set_precision(G.MGWR_DD)
    s.set_order(order)
    return s


@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 15, 256), (2, 31, 1024), (1, 7, 4096), (1, 7, 8192)])
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_dd_sweep(d, n, M, order):
    name = "text" if order == G.MGWR_ORDER_TEXT else "table"
    W = omg.WRMG(d, n, M, 1.0, 0.45, order=name) if M <= 4096 else None
    with _dd_solver(d, n, M, order=order) as s:
        l = s.num_levels() - 1
        N = n ** d
        u = inputs.random_field(N, M, seed=10)
        f = inputs.random_field(N, M, seed=20)
        s.field_set(G.MGWR_HDD, l, G.MGWR_U, u)
        s.field_set(G.MGWR_HDD, l, G.MGWR_F, f)
        ref = u.copy()
        for colour in (G.MGWR_RED, G.MGWR_BLACK):
            s.smooth(G.MGWR_HDD, l, colour)
            if W is not None:
                W.sweep(l, ref, f, colour)
                assert rel(s.field_get(G.MGWR_HDD, l, G.MGWR_U), ref) <= TOLDD
        if W is None:  # long lines: against the FP64 hierarchy's partitioned sweep
            with G.Solver(d, n, M, 1.0, 0.45) as s64:
                s64.set_order(order)
                s64.field_set(G.MGWR_H64, l, G.MGWR_U, u)
                s64.field_set(G.MGWR_H64, l, G.MGWR_F, f)
                for colour in (G.MGWR_RED, G.MGWR_BLACK):
                    s64.smooth(G.MGWR_H64, l, colour)
                ref = s64.field_get(G.MGWR_H64, l, G.MGWR_U)
            assert rel(s.field_get(G.MGWR_HDD, l, G.MGWR_U), ref) <= TOLDD


@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 15, 256), (2, 31, 1024), (1, 7, 4096)])
def test_dd_defect(d, n, M):
    W = omg.WRMG(d, n, M, 1.0, 0.45)
    with _dd_solver(d, n, M) as s:
        for l in range(s.num_levels()):
            N = s.level_n(l) ** d
            u = inputs.random_field(N, M, seed=30 + l)
            f = inputs.random_field(N, M, seed=40 + l, scale=W.levels[l].sigma)
            s.field_set(G.MGWR_HDD, l, G.MGWR_U, u)
            s.field_set(G.MGWR_HDD, l, G.MGWR_F, f)
            s.defect(G.MGWR_HDD, l)
            got = s.field_get(G.MGWR_HDD, l, G.MGWR_R)
            ref = W.defect(l, u, f)
            scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(u).max()
            assert np.abs(got - ref).max() <= TOLDD * scale, (l, np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("d,n,M,kind", [(2, 63, 128, "t2"), (1, 255, 1024, "talpha"), (2, 31, 4096, "t2")])
def test_dd_solve_matches_oracle(d, n, M, kind):
    prob = inputs.Problem(d, n, M, 1.0, 0.5, kind)
    f = prob.rhs()
    with _dd_solver(d, n, M, alpha=0.5) as s:
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-11, max_cycles=40, allow_noconv=True)
        u = s.solution()
        r64 = s.residual()
    assert st.relres <= 1e-10 and r64 <= 1e-10
    if M <= 128:
        ref = direct.time_stepping(d, n, M, 1.0, 0.5, f)
    else:
        ref = separable.solution(d, n, M, 1.0, 0.5, prob.rhs_profile(), inputs.phi(d, n))
    assert rel(u, ref) <= 1e-10


def test_dd_converges_like_fp64():
    # the inner double-float cycles reduce the defect as FP64 cycles do: the count
    # (inner cycles, two per outer step) rounds the FP64 count up to an outer step
    d, n, M = 2, 127, 512
    f = inputs.Problem(d, n, M, 1.0, 0.5, "t2").rhs()
    out = {}
    for prec in (G.MGWR_FP64, G.MGWR_DD):
        with G.Solver(d, n, M, 1.0, 0.5) as s:
            s.set_precision(prec)
            s.set_rhs(f)
            out[prec] = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
    assert out[G.MGWR_DD].cycles <= out[G.MGWR_FP64].cycles + 2


@pytest.mark.parametrize("cyc", [(1, 1, 1), (0, 1, 1), (1, 0, 2)])
def test_dd_graph_replayed_solve_equals_direct_launches(cyc):
    nu1, nu2, gamma = cyc
    d, n, M = 2, 31, 64
    f = inputs.Problem(d, n, M, 1.0, 0.4, "t2").rhs()
    res = []
    for graphs in (True, False):
        with _dd_solver(d, n, M, alpha=0.4) as s:
            s.set_graphs(graphs)
            s.set_rhs(f)
            st = s.solve(gamma, nu1, nu2, tol=1e-10, max_cycles=40)
            res.append((s.solution(), st.cycles, st.relres))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1:] == res[1][1:]


def test_dd_batch_matches_oracle_per_instance():
    d, n, M = 2, 31, 64
    TS, ALPHAS = [1.0, 0.7, 2.0], [0.15, 0.5, 0.85]
    f = np.stack([inputs.Problem(d, n, M, T, a, "t2").rhs() for T, a in zip(TS, ALPHAS)])
    with G.Solver(d, n, M, TS, ALPHAS) as s:
        s.set_precision(G.MGWR_DD)
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-11, max_cycles=40, allow_noconv=True)
        u = s.solution()
    for b, (T, a) in enumerate(zip(TS, ALPHAS)):
        assert rel(u[b], direct.time_stepping(d, n, M, T, a, f[b])) <= 1e-10, b


def test_dd_fine_1d_grid_where_fp32_cycles_stall():
    # h = 1/4096: FP32 rounding of the correction caps the mixed refinement at about
    # 0.4 per outer step; double-float cycles converge like FP64 (partitioned lines)
    d, n, M, alpha = 1, 4095, 8192, 0.2
    prob = inputs.Problem(d, n, M, 1.0, alpha, "talpha")
    stats = {}
    for prec in (G.MGWR_FP64, G.MGWR_DD):
        with G.Solver(d, n, M, 1.0, alpha) as s:
            s.set_precision(prec)
            s.set_rhs(prob.rhs())
            stats[prec] = s.solve(1, 1, 1, tol=1e-8, max_cycles=40)
            if prec == G.MGWR_DD:
                u = s.solution()
    assert stats[G.MGWR_DD].cycles <= stats[G.MGWR_FP64].cycles + 2
    ref = separable.solution(d, n, M, 1.0, alpha, prob.rhs_profile(), inputs.phi(d, n))
    assert rel(u, ref) <= 1e-7


def test_auto_precision_resolves_on_the_handle_and_converges():
    # MGWR_AUTO: double-float inner cycles on h = 1/4096, the FP32 refinement on h = 1/256.
    # On h = 1/4096 the double-float iterate's own rounding, amplified by 4/h^2, leaves
    # a relative defect of a few 1e-9: the tolerance there is 1e-8.
    for d, n, M, want, tol in [(1, 4095, 256, G.MGWR_DD, 1e-8), (2, 255, 64, G.MGWR_MIXED_DD, 1e-10)]:
        prob = inputs.Problem(d, n, M, 1.0, 0.3, "talpha")
        with G.Solver(d, n, M, 1.0, 0.3) as s:
            s.set_precision(G.MGWR_AUTO)
            assert s.precision() == want == G.auto_precision(d, n, M)
            s.set_rhs(prob.rhs())
            st = s.solve(1, 1, 1, tol=tol, max_cycles=40)
            u = s.solution()
        assert st.outer <= 6, (d, n, st.outer)
        ref = separable.solution(d, n, M, 1.0, 0.3, prob.rhs_profile(), inputs.phi(d, n))
        assert rel(u, ref) <= 100 * tol


def test_double_float_split_is_the_rounded_pair():
    # A MGWR_MIXED_DD solve holds its iterate as double-float pairs split on the
    # device and joins them back at its end; with a tolerance the first defect
    # already meets (relative defect 1 <= 2) it stops before any cycle, so the
    # solution is hi + lo of the split of every value: hi = RN32(x) (ties to
    # even), lo = RN32(x - hi), formed by integer and FP32 operations on the
    # device and here by IEEE conversions.  Values: rounding ties and their
    # neighbours, signed zeros, the ends of the integer path's exponent range
    # (2^-74) and beyond it (smaller, subnormal), random magnitudes 2^-80..2^60.
    d, n, M = 1, 63, 64
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n * M) * np.exp2(rng.integers(-80, 61, n * M).astype(float))
    one = 1.0
    special = [0.0, -0.0, one + 2.0 ** -24, one + 3 * 2.0 ** -24, -(one + 3 * 2.0 ** -24),
               one + 2.0 ** -24 + 2.0 ** -52, one + 2.0 ** -24 - 2.0 ** -53, 3.0 - 2.0 ** -23,
               (2.0 - 2.0 ** -24) * 2.0 ** 40, 2.0 ** -74, 1.5 * 2.0 ** -74, 2.0 ** -75,
               -1.25 * 2.0 ** -75, 1e-30, 5e-324, -1e-310, 2.0 ** 59 * (1 + 2.0 ** -30)]
    x[:len(special)] = special
    u0 = x.reshape(n, M)
    with G.Solver(d, n, M, 1.0, 0.5) as s:
        s.set_precision(G.MGWR_MIXED_DD)
        s.set_rhs(np.zeros((n, M)))
        s.set_initial(u0)
        st = s.solve(1, 1, 1, tol=2.0, max_cycles=4)
        got = s.solution()
    assert st.cycles == 0
    hi = u0.astype(np.float32)
    lo = (u0 - hi.astype(np.float64)).astype(np.float32)
    want = hi.astype(np.float64) + lo.astype(np.float64)
    np.testing.assert_array_equal(got.view(np.uint64), want.view(np.uint64))
