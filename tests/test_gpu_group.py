"""Solves of uneven size advancing together (mgwr_group_*), and handles set up
again for new (T, alpha) in place (mgwr_set_problem).

A group runs every iteration of all its running members as one CUDA graph
launch, each member with exactly the launches of its solo solve, so results
must be bitwise those of solo solves, for members that differ in d, n, M,
alpha, T, precision and cycle, also when members join between iterations.
Every member must also match the oracle's exact discrete solution of its
separable source."""
import numpy as np
import pytest

from oracle import separable
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

# (d, n, M, T, alpha, kind, precision, (cycle, nu1, nu2), tol)
MEMBERS = [
    (1, 63, 64, 1.0, 0.3, "t2", G.MGWR_FP64, (1, 1, 1), 1e-11),
    (2, 31, 128, 1.0, 0.5, "talpha", G.MGWR_MIXED, (1, 1, 1), 1e-9),
    (2, 15, 256, 0.7, 0.7, "t2", G.MGWR_MIXED_DD, (2, 1, 0), 1e-9),
    (1, 255, 512, 1.0, 0.2, "talpha", G.MGWR_DD, (1, 1, 1), 1e-9),
    (2, 63, 64, 2.0, 0.9, "t2", G.MGWR_MIXED, (1, 0, 1), 1e-9),
    (1, 1023, 128, 1.0, 0.6, "t2", G.MGWR_FP64, (1, 1, 1), 1e-10),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _make(m):
    d, n, M, T, alpha, kind, prec, _, _ = m
    s = G.Solver(d, n, M, T, alpha)
    if prec != G.MGWR_FP64:
        s.set_precision(prec)
    s.set_rhs(inputs.Problem(d, n, M, T, alpha, kind).rhs())
    return s


def _solo(m):
    with _make(m) as s:
        cyc, nu1, nu2 = m[7]
        st = s.solve(cyc, nu1, nu2, tol=m[8], max_cycles=60)
        return s.solution(), st


def _ref(m):
    d, n, M, T, alpha, kind = m[:6]
    prob = inputs.Problem(d, n, M, T, alpha, kind)
    return separable.solution(d, n, M, T, alpha, prob.rhs_profile(), inputs.phi(d, n))


def _stats_tuple(st):
    return (st.cycles, st.outer, st.relres, st.status)


def test_group_of_uneven_solves_is_bitwise_solo_and_matches_oracle():
    solo = [_solo(m) for m in MEMBERS]
    solvers = [_make(m) for m in MEMBERS]
    try:
        with G.Group() as g:
            for s, m in zip(solvers, MEMBERS):
                cyc, nu1, nu2 = m[7]
                g.add(s, cyc, nu1, nu2, tol=m[8], max_cycles=60)
            done = dict((id(s), st) for s, st in g.run())
            info = g.info()
        for s, m, (u1, st1) in zip(solvers, MEMBERS, solo):
            st = done[id(s)]
            assert st.status == G.MGWR_OK
            assert _stats_tuple(st) == (st1.cycles, st1.outer, st1.relres, G.MGWR_OK)
            u = s.solution()
            np.testing.assert_array_equal(u, u1)
            ref = _ref(m)
            err = np.abs(u - ref).max() / np.abs(ref).max()
            assert err <= (1e-9 if m[6] == G.MGWR_FP64 else 1e-7), (m, err)
        # one launch served several members, and fewer launches than member iterations
        assert info["max_members"] == len(MEMBERS)
        assert info["member_iterations"] > info["launches"]
    finally:
        for s in solvers:
            s.close()


def test_members_join_between_iterations():
    solo = [_solo(m) for m in MEMBERS[:4]]
    solvers = [_make(m) for m in MEMBERS[:4]]
    try:
        with G.Group() as g:
            for s, m in list(zip(solvers, MEMBERS))[:2]:
                g.add(s, *m[7], tol=m[8], max_cycles=60)
            g.step()
            g.step()
            for s, m in list(zip(solvers, MEMBERS))[2:4]:
                g.add(s, *m[7], tol=m[8], max_cycles=60)
            finished = g.run()
        assert len(finished) == 4
        for s, (u1, st1) in zip(solvers, solo):
            np.testing.assert_array_equal(s.solution(), u1)
    finally:
        for s in solvers:
            s.close()


def test_group_checks_its_members():
    with G.Solver(1, 31, 64, 1.0, 0.5) as a, G.Solver(1, 31, 64, 1.0, 0.5) as b:
        f = inputs.Problem(1, 31, 64, 1.0, 0.5, "t2").rhs()
        a.set_rhs(f)
        b.set_rhs(f)
        with G.Group() as g:
            g.add(a, 1, 1, 1, 1e-10, 40)
            with pytest.raises(G.MGWRError):
                g.add(a, 1, 1, 1, 1e-10, 40)  # already a member
            b.profile(True)
            with pytest.raises(G.MGWRError):
                g.add(b, 1, 1, 1, 1e-10, 40)  # profiled handles run solo only
            b.profile(False)
            g.add(b, 1, 1, 1, 1e-10, 40)
            out = g.run()
        assert [st.status for _, st in out] == [G.MGWR_OK, G.MGWR_OK]
        np.testing.assert_array_equal(a.solution(), b.solution())


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD, G.MGWR_DD])
@pytest.mark.parametrize("d,n,M", [(2, 31, 256), (1, 127, 64), (2, 15, 1024)])
def test_set_problem_solves_as_a_fresh_handle(precision, d, n, M):
    T2, a2 = 0.8, 0.35
    f = inputs.Problem(d, n, M, T2, a2, "talpha").rhs()
    with G.Solver(d, n, M, T2, a2) as fresh:
        fresh.set_precision(precision)
        fresh.set_rhs(f)
        st0 = fresh.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u0 = fresh.solution()
    with G.Solver(d, n, M, 1.0, 0.8) as s:
        s.set_precision(precision)
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-10, max_cycles=40)  # set up and used for another problem
        s.set_problem(T2, a2)
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        np.testing.assert_array_equal(s.solution(), u0)
        assert (st.cycles, st.outer, st.relres) == (st0.cycles, st0.outer, st0.relres)
        s.set_problem(T2, a2)  # the same values: nothing recomputed, same again
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        np.testing.assert_array_equal(s.solution(), u0)
        with pytest.raises(G.MGWRError):
            s.set_problem(1.0, 1.5)
