"""Batched instances: one handle, many same-shape problems with their own T and
alpha, every kernel launch serving all of them.  Each instance must behave
exactly as the same problem solved alone (same kernels, same arithmetic), and
match the oracle."""
import numpy as np
import pytest

from oracle import direct, l1, toeplitz
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


ALPHAS = [0.15, 0.5, 0.85]
TS = [1.0, 0.7, 2.0]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


@pytest.mark.parametrize("d,n,M", [(2, 15, 64), (1, 31, 128)])
def test_batched_setup_per_instance(d, n, M):
    with G.Solver(d, n, M, TS, ALPHAS) as s:
        r = s.toeplitz_column()
        k = s.inverse_column(s.num_levels() - 1)
    for b, (T, a) in enumerate(zip(TS, ALPHAS)):
        ref = l1.toeplitz_column(a, T, M)
        assert np.abs(r[b] - ref).max() <= 1e-14 * abs(ref[0])
        sigma = 2.0 * d * (n + 1) ** 2
        assert rel(k[b], toeplitz.inverse_column(a, T, M, sigma)) <= 1e-13


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("d,n,M,cyc", [(2, 15, 32, (1, 1, 1)), (1, 31, 64, (0, 1, 2))])
def test_batched_cycles_equal_single_instance_cycles(hier, d, n, M, cyc):
    nu1, nu2, gamma = cyc
    N = n ** d
    f = np.stack([inputs.random_field(N, M, seed=100 + b) for b in range(len(ALPHAS))])
    with G.Solver(d, n, M, TS, ALPHAS) as sb:
        if hier == G.MGWR_H32:
            sb.set_precision(G.MGWR_MIXED)
        L = sb.num_levels() - 1
        sb.field_set(hier, L, G.MGWR_F, f)
        sb.field_set(hier, L, G.MGWR_U, np.zeros_like(f))
        for _ in range(3):
            sb.cycle(hier, gamma, nu1, nu2)
        ub = sb.field_get(hier, L, G.MGWR_U)
    for b, (T, a) in enumerate(zip(TS, ALPHAS)):
        with G.Solver(d, n, M, T, a) as s1:
            if hier == G.MGWR_H32:
                s1.set_precision(G.MGWR_MIXED)
            s1.field_set(hier, L, G.MGWR_F, f[b])
            s1.field_set(hier, L, G.MGWR_U, np.zeros_like(f[b]))
            for _ in range(3):
                s1.cycle(hier, gamma, nu1, nu2)
            np.testing.assert_array_equal(ub[b], s1.field_get(hier, L, G.MGWR_U))


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD])
def test_batched_solve_matches_oracle(precision):
    d, n, M = 2, 31, 64
    probs = [inputs.Problem(d, n, M, T, a, "t2") for T, a in zip(TS, ALPHAS)]
    f = np.stack([p.rhs() for p in probs])
    with G.Solver(d, n, M, TS, ALPHAS) as s:
        s.set_precision(precision)
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-12, max_cycles=40, allow_noconv=True)
        u = s.solution()
        per = s.instance_relres()
    assert per.shape == (3,) and per.max() == st.relres and st.relres <= 2e-12
    for b, (T, a) in enumerate(zip(TS, ALPHAS)):
        ref = direct.time_stepping(d, n, M, T, a, f[b])
        assert rel(u[b], ref) <= (1e-11 if precision == G.MGWR_FP64 else 1e-9), b


def test_batched_initial_condition_per_instance():
    d, n, M = 1, 15, 32
    g = np.stack([inputs.phi(d, n) * (1 + b) for b in range(3)])
    f = np.stack([inputs.random_field(n, M, seed=7 + b) for b in range(3)])
    with G.Solver(d, n, M, TS, ALPHAS) as s:
        s.set_rhs(f, g)
        s.solve(1, 1, 1, tol=1e-12, max_cycles=40, allow_noconv=True)
        u = s.solution()
    for b, (T, a) in enumerate(zip(TS, ALPHAS)):
        assert rel(u[b], direct.time_stepping(d, n, M, T, a, f[b], g[b])) <= 1e-11
