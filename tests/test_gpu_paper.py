"""The paper's experiments run through the C ABI at the paper's own sizes:
Table table_it_1d (V(0,1), 128^2 .. 2048^2), Table table_it_2d (V(1,1),
32^3 .. 256^3), the measured W-cycle factors of Table lambdas_m (random
initial guess, zero right-hand side), and the first experiment's exact
solution u = E_alpha(-t^alpha) sin x, whose L1 error falls as tau^alpha
(Sec. 7).  Stored values: tests/golden/ (the paper's, cited there)."""
import math
import os

import numpy as np
import pytest

from oracle import l1, separable
from oracle.mittag_leffler import mittag_leffler
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _paper_1d(delta, n, M):
    # f = 0, g = sin x on [0, pi] x [0, 1], mapped to (0,1): x -> x / pi, t -> t pi^(-2/delta).
    # The initial value enters the right-hand side as c d_m g (Sec. 2, Eq. L1_scheme2) and
    # the solve starts from u = 0: from u^0 = g the initial defect is only -A_h g
    # (T_M g = c d_m g), about pi^2 |g|, and the FP64 rounding floor of the defect,
    # eps 4/h^2 |u|, reaches 1e-10 of it at h = 1/2048.
    T = math.pi ** (-2.0 / delta)
    g = inputs.phi(1, n)
    f = l1.l1_scale(delta, T, M) * np.outer(g, l1.l1_weights(delta, M)[1:])
    return T, f, g


@pytest.mark.parametrize("row", _table("table_it_1d.txt"), ids=lambda r: f"d{r[0]}-{int(r[1])}")
def test_table_1d_iterations(row):
    delta, grid, M, its, factor = row
    n, M = int(grid) - 1, int(M)
    T, f, _ = _paper_1d(delta, n, M)
    # FP64 rounding floor of the relative defect: eps |A_h| |u| / |r_0| with |u| <= 1 and
    # |r_0| = max |f| = c (delta = 0.1 on 2048^2: 1.7e-10, above the tolerance)
    floor = np.finfo(float).eps * 4.0 * (n + 1) ** 2 / np.abs(f).max()
    if floor > 5e-11:
        pytest.skip(f"FP64 defect floor {floor:.1e} is at the tolerance 1e-10")
    with G.Solver(1, n, M, T, delta) as s:
        s.set_order(G.MGWR_ORDER_TABLE)
        s.set_rhs(f)
        st = s.solve(1, 0, 1, tol=1e-10, max_cycles=40)
    assert abs(st.cycles - its) <= 1, (delta, grid, st.cycles, its)
    # the mean factor is no worse than the paper's (its delta = 1.0 entries, 0.05 for
    # 6 cycles, are not consistent with a 1e-10 reduction: 0.05^6 = 1.6e-8)
    assert st.factor <= factor + 0.025, (delta, grid, st.factor, factor)


@pytest.mark.parametrize("row", _table("table_it_2d.txt"), ids=lambda r: f"d{r[0]}-{int(r[1])}")
def test_table_2d_iterations(row):
    # the paper's problem on (0,2)^2 maps to (0,1)^2 by x -> x/2, t -> t 4^(-1/delta);
    # iteration counts and factors are invariant under that rescaling
    delta, grid, M, its, factor = row
    n, M = int(grid) - 1, int(M)
    T = 4.0 ** (-1.0 / delta)
    prob = inputs.Problem(2, n, M, T, delta, "t2")
    with G.Solver(2, n, M, T, delta) as s:
        s.set_rhs(prob.rhs())
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
    assert abs(st.cycles - its) <= 2, (delta, grid, st.cycles, its)
    assert abs(st.factor - factor) <= 0.04, (delta, grid, st.factor, factor)


def _w_factor(s, n, M, cycles=20, seed=0):
    L = s.num_levels() - 1
    u = inputs.random_field(n, M, seed=seed)
    s.field_set(G.MGWR_H64, L, G.MGWR_F, np.zeros_like(u))
    norms = []
    for _ in range(cycles):
        s.field_set(G.MGWR_H64, L, G.MGWR_U, u)
        s.cycle(G.MGWR_H64, 2, 1, 0)
        u = s.field_get(G.MGWR_H64, L, G.MGWR_U)
        nrm = np.abs(u).max()
        norms.append(nrm)
        u = u / nrm
    return float(np.exp(np.mean(np.log(norms[-4:]))))


@pytest.mark.parametrize("row", _table("sama_lambda_table.txt"), ids=lambda r: f"l{int(r[0])}-M{int(r[1])}")
def test_w_cycle_factors(row):
    # Table lambdas_m, bracketed rows: W(1,0), delta = 0.4, 256 x M grid, lambda =
    # tau^delta Gamma(2-delta) / h^2; same acceptance as the oracle's harness (settled
    # factors within 12 %, the slowly drifting small-lambda rows bracketed)
    log2lam, M, rho_h = row
    delta, n = 0.4, 255
    M = int(M)
    h = 1.0 / (n + 1)
    tau = (2.0 ** log2lam * h * h / math.gamma(2 - delta)) ** (1 / delta)
    with G.Solver(1, n, M, M * tau, delta) as s:
        rho = _w_factor(s, n, M)
    if log2lam >= -2:
        assert abs(rho - rho_h) <= 0.12 * rho_h + 0.003, (log2lam, M, rho, rho_h)
    else:
        assert rho_h * 0.8 <= rho <= 2.5 * rho_h, (log2lam, M, rho, rho_h)


@pytest.mark.parametrize("alpha", [0.4, 0.7])
def test_mittag_leffler_solution_error_falls_as_tau_to_alpha(alpha):
    # first experiment of Sec. 7 on (0,1): u = E_alpha(-pi^2 t^alpha) sin(pi x) with
    # T = pi^(-2/alpha); 4095 points (h^2 negligible) and M up to 8192 (partitioned
    # lines).  The GPU solution matches the oracle's discrete solution, and its error
    # against the continuous one falls at the L1 order alpha.
    n = 4095
    errs = []
    for M in (1024, 2048, 4096, 8192):
        T, f, g = _paper_1d(alpha, n, M)
        with G.Solver(1, n, M, T, alpha) as s:
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40, allow_noconv=True)
            u = s.solution()
        assert st.relres <= 1e-9
        t = T * np.arange(1, M + 1) / M
        F = l1.l1_scale(alpha, T, M) * l1.l1_weights(alpha, M)[1:]
        w_disc = separable.time_factor(1, n, M, T, alpha, F)
        ref = np.outer(g, w_disc)
        assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()
        exact = np.outer(g, mittag_leffler(alpha, -math.pi ** 2 * t ** alpha))
        errs.append(np.abs(u - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(0.85 * alpha <= r <= 1.02 * alpha for r in rates), rates
