"""The device-side solve loop (mgwr_set_device_loop): an MGWR_FP64 solve's
iterations after the first run as one graph launch, a WHILE node whose body is
one iteration and a kernel that decides on the device whether another follows.
It must give the host loop's solve bitwise (the same launches in the same
order, the same stopping decision), also when max_cycles ends it, and it must
actually run (one deciding kernel per device iteration, one initialising
launch)."""
import numpy as np
import pytest

from oracle import direct
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _solve(d, n, M, cyc, nu1, nu2, tol, max_cycles, device_loop, batch=1):
    alphas = 0.6 if batch == 1 else list(np.linspace(0.2, 0.8, batch))
    with G.Solver(d, n, M, 1.0, alphas) as s:
        s.set_device_loop(device_loop)
        if batch == 1:
            f = inputs.Problem(d, n, M, 1.0, 0.6, "talpha").rhs()
        else:
            f = np.stack([inputs.Problem(d, n, M, 1.0, a, "t2").rhs() for a in alphas])
        s.set_rhs(f)
        s.solve(cyc, nu1, nu2, tol=1e-3, max_cycles=3, allow_noconv=True)  # graphs captured
        s.set_rhs(f)
        before = G.launch_count()
        st = s.solve(cyc, nu1, nu2, tol=tol, max_cycles=max_cycles, allow_noconv=True)
        launches = G.launch_count() - before
        return s.solution(), st, launches, f


@pytest.mark.parametrize("d,n,M,cyc,nu1,nu2,batch", [
    (1, 63, 64, 1, 1, 1, 1),      # the C1 shape
    (2, 31, 256, 1, 1, 1, 1),
    (2, 31, 128, 1, 0, 1, 1),
    (2, 15, 64, 2, 1, 1, 1),      # W cycle
    (2, 31, 128, 1, 1, 0, 1),     # ends with the interpolation: full defects
    (2, 15, 128, 1, 1, 1, 3),     # batch of three
])
def test_device_loop_is_bitwise_the_host_loop(d, n, M, cyc, nu1, nu2, batch):
    u_h, st_h, l_h, f = _solve(d, n, M, cyc, nu1, nu2, 1e-10, 60, False, batch)
    u_d, st_d, l_d, _ = _solve(d, n, M, cyc, nu1, nu2, 1e-10, 60, True, batch)
    np.testing.assert_array_equal(u_d, u_h)
    assert (st_d.cycles, st_d.outer, st_d.relres, st_d.status) == \
        (st_h.cycles, st_h.outer, st_h.relres, st_h.status)
    assert st_d.status == G.MGWR_OK and st_d.cycles >= 3
    # the loop ran: the host loop's launches, one deciding kernel per device
    # iteration (all but the first) and one initialising launch
    assert l_d == l_h + (st_d.cycles - 1) + 1
    if batch == 1:
        ref = direct.time_stepping(d, n, M, 1.0, 0.6, f)
        assert np.abs(u_d - ref).max() <= 1e-9 * np.abs(ref).max()


def test_device_loop_stops_at_max_cycles_like_the_host_loop():
    u_h, st_h, _, _ = _solve(2, 31, 256, 1, 1, 1, 1e-14, 4, False)
    u_d, st_d, _, _ = _solve(2, 31, 256, 1, 1, 1, 1e-14, 4, True)
    assert st_h.status == st_d.status == G.MGWR_E_NOCONV
    assert (st_d.cycles, st_d.relres) == (st_h.cycles, st_h.relres) == (4, st_h.relres)
    np.testing.assert_array_equal(u_d, u_h)


@pytest.mark.parametrize("nu1,nu2", [(0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("device_loop", [False, True])
def test_second_solve_on_a_handle_replays_the_right_iterations(nu1, nu2, device_loop):
    # A replayed iteration graph sets the defect states its capture left, so the
    # second solve on a handle (its first iteration replayed from u = 0, the
    # others after it) runs the launches of a solve without graphs.  With nu1 = 0
    # the first iteration restricts f itself and the later ones the defect: a
    # replay that kept the start's state would repeat the first form.
    d, n, M = 2, 31, 128
    f = inputs.Problem(d, n, M, 1.0, 0.6, "talpha").rhs()
    with G.Solver(d, n, M, 1.0, 0.6) as ref:
        ref.set_graphs(False)
        ref.set_rhs(f)
        st0 = ref.solve(1, nu1, nu2, tol=1e-10, max_cycles=60)
        u0 = ref.solution()
    with G.Solver(d, n, M, 1.0, 0.6) as s:
        s.set_device_loop(device_loop)
        for _ in range(3):
            s.set_rhs(f)
            st = s.solve(1, nu1, nu2, tol=1e-10, max_cycles=60)
            np.testing.assert_array_equal(s.solution(), u0)
            assert (st.cycles, st.relres) == (st0.cycles, st0.relres)
