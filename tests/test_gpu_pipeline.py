"""Pipelined transfers (mgwr_stage_rhs / mgwr_take_rhs / mgwr_stage_solution /
mgwr_wait_staged): a stream of problems through one handle, each right-hand
side staged while the previous solve runs and each solution returned while the
next one runs, must give every solve's result bitwise as the synchronous calls
(mgwr_set_rhs, mgwr_get_solution) do, and the calls must keep their order."""
import numpy as np
import pytest
import torch

from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def _pinned(shape):
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M", [(2, 31, 256), (1, 127, 64)])
def test_pipelined_stream_of_solves_is_bitwise_the_synchronous_one(precision, d, n, M):
    fs = [inputs.Problem(d, n, M, 1.0, 0.5, kind).rhs() for kind in ("t2", "talpha", "t2")]
    fs[2] = 0.5 * fs[2] + fs[1]
    ref = []
    with G.Solver(d, n, M, 1.0, 0.5) as s:
        s.set_precision(precision)
        for f in fs:
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-9, max_cycles=60)
            ref.append((s.solution(), st.cycles, st.relres))
    pin_f = [_pinned(f.shape) for f in fs]
    for p, f in zip(pin_f, fs):
        p[...] = f
    pin_u = [_pinned(fs[0].shape) for _ in fs]
    with G.Solver(d, n, M, 1.0, 0.5) as s:
        s.set_precision(precision)
        s.stage_rhs(pin_f[0])
        got = []
        for k in range(len(fs)):
            s.take_rhs()
            if k + 1 < len(fs):
                s.stage_rhs(pin_f[k + 1])
            st = s.solve(1, 1, 1, tol=1e-9, max_cycles=60)
            got.append((st.cycles, st.relres))
            s.stage_solution(pin_u[k])
        s.wait_staged()
    for (u0, c0, r0), u, (c, r) in zip(ref, pin_u, got):
        np.testing.assert_array_equal(u, u0)
        assert (c, r) == (c0, r0)


def test_pipelined_calls_check_their_order():
    with G.Solver(1, 31, 64, 1.0, 0.5) as s:
        f = _pinned((31, 64))
        f[...] = inputs.Problem(1, 31, 64, 1.0, 0.5, "t2").rhs()
        with pytest.raises(G.MGWRError):
            s.take_rhs()  # nothing staged
        s.stage_rhs(f)
        with pytest.raises(G.MGWRError):
            s.stage_rhs(f)  # the first one not taken yet
        s.take_rhs()
        s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u = _pinned((31, 64))
        s.stage_solution(u)
        s.wait_staged()
        np.testing.assert_array_equal(u, s.solution())
