"""Serving runtime (mgwr_submit / mgwr_poll): results of requests solved in a
mix, concurrently on several slots, are identical to the same requests solved
alone; admission respects the memory budget; polling and errors behave as
documented."""
import numpy as np
import pytest

from oracle import direct
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

REQUESTS = [  # d, n, M, alpha, kind, precision
    (1, 63, 64, 0.5, "t2", G.MGWR_FP64),
    (2, 31, 128, 0.3, "talpha", G.MGWR_MIXED),
    (1, 255, 256, 0.8, "t2", G.MGWR_MIXED),
    (2, 63, 64, 0.65, "t2", G.MGWR_FP64),
    (2, 15, 512, 0.2, "talpha", G.MGWR_MIXED),
    (1, 31, 1024, 0.45, "t2", G.MGWR_FP64),
    (2, 127, 128, 0.9, "t2", G.MGWR_MIXED_DD),
    (1, 7, 4096, 0.35, "talpha", G.MGWR_FP64),
    (2, 31, 1024, 0.55, "t2", G.MGWR_MIXED_DD),
    (2, 31, 256, 0.5, "t2", G.MGWR_DD),
    (1, 4095, 128, 0.3, "talpha", G.MGWR_AUTO),  # resolves to MGWR_DD (h = 1/4096)
    (1, 255, 128, 0.6, "t2", G.MGWR_AUTO),       # resolves to MGWR_MIXED_DD
]
# the relative defect a request can reach: about eps (4/h^2) |u| / |f| of the
# iterate's precision (FP64 or double-float); 1e-8 on h = 1/4096
TOL = {4095: 1e-8}


def _alone(d, n, M, a, f, precision, tol):
    with G.Solver(d, n, M, 1.0, a) as s:
        s.set_precision(precision)
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=tol, max_cycles=100)
        return s.solution(), st


def test_results_in_the_mix_equal_results_alone():
    fs = [inputs.Problem(d, n, M, 1.0, a, k).rhs() for d, n, M, a, k, _ in REQUESTS]
    with G.Server(hbm_budget=8 << 30, slots=4) as srv:
        tickets = [srv.submit(d, n, M, 1.0, a, f, precision=p, tol=TOL.get(n, 1e-10))
                   for (d, n, M, a, k, p), f in zip(REQUESTS, fs)]
        results = [srv.poll(t, timeout_us=120_000_000) for t in tickets]
        info = srv.info()
    assert info["completed"] == len(REQUESTS) and info["peak_bytes"] <= info["budget_bytes"]
    for (d, n, M, a, k, p), f, res in zip(REQUESTS, fs, results):
        assert res is not None and res.status == G.MGWR_OK
        assert res.latency_s >= res.queue_s >= 0.0
        u, st = _alone(d, n, M, a, f, p, TOL.get(n, 1e-10))
        np.testing.assert_array_equal(res.u, u)
        assert res.stats.cycles == st.cycles and res.stats.relres == st.relres


def test_zero_copy_submission_equals_copied_submission():
    # f written into page-locked buffers lent by the server and handed over
    # without a copy: the same results, bitwise, as mgwr_submit's copies; a
    # buffer can be given back unsubmitted, and an array the server did not
    # lend is refused
    reqs = REQUESTS[:6]
    fs = [inputs.Problem(d, n, M, 1.0, a, k).rhs() for d, n, M, a, k, _ in reqs]
    with G.Server(hbm_budget=8 << 30, slots=3) as srv:
        copied = [srv.submit(d, n, M, 1.0, a, f, precision=p, tol=1e-10)
                  for (d, n, M, a, k, p), f in zip(reqs, fs)]
        lent = []
        for (d, n, M, a, k, p), f in zip(reqs, fs):
            buf = srv.buffer(n ** d, M)
            inputs.Problem(d, n, M, 1.0, a, k).rhs(out=buf)
            lent.append(srv.submit_buffer(d, n, M, 1.0, a, buf, precision=p, tol=1e-10))
        spare = srv.buffer(31, 64)
        srv.release(spare)
        with pytest.raises(G.MGWRError):
            srv.release(spare)  # no longer lent
        foreign = np.zeros((31, 64))
        with pytest.raises(G.MGWRError):
            srv.submit_buffer(1, 31, 64, 1.0, 0.5, foreign, precision=G.MGWR_FP64)
        for a, b in zip(copied, lent):
            ra, rb = srv.poll(a, timeout_us=120_000_000), srv.poll(b, timeout_us=120_000_000)
            assert ra.status == rb.status == G.MGWR_OK
            np.testing.assert_array_equal(ra.u, rb.u)
            assert ra.stats.cycles == rb.stats.cycles and ra.stats.relres == rb.stats.relres
        info = srv.info()
    assert info["pinned_buffers"] >= 1 and info["prepare_s"] > 0.0


def test_served_result_matches_oracle():
    d, n, M, a = 2, 31, 64, 0.4
    f = inputs.Problem(d, n, M, 1.0, a, "t2").rhs()
    with G.Server(hbm_budget=1 << 30, slots=2) as srv:
        res = srv.poll(srv.submit(d, n, M, 1.0, a, f, precision=G.MGWR_MIXED, tol=1e-10),
                       timeout_us=60_000_000)
    ref = direct.time_stepping(d, n, M, 1.0, a, f)
    assert np.abs(res.u - ref).max() <= 1e-9 * np.abs(ref).max()


def test_admission_budget_and_refusal():
    fp = G.footprint(2, 63, 256, 1, G.MGWR_FP64)
    f = inputs.Problem(2, 63, 256, 1.0, 0.5, "t2").rhs()
    # room for one such request at a time: all complete, never two at once
    with G.Server(hbm_budget=int(1.5 * fp), slots=4) as srv:
        ts = [srv.submit(2, 63, 256, 1.0, 0.5, f, precision=G.MGWR_FP64) for _ in range(3)]
        for t in ts:
            assert srv.poll(t, timeout_us=60_000_000).status == G.MGWR_OK
        assert srv.info()["peak_bytes"] <= int(1.5 * fp)
    # larger than the whole budget: refused at submit
    with G.Server(hbm_budget=fp // 2, slots=2) as srv:
        with pytest.raises(G.MGWRError) as e:
            srv.submit(2, 63, 256, 1.0, 0.5, f)
        assert e.value.status == G.MGWR_E_TOOBIG


def test_poll_timeout_unknown_ticket_and_numeric_failure():
    f = inputs.Problem(2, 255, 1024, 1.0, 0.5, "t2").rhs()
    bad = inputs.Problem(1, 31, 64, 1.0, 0.5, "t2").rhs()
    bad[3, 5] = np.nan
    with G.Server(hbm_budget=8 << 30, slots=2) as srv:
        t = srv.submit(2, 255, 1024, 1.0, 0.5, f, precision=G.MGWR_FP64, tol=1e-10)
        assert srv.poll(t, timeout_us=0) is None          # still running: not ready
        assert srv.poll(t, timeout_us=120_000_000).status == G.MGWR_OK
        assert srv.lib.mgwr_poll(srv.h, 987654, 0, None, None) == G.MGWR_E_INVAL
        tb = srv.submit(1, 31, 64, 1.0, 0.5, bad, precision=G.MGWR_FP64)
        rb = srv.poll(tb, timeout_us=60_000_000)
        assert rb.status == G.MGWR_E_NUMERIC


@pytest.mark.parametrize("policy", [G.MGWR_POLICY_FIFO, G.MGWR_POLICY_SMALLEST])
def test_admission_policy_orders_queued_requests(policy):
    # one slot: a blocker runs while a large and then three small requests queue;
    # first in first out finishes the large one first, smallest first the small ones
    blocker = inputs.Problem(2, 127, 512, 1.0, 0.5, "t2").rhs()
    large = inputs.Problem(2, 255, 1024, 1.0, 0.5, "t2").rhs()
    small = inputs.Problem(1, 63, 64, 1.0, 0.5, "t2").rhs()
    with G.Server(hbm_budget=16 << 30, slots=1) as srv:
        srv.set_policy(policy)
        tb = srv.submit(2, 127, 512, 1.0, 0.5, blocker, precision=G.MGWR_FP64)
        tl = srv.submit(2, 255, 1024, 1.0, 0.5, large, precision=G.MGWR_FP64)
        ts = [srv.submit(1, 63, 64, 1.0, 0.5, small, precision=G.MGWR_FP64) for _ in range(3)]
        rb = srv.poll(tb, timeout_us=120_000_000, copy_solution=False)
        rl = srv.poll(tl, timeout_us=120_000_000, copy_solution=False)
        rs = [srv.poll(t, timeout_us=120_000_000, copy_solution=False) for t in ts]
    assert rb.status == rl.status == G.MGWR_OK and all(r.status == G.MGWR_OK for r in rs)
    if policy == G.MGWR_POLICY_SMALLEST:
        assert max(r.latency_s for r in rs) < rl.latency_s
    else:
        assert min(r.latency_s for r in rs) > rl.latency_s
    with pytest.raises(G.MGWRError):
        G.Server(hbm_budget=1 << 30, slots=1).set_policy(7)


def test_requests_in_flight_share_graph_launches_and_reuse_handles():
    # requests submitted together run in the server's group: one graph launch
    # advances several of them; a later request of a shape seen before is served
    # by the idle handle of that shape, set up again for its (T, alpha); every
    # result is bitwise the request solved alone
    reqs = [(1, 63, 64, 0.5, "t2", G.MGWR_FP64), (2, 31, 128, 0.3, "talpha", G.MGWR_MIXED),
            (2, 15, 256, 0.7, "t2", G.MGWR_MIXED_DD), (1, 255, 512, 0.45, "t2", G.MGWR_MIXED),
            (2, 63, 64, 0.9, "t2", G.MGWR_FP64), (1, 127, 256, 0.25, "talpha", G.MGWR_DD)]
    fs = [inputs.Problem(d, n, M, 1.0, a, k).rhs() for d, n, M, a, k, _ in reqs]
    with G.Server(hbm_budget=8 << 30, slots=6) as srv:
        tickets = [srv.submit(d, n, M, 1.0, a, f, precision=p, tol=1e-10)
                   for (d, n, M, a, k, p), f in zip(reqs, fs)]
        results = [srv.poll(t, timeout_us=120_000_000) for t in tickets]
        info = srv.info()
        # the same shapes again with other orders: idle handles set up in place
        again = [(d, n, M, min(a + 0.05, 0.95), k, p) for d, n, M, a, k, p in reqs]
        fs2 = [inputs.Problem(d, n, M, 1.0, a, k).rhs() for d, n, M, a, k, _ in again]
        results2 = []
        for (d, n, M, a, k, p), f in zip(again, fs2):
            t = srv.submit(d, n, M, 1.0, a, f, precision=p, tol=1e-10)
            results2.append(srv.poll(t, timeout_us=120_000_000))
        info2 = srv.info()
    assert info["max_group_members"] >= 2
    assert info["member_iterations"] > info["group_launches"]
    assert info2["reused_handles"] >= len(again)
    for rq, f, res in list(zip(reqs, fs, results)) + list(zip(again, fs2, results2)):
        d, n, M, a, k, p = rq
        assert res.status == G.MGWR_OK
        u, st = _alone(d, n, M, a, f, p, 1e-10)
        np.testing.assert_array_equal(res.u, u)
        assert res.stats.cycles == st.cycles and res.stats.relres == st.relres
