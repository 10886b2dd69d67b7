"""Serving host logic without a GPU (QE_SERVE_FAKE_SOLVER: a solve sleeps
max_iter ms): admission in arrival order under a device-memory budget and a
slot limit, continuous admission as requests finish, queue-full back-pressure,
poll timeouts, cancellation and shutdown.  The paper's outlook (Sec. 4) and the
over-subscription note of Sec. 3.3 motivate serving many independent solves on
one GPU; failures are made on the host here, never on a GPU."""
import time

import numpy as np
import pytest

import qeinputs


@pytest.fixture(scope="module")
def q():
    from paper_2104_10502_gb300.build import build
    build()
    import paper_2104_10502_gb300 as q
    return q


def _req(q, nb=4):
    c = qeinputs.config("SMALL")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    _, kin = q.gsphere(lat, k, ecut, grid)
    v = np.zeros((grid[2], grid[1], grid[0]))
    prob = q.problem(lat, k, ecut, grid, v, None, None, nb)
    psi0 = qeinputs.start_bands(kin, nb, 0)
    return prob, psi0, v


def test_requests_complete_and_report_latency(q):
    prob, psi0, keep = _req(q)
    with q.Server(budget_bytes=1 << 34, max_slots=2, fake=True) as s:
        t = [s.submit(prob, psi0, max_iter=30) for _ in range(4)]
        res = [s.poll(x) for x in t]
        assert all(r["status"] == q.QE_OK for r in res)
        assert all(np.array_equal(r["psi"], psi0) for r in res)
        lat = sorted(r["latency_s"] for r in res)
        # two slots: the last two requests waited for a slot
        assert lat[0] >= 0.025 and lat[-1] >= 0.055
        st = s.stats()
        assert st["completed"] == 4 and st["running"] == 0 and st["queued"] == 0


def test_budget_limits_concurrency(q):
    prob, psi0, keep = _req(q)
    with q.Server(budget_bytes=1 << 34, max_slots=4, fake=True) as s0:
        t = s0.submit(prob, psi0, max_iter=1)
        s0.poll(t)
    # find the footprint of one request by binary search on the budget
    lo, hi = 1, 1 << 34
    while hi - lo > 1:
        mid = (lo + hi) // 2
        try:
            with q.Server(budget_bytes=mid, max_slots=4, fake=True) as s1:
                s1.poll(s1.submit(prob, psi0, max_iter=0))
            hi = mid
        except q.QEError:
            lo = mid
    need = hi
    # budget for exactly two concurrent requests, four slots
    with q.Server(budget_bytes=2 * need + need // 2, max_slots=4, fake=True) as s:
        t = [s.submit(prob, psi0, max_iter=60) for _ in range(4)]
        time.sleep(0.02)
        st = s.stats()
        assert st["running"] == 2 and st["queued"] == 2
        assert st["bytes_in_use"] <= 2 * need + need // 2
        for x in t:
            assert s.poll(x)["status"] == q.QE_OK
    with q.Server(budget_bytes=need - 1, max_slots=1, fake=True) as s:
        with pytest.raises(q.QEError) as e:
            s.submit(prob, psi0)
        assert e.value.code == q.QE_EINVAL


def test_queue_full_pending_and_cancel(q):
    prob, psi0, keep = _req(q)
    with q.Server(budget_bytes=1 << 34, max_slots=1, max_queue=2, fake=True) as s:
        a = s.submit(prob, psi0, max_iter=200)
        time.sleep(0.02)                    # a is running
        b = s.submit(prob, psi0, max_iter=5)
        c = s.submit(prob, psi0, max_iter=5)
        assert s.submit(prob, psi0, max_iter=5) is None      # QE_EAGAIN: queue full
        assert s.poll(b, timeout_ms=0) is None                # still queued
        assert s.poll(b, timeout_ms=10) is None
        s.cancel(b)
        assert s.poll(b)["status"] == q.QE_ECANCELED
        s.cancel(a)                                           # running: finishes, reports cancelled
        assert s.poll(a)["status"] == q.QE_ECANCELED
        r = s.poll(c)
        assert r["status"] == q.QE_OK
        with pytest.raises(q.QEError):
            s.poll(c)                                         # consumed ticket


def test_nonconvergence_status_passes_through(q):
    prob, psi0, keep = _req(q)
    with q.Server(budget_bytes=1 << 34, max_slots=1, fake=True) as s:
        t = s.submit(prob, psi0, tol=2.0, max_iter=1)         # the fake reports QE_ENOCONV for tol > 1
        assert s.poll(t)["status"] == q.QE_ENOCONV


def test_destroy_with_work_in_flight(q):
    prob, psi0, keep = _req(q)
    s = q.Server(budget_bytes=1 << 34, max_slots=1, fake=True)
    for _ in range(3):
        s.submit(prob, psi0, max_iter=50)
    time.sleep(0.01)
    t0 = time.time()
    s.close()                                                 # running one finishes, queued cancelled
    assert time.time() - t0 < 1.0


def test_invalid_submissions(q):
    prob, psi0, keep = _req(q)
    with q.Server(budget_bytes=1 << 34, max_slots=1, fake=True) as s:
        bad = q.problem(prob.lat, prob.k, prob.ecutwfc, (3, 3, 3), keep, None, None, 4)
        with pytest.raises(q.QEError):
            s.submit(bad, psi0)                               # grid smaller than the sphere
        with pytest.raises(q.QEError):
            s.submit(prob, psi0, tol=-1.0)
