"""Serving on the GPU: a request's result is the same alone and in a mix of
concurrent requests of other cells, cut-offs and band counts (bitwise: kernels
are deterministic and every slot owns its buffers), and each result still
matches the oracle's reference eigenvalues (1e-10 Ry FP64, 1e-6 Ry mixed)."""
import os

import numpy as np
import pytest

import oracle
import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _host_request(q, ctx, name, nb=None, seed=None, **over):
    c = dict(qeinputs.config(name))
    c.update(over)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    nb = c["nbnd"] if nb is None else nb
    _, kin = q.gsphere(lat, k, ecut, grid)
    v = np.zeros((grid[2], grid[1], grid[0]))
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    nproj = 4 * len(c["widths"]) * len(c["tau"])
    beta = np.zeros((nproj, len(kin), 2))
    ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    prob = q.problem(lat, k, ecut, grid, v, beta, d, nb)
    psi0 = qeinputs.start_bands(kin, nb, c["psi_seed"] if seed is None else seed)
    return prob, psi0, (v, beta, d)


def test_result_alone_equals_result_in_the_mix():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        a = _host_request(q, ctx, "C0")
        others = [
            _host_request(q, ctx, "SMALL"),
            _host_request(q, ctx, "C0", seed=5, nb=12),
            _host_request(q, ctx, "SMALL", nb=3, seed=9),
            _host_request(q, ctx, "C0", nb=6, seed=2, ecut=15.0),
        ]
    with q.Server(budget_bytes=16 << 30, max_slots=1) as s:
        alone = s.poll(s.submit(a[0], a[1], tol=1e-8))
    assert alone["status"] == q.QE_OK
    ref = np.loadtxt(os.path.join(GOLDEN, "c0_dense_eigs.txt"))[:8]
    assert np.abs(alone["evals"] - ref).max() <= 1e-10
    with q.Server(budget_bytes=16 << 30, max_slots=4) as s:
        t_other = [s.submit(p, x, tol=1e-8) for p, x, _ in others[:2]]
        t_a = s.submit(a[0], a[1], tol=1e-8)
        t_mix = s.submit(others[0][0], others[0][1], precision=q.QE_MIXED, tol=1e-5)
        t_other += [s.submit(p, x, tol=1e-8) for p, x, _ in others[2:]]
        mixed = s.poll(t_a)
        rest = [s.poll(t) for t in t_other]
        rmix = s.poll(t_mix)
    assert mixed["status"] == q.QE_OK
    assert np.array_equal(mixed["evals"], alone["evals"])
    assert np.array_equal(mixed["psi"], alone["psi"])
    assert all(r["status"] == q.QE_OK for r in rest)
    small_ref = np.loadtxt(os.path.join(GOLDEN, "small_dense_eigs.txt"))
    assert np.abs(rest[0]["evals"] - small_ref[:7]).max() <= 1e-10
    assert np.abs(rest[2]["evals"] - small_ref[:3]).max() <= 1e-10
    assert rmix["status"] == q.QE_OK
    assert np.abs(rmix["evals"] - small_ref[:7]).max() <= 1e-6
    assert mixed["latency_s"] > 0 and alone["latency_s"] > 0


def _footprint(q, prob, psi0):
    """Smallest budget that accepts the request (host-only fake-solver servers)."""
    lo, hi = 1, 1 << 36
    while hi - lo > 1:
        mid = (lo + hi) // 2
        try:
            with q.Server(budget_bytes=mid, max_slots=1, fake=True) as s:
                s.poll(s.submit(prob, psi0, max_iter=0))
            hi = mid
        except q.QEError:
            lo = mid
    return hi


def test_budget_is_respected_on_the_gpu():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        reqs = [_host_request(q, ctx, "C0", seed=s) for s in range(6)]
    need = _footprint(q, reqs[0][0], reqs[0][1])
    budget = 2 * need + need // 2                      # room for two at a time
    with q.Server(budget_bytes=budget, max_slots=6) as s:
        ts = [s.submit(p, x, tol=1e-8) for p, x, _ in reqs]
        peak, peak_running = 0, 0
        while True:
            st = s.stats()
            peak = max(peak, st["bytes_in_use"])
            peak_running = max(peak_running, st["running"])
            if st["completed"] >= len(ts):
                break
        res = [s.poll(t) for t in ts]
    assert all(r["status"] == q.QE_OK for r in res)
    assert 0 < peak <= budget and 1 <= peak_running <= 2
    # different start bands, same operator: the same eigenvalues whatever the admission order
    for r in res[1:]:
        assert np.abs(r["evals"] - res[0]["evals"]).max() <= 1e-10
