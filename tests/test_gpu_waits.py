"""Bounded device waits: a grid-wide barrier that runs out ends its kernel with
an error status that the host reads (QE_ETIMEOUT), and the context stays
usable.

The test hook qe_test_grid_wait makes every grid barrier of the cooperative
dense-eigensolver kernels wait for one arrival more than its grid supplies (a
count that nothing reaches), with a 20 ms limit; each waiting CTA gives up,
sets the shared error word and returns.  No tensor-core or TMA kernel is
involved (the barriers are plain spin waits with nothing in flight).  A
Davidson solve with more than 64 bands runs the multi-CTA tridiagonalisation
in its first Rayleigh-Ritz, so its first barrier runs out; the solve must
return QE_ETIMEOUT, and the next solve on the same context, with the hook off,
must converge to the stored dense eigenvalues.
"""
import os

import numpy as np
import pytest

import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _problem(q, ctx, nb, seed):
    c = qeinputs.config("C0")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    dev = torch.device("cuda", 0)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    nproj = 4 * len(c["widths"]) * len(c["tau"])
    beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
    ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
    d = torch.from_numpy(qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))).to(dev)
    psi0 = qeinputs.start_bands(kin, nb, seed)
    pt = torch.from_numpy(psi0.view(np.float64).reshape(nb, npw, 2).copy()).to(dev)
    return ctx.problem(lat, k, ecut, grid, v, beta, d, nb), pt, (v, beta, d)


def test_grid_barrier_time_out_returns_status_and_context_survives():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        prob, pt, keep = _problem(q, ctx, 72, 0)
        ev = torch.zeros(72, dtype=torch.float64, device="cuda")
        ctx.test_grid_wait(20_000_000)                 # 20 ms, and a barrier nobody completes
        with pytest.raises(q.QEError) as e:
            ctx.davidson(prob, pt, ev, None, precision=q.QE_FP64 | q.QE_NO_GAMMA, tol=1e-8,
                         max_iter=3)
        assert e.value.code == q.QE_ETIMEOUT
        assert "barrier" in str(e.value)
        ctx.test_grid_wait(0)
        # the same context afterwards: a normal solve converges to the reference
        prob, pt, keep = _problem(q, ctx, 8, 0)
        ev = torch.zeros(8, dtype=torch.float64, device="cuda")
        rc, it = ctx.davidson(prob, pt, ev, None, precision=q.QE_FP64, tol=1e-8)
        torch.cuda.synchronize()
        assert rc == q.QE_OK
        ref = np.loadtxt(os.path.join(GOLDEN, "c0_dense_eigs.txt"))[:8]
        assert np.abs(ev.cpu().numpy() - ref).max() <= 1e-10
