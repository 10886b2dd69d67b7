"""The allocation-free H|psi> entry point (qe_hpsi_noalloc) against qe_hpsi.

qe_hpsi_noalloc serves callers that cannot allocate device memory: it takes
its workspace from a fixed array inside the library instead of the context's
buffers.  Called in a row through the C ABI (two different cells, so the
second call re-plans into the array the first one left behind, then the same
cell again, whose plan the array already holds), each result must equal the
regular entry point's within the parity tolerance of the other tests (per band
1e-12 relative in FP64, 2e-5 with QE_MIXED).  A problem too large for the array must
be refused with QE_EINVAL before any work is queued.

This file is collected last so that a failure here cannot stop the others.
"""
import numpy as np
import pytest

import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(q, ctx, name, nb, seed):
    c = qeinputs.config(name)
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
    psi = qeinputs.random_vectors(nb, npw, seed=seed)
    pt = torch.from_numpy(psi.view(np.float64).reshape(nb, npw, 2).copy()).to(dev)
    prob = ctx.problem(lat, k, ecut, grid, v, beta, d, nb)
    return prob, pt, (v, beta, d)


def _rel(a, b):
    a = a[..., 0] + 1j * a[..., 1]
    b = b[..., 0] + 1j * b[..., 1]
    return float((np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_noalloc_matches_hpsi_on_two_calls_in_a_row(prec, tol):
    import paper_2104_10502_gb300 as q
    precision = q.QE_FP64 if prec == "fp64" else q.QE_MIXED
    torch.cuda.set_device(0)
    with q.Context(0) as ctx:
        cases = [_setup(q, ctx, "C0", 8, 21), _setup(q, ctx, "SMALL", 5, 22)]
        refs = []
        for prob, pt, keep in cases:
            ht = torch.empty_like(pt)
            ctx.hpsi(prob, pt, ht, precision)
            refs.append(ht)
        # two calls in a row on different cells (the second replaces the plan the
        # first left in the array), then the second cell again (its plan is
        # already there) and the first again
        order = [0, 1, 1, 0]
        outs = []
        for i in order:
            prob, pt, keep = cases[i]
            out = torch.full_like(pt, float("nan"))
            q.hpsi_noalloc(prob, pt, out, precision)
            outs.append(out)
        torch.cuda.synchronize()
        for i, out in zip(order, outs):
            assert _rel(out.cpu().numpy(), refs[i].cpu().numpy()) <= tol


def test_noalloc_refuses_problems_beyond_its_array():
    import paper_2104_10502_gb300 as q
    torch.cuda.set_device(0)
    lat = qeinputs.cubic(40.0)
    grid = (192, 192, 192)                    # the permuted potential alone is 56 MiB
    _, kin = q.gsphere(lat, np.zeros(3), 40.0, grid)
    v = torch.zeros((192, 192, 192), dtype=torch.float64, device="cuda")
    with q.Context(0) as ctx:
        prob = ctx.problem(lat, np.zeros(3), 40.0, grid, v, None, None, 1)
    pt = torch.zeros((1, len(kin), 2), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QEError) as e:
        q.hpsi_noalloc(prob, pt, torch.empty_like(pt), q.QE_FP64)
    assert e.value.code == q.QE_EINVAL
    assert "64" in str(e.value) or "holds" in str(e.value)


def test_noalloc_refuses_calls_under_stream_capture():
    import paper_2104_10502_gb300 as q
    torch.cuda.set_device(0)
    with q.Context(0) as ctx:
        prob, pt, keep = _setup(q, ctx, "C0", 2, 23)
        out = torch.empty_like(pt)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        caught = []
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                try:
                    q.hpsi_noalloc(prob, pt, out, q.QE_FP64, stream=s.cuda_stream)
                except q.QEError as e:      # refused before queueing anything
                    caught.append(e)
        torch.cuda.synchronize()
        assert caught and caught[0].code == q.QE_EINVAL
        assert "captur" in str(caught[0])
        # the stream is usable again afterwards
        q.hpsi_noalloc(prob, pt, out, q.QE_FP64)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
