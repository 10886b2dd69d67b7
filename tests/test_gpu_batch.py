"""Batched H|psi> (one persistent launch per FFT stage over many problems),
its CUDA-graph replay, and the FFT launch-shape autotuner.

Problems of different cells, k points, grids, plane-wave and band counts go
through one batch; every problem's result must equal qe_hpsi on that problem
alone bit for bit (the tiles are the same code; only their scheduling differs),
and the FP64 results must match the oracle within 1e-12 per band.  The k-point
workload follows the paper's pools (Sec. 3.3): k points of one cell as
independent problems.
"""
import numpy as np
import pytest

import oracle
import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prob(q, ctx, lat, k, ecut, grid, tau, widths, nb, seed):
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    dev = torch.device("cuda", 0)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    ctx.vloc_gaussian(lat, grid, tau, v)
    nproj = 4 * len(widths) * len(tau)
    beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
    ctx.beta_gaussian(lat, k, ecut, tau, widths, beta)
    d = torch.from_numpy(qeinputs.d_matrix(len(tau), len(widths))).to(dev)
    psi = qeinputs.random_vectors(nb, npw, seed=seed)
    pt = torch.from_numpy(psi.view(np.float64).reshape(nb, npw, 2).copy()).to(dev)
    prob = ctx.problem(lat, k, ecut, grid, v, beta, d, nb)
    return dict(prob=prob, psi=pt, keep=(v, beta, d), host=psi,
                args=(lat, k, ecut, grid, tau, widths))


def _mix(q, ctx):
    c0 = qeinputs.config("C0")
    sm = qeinputs.config("SMALL")
    t = qeinputs.config("C3T")
    b = oracle.reciprocal(t["lat"])
    out = [
        _prob(q, ctx, c0["lat"], c0["k"], c0["ecut"], c0["grid"], c0["tau"], c0["widths"], 8, 1),
        _prob(q, ctx, sm["lat"], sm["k"], sm["ecut"], sm["grid"], sm["tau"], sm["widths"], 7, 2),
        _prob(q, ctx, t["lat"], 0.25 * b[0] + 0.5 * b[1], t["ecut"], t["grid"], t["tau"], t["widths"], 12, 3),
        _prob(q, ctx, qeinputs.cubic(8.0), np.zeros(3), 18.0, (27, 27, 27),
              np.array([[1.0, 1.0, 1.0], [5.0, 4.0, 3.0]]), (1.0,), 5, 4),
        _prob(q, ctx, c0["lat"], c0["k"], 15.0, (30, 30, 30), c0["tau"], c0["widths"], 0, 5),
    ]
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_single_problem_calls(prec):
    import paper_2104_10502_gb300 as q
    precision = q.QE_FP64 if prec == "fp64" else q.QE_MIXED
    with q.Context(0) as ctx:
        items = _mix(q, ctx)
        singles = []
        for it in items:
            h = torch.empty_like(it["psi"])
            if it["prob"].nbnd:
                ctx.hpsi(it["prob"], it["psi"], h, precision)
            singles.append(h)
        outs = [torch.full_like(it["psi"], float("nan")) for it in items]
        ctx.hpsi_batch([it["prob"] for it in items], [it["psi"] for it in items], outs, precision)
        torch.cuda.synchronize()
        for it, s, o in zip(items, singles, outs):
            if it["prob"].nbnd:
                assert torch.equal(s, o)


def test_batch_fp64_matches_oracle():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        items = _mix(q, ctx)[:4]
        outs = [torch.empty_like(it["psi"]) for it in items]
        ctx.hpsi_batch([it["prob"] for it in items], [it["psi"] for it in items], outs, q.QE_FP64)
        torch.cuda.synchronize()
        for it, o in zip(items, outs):
            lat, k, ecut, grid, tau, widths = it["args"]
            v = oracle.vloc_gaussian(lat, grid, tau)
            beta = oracle.beta_gaussian(lat, k, ecut, tau, widths)
            d = qeinputs.d_matrix(len(tau), len(widths))
            want = oracle.hpsi(lat, k, ecut, grid, v, beta, d, it["host"])
            got = o.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            rel = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
            assert rel.max() <= 1e-12


def test_graph_replay_equals_eager_batch():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        items = _mix(q, ctx)[:4]
        probs = [it["prob"] for it in items]
        psis = [it["psi"] for it in items]
        eager = [torch.empty_like(p) for p in psis]
        ctx.hpsi_batch(probs, psis, eager, q.QE_FP64)
        outs = [torch.full_like(p, float("nan")) for p in psis]
        g = ctx.batch_create(probs, psis, outs, q.QE_FP64)
        for _ in range(2):
            for o in outs:
                o.fill_(float("nan"))
            g.run()
            torch.cuda.synchronize()
            assert all(torch.equal(a, b) for a, b in zip(eager, outs))
        # new contents, same addresses: the replay follows the data
        for p in psis:
            p.mul_(0.5)
        g.run()
        ctx.hpsi_batch(probs, psis, eager, q.QE_FP64)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(eager, outs))
        g.close()


def test_autotune_keeps_results_bit_identical():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        it = _mix(q, ctx)[0]
        before = torch.empty_like(it["psi"])
        ctx.hpsi(it["prob"], it["psi"], before, q.QE_FP64)
        ctx.autotune(it["prob"], q.QE_FP64)
        ctx.autotune(it["prob"], q.QE_MIXED)
        after = torch.empty_like(it["psi"])
        ctx.hpsi(it["prob"], it["psi"], after, q.QE_FP64)
        torch.cuda.synchronize()
        assert torch.equal(before, after)


def test_batch_rejects_host_arrays():
    import paper_2104_10502_gb300 as q
    c = qeinputs.config("SMALL")
    _, kin = q.gsphere(c["lat"], c["k"], c["ecut"], c["grid"])
    v = np.zeros((c["grid"][2], c["grid"][1], c["grid"][0]))
    with q.Context(0) as ctx:
        prob = ctx.problem(c["lat"], c["k"], c["ecut"], c["grid"], v, None, None, 1)
        psi = np.zeros((1, len(kin)), dtype=complex)
        with pytest.raises((q.QEError, ValueError)):
            ctx.hpsi_batch([prob], [psi], [psi.copy()], q.QE_FP64)


def _dv_items(q, ctx):
    """Davidson problems of different cells, k points, grids and band counts."""
    c0 = qeinputs.config("C0")
    sm = qeinputs.config("SMALL")
    t = qeinputs.config("C3T")
    b = oracle.reciprocal(t["lat"])
    specs = [
        (c0["lat"], c0["k"], c0["ecut"], c0["grid"], c0["tau"], c0["widths"], c0["nbnd"]),
        (sm["lat"], sm["k"], sm["ecut"], sm["grid"], sm["tau"], sm["widths"], sm["nbnd"]),
        (t["lat"], 0.25 * b[0] + 0.5 * b[1], t["ecut"], t["grid"], t["tau"], t["widths"], 12),
        (c0["lat"], c0["k"], 15.0, (30, 30, 30), c0["tau"], c0["widths"], 0),
        (t["lat"], np.zeros(3), t["ecut"], t["grid"], t["tau"], t["widths"], 10),
    ]
    items = []
    for lat, k, ecut, grid, tau, widths, nb in specs:
        it = _prob(q, ctx, lat, k, ecut, grid, tau, widths, nb, 0)
        _, kin = q.gsphere(lat, k, ecut, grid)
        psi0 = qeinputs.start_bands(kin, nb, 7)
        it["psi"] = torch.from_numpy(psi0.view(np.float64).reshape(nb, len(kin), 2).copy()).to(0)
        items.append(it)
    return items


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_davidson_batch_equals_single_solves(prec):
    """Lockstep batch: every solve's eigenvalues, vectors and iteration count
    equal qe_davidson on that problem alone, bit for bit."""
    import paper_2104_10502_gb300 as q
    precision = q.QE_FP64 if prec == "fp64" else q.QE_MIXED
    tol = 1e-8 if prec == "fp64" else 1e-5
    with q.Context(0) as ctx:
        items = _dv_items(q, ctx)
        single = []
        for it in items:
            nb = it["prob"].nbnd
            psi = it["psi"].clone()
            ev = torch.zeros(nb, dtype=torch.float64, device="cuda")
            if nb:
                rc, its = ctx.davidson(it["prob"], psi, ev, None, precision=precision, tol=tol)
                assert rc == q.QE_OK
            else:
                its = 0
            single.append((psi, ev, its))
        psis = [it["psi"].clone() for it in items]
        evs = [torch.full((it["prob"].nbnd,), float("nan"), dtype=torch.float64, device="cuda")
               for it in items]
        rss = [torch.zeros_like(e) for e in evs]
        rc, sts, its = ctx.davidson_batch([it["prob"] for it in items], psis, evs, rss,
                                          precision=precision, tol=tol)
        torch.cuda.synchronize()
        assert rc == q.QE_OK and all(s == q.QE_OK for s in sts)
        for (psi, ev, it1), p, e, r, it2 in zip(single, psis, evs, rss, its):
            assert it1 == it2
            assert torch.equal(ev, e) and torch.equal(psi, p)
            if len(r):
                assert r.max().item() <= tol


def test_davidson_batch_against_dense_references():
    """The C0 and SMALL members of a batch against the oracle's dense
    diagonalisation (1e-10 Ry)."""
    import os
    import paper_2104_10502_gb300 as q
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with q.Context(0) as ctx:
        items = _dv_items(q, ctx)[:2]
        evs = [torch.zeros(it["prob"].nbnd, dtype=torch.float64, device="cuda") for it in items]
        rc, sts, its = ctx.davidson_batch([it["prob"] for it in items], [it["psi"] for it in items],
                                          evs, tol=1e-8)
        assert rc == q.QE_OK
        for name, it, e in zip(("c0_dense_eigs.txt", "small_dense_eigs.txt"), items, evs):
            ref = np.loadtxt(os.path.join(golden, name))[:it["prob"].nbnd]
            assert np.abs(e.cpu().numpy() - ref).max() <= 1e-10


def test_davidson_batch_reports_nonconvergence_per_problem():
    import paper_2104_10502_gb300 as q
    with q.Context(0) as ctx:
        items = _dv_items(q, ctx)[:3]
        evs = [torch.zeros(it["prob"].nbnd, dtype=torch.float64, device="cuda") for it in items]
        rc, sts, its = ctx.davidson_batch([it["prob"] for it in items], [it["psi"] for it in items],
                                          evs, tol=1e-12, max_iter=1)
        assert rc == q.QE_ENOCONV
        assert sts == [q.QE_ENOCONV] * 3 and its == [1, 1, 1]
        assert all(torch.isfinite(e).all() for e in evs)


def test_c3_cubes_batched_davidson_against_oracle():
    """The 32 cubic cells of the batched workload (grids 15^3..27^3, 16..96
    bands) solved as one lockstep batch; the cells small enough for the
    oracle's dense diagonalisation (a <= 9 bohr) within 1e-10 Ry."""
    import paper_2104_10502_gb300 as q
    specs = qeinputs.c3_problems()[16:]
    with q.Context(0) as ctx:
        items = [_prob(q, ctx, p["lat"], p["k"], p["ecut"], p["grid"], p["tau"], p["widths"],
                       p["nbnd"], 0) for p in specs]
        for it, p in zip(items, specs):
            _, kin = q.gsphere(p["lat"], p["k"], p["ecut"], p["grid"])
            psi0 = qeinputs.start_bands(kin, p["nbnd"], p["psi_seed"])
            it["psi"] = torch.from_numpy(psi0.view(np.float64).reshape(p["nbnd"], len(kin), 2).copy()).to(0)
        evs = [torch.zeros(p["nbnd"], dtype=torch.float64, device="cuda") for p in specs]
        rc, sts, its = ctx.davidson_batch([it["prob"] for it in items], [it["psi"] for it in items],
                                          evs, tol=1e-8, max_iter=300)
        assert rc == q.QE_OK, (sts, its)
        checked = 0
        for p, e in zip(specs, evs):
            if p["lat"][0, 0] > 9.0:
                continue
            v = oracle.vloc_gaussian(p["lat"], p["grid"], p["tau"])
            beta = oracle.beta_gaussian(p["lat"], p["k"], p["ecut"], p["tau"], p["widths"])
            d = qeinputs.d_matrix(len(p["tau"]), len(p["widths"]))
            h = oracle.dense_h(p["lat"], p["k"], p["ecut"], p["grid"], v, beta, d)
            ref = np.linalg.eigvalsh(h)[:p["nbnd"]]
            assert np.abs(e.cpu().numpy() - ref).max() <= 1e-10
            checked += 1
        assert checked >= 4
