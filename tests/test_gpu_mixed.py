"""The mixed-precision path against the FP64 oracle at full size (Sec. 3.3:
the Hamiltonian's kinetic, local-potential and pseudopotential contributions,
here with FP32 FFTs and TF32x3 tensor-core projector products).

Every mixed result is compared band by band with the oracle's FP64 H|psi> on
the same seeded inputs, per band ||Hpsi_gpu - Hpsi_ref|| / ||Hpsi_ref|| <= 2e-5:

* the C1 workload (128 bands, 34 265 plane waves, 512 projectors), bands
  sampled in both chunks of the stick buffer (68 FP32 bands per chunk) and at
  both ends of the tensor-core tiles; the projections reduce over every
  split-K slice of the plane-wave axis for every band;
* the k = 0 band pairs (QE_GAMMA) on C1 with an odd band count (the last band
  alone in its FFT);
* a batched call over k points of the tetragonal cell and two cubic cells of
  the batched workload.

Davidson with the mixed path's two Rayleigh-Ritz arithmetics (FP64 by default,
FP32 with QE_RR_FP32) against the stored dense and C2 eigenvalues (1e-6 Ry).
"""
import os

import numpy as np
import pytest

import oracle
import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 2e-5


@pytest.fixture(scope="module")
def q():
    import paper_2104_10502_gb300 as q
    return q


@pytest.fixture(scope="module")
def ctx(q):
    c = q.Context(0)
    yield c
    c.close()


def _to_t(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.float64).reshape(x.shape + (2,))).cuda()


def _from_t(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _rel_band(got, want):
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _gpu_problem(q, ctx, lat, k, ecut, grid, tau, widths, nb):
    miller, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    dev = torch.device("cuda", 0)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    ctx.vloc_gaussian(lat, grid, tau, v)
    nproj = 4 * len(widths) * len(tau)
    beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
    ctx.beta_gaussian(lat, k, ecut, tau, widths, beta)
    d = torch.from_numpy(qeinputs.d_matrix(len(tau), len(widths))).to(dev)
    return ctx.problem(lat, k, ecut, grid, v, beta, d, nb), (v, beta, d), np.asarray(miller), kin


def _oracle_h(lat, k, ecut, grid, tau, widths, psi):
    v = oracle.vloc_gaussian(lat, grid, tau)
    beta = oracle.beta_gaussian(lat, k, ecut, tau, widths)
    d = qeinputs.d_matrix(len(tau), len(widths))
    return oracle.hpsi(lat, k, ecut, grid, v, beta, d, psi)


def _mirror(miller):
    key = {tuple(m): i for i, m in enumerate(miller)}
    return np.array([key[tuple(-m)] for m in miller])


def test_hpsi_mixed_c1_sampled(q, ctx):
    c = qeinputs.config("C1")
    args = (c["lat"], c["k"], c["ecut"], c["grid"], c["tau"], c["widths"])
    nb = c["nbnd"]
    prob, keep, miller, kin = _gpu_problem(q, ctx, *args, nb)
    psi = qeinputs.start_bands(kin, nb, c["psi_seed"])
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_MIXED)
    torch.cuda.synchronize()
    got = _from_t(ht)
    # first and last bands of both stick chunks, and bands inside them
    sel = np.array([0, 1, 37, 66, 67, 68, 69, 101, 126, 127])
    want = _oracle_h(*args, psi[sel])
    assert _rel_band(got[sel], want).max() <= TOL


def test_hpsi_mixed_gamma_c1_odd_band_count(q, ctx):
    c = qeinputs.config("C1")
    args = (c["lat"], c["k"], c["ecut"], c["grid"], c["tau"], c["widths"])
    nb = 127
    prob, keep, miller, kin = _gpu_problem(q, ctx, *args, nb)
    mg = _mirror(miller)
    psi = qeinputs.start_bands(kin, nb, c["psi_seed"])
    psi = 0.5 * (psi + np.conj(psi[:, mg]))          # real in r
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_MIXED | q.QE_GAMMA)
    torch.cuda.synchronize()
    got = _from_t(ht)
    sel = np.array([0, 1, 66, 67, 68, 69, 124, 125, 126])   # 126: the unpaired last band
    want = _oracle_h(*args, psi[sel])
    assert _rel_band(got[sel], want).max() <= TOL


def test_hpsi_batch_mixed_against_oracle(q, ctx):
    """Two k points of the tetragonal cell and two cubic cells of the batched
    workload in one mixed-precision batched call, against the oracle."""
    specs = qeinputs.c3_problems()
    chosen = [specs[0], specs[5], specs[16], specs[17]]
    items = []
    for p in chosen:
        nb = min(p["nbnd"], 24)
        prob, keep, miller, kin = _gpu_problem(q, ctx, p["lat"], p["k"], p["ecut"], p["grid"],
                                               p["tau"], p["widths"], nb)
        psi = qeinputs.start_bands(kin, nb, p["psi_seed"])
        items.append((p, prob, keep, psi, _to_t(psi)))
    outs = [torch.full_like(it[4], float("nan")) for it in items]
    ctx.hpsi_batch([it[1] for it in items], [it[4] for it in items], outs, q.QE_MIXED)
    torch.cuda.synchronize()
    for (p, prob, keep, psi, pt), o in zip(items, outs):
        want = _oracle_h(p["lat"], p["k"], p["ecut"], p["grid"], p["tau"], p["widths"], psi)
        assert _rel_band(_from_t(o), want).max() <= TOL


def _device_problem(q, ctx, name):
    c = qeinputs.config(name)
    prob, keep, miller, kin = _gpu_problem(q, ctx, c["lat"], c["k"], c["ecut"], c["grid"],
                                           c["tau"], c["widths"], c["nbnd"])
    psi0 = qeinputs.start_bands(kin, c["nbnd"], c["psi_seed"])
    return c, prob, keep, _to_t(psi0)


@pytest.mark.parametrize("rr32", [False, True])
def test_c0_mixed_davidson_both_rayleigh_ritz_arithmetics(q, ctx, rr32):
    c, prob, keep, pt = _device_problem(q, ctx, "C0")
    nb = c["nbnd"]
    ev = torch.zeros(nb, dtype=torch.float64, device="cuda")
    rs = torch.zeros_like(ev)
    prec = q.QE_MIXED | (q.QE_RR_FP32 if rr32 else 0)
    rc, it = ctx.davidson(prob, pt, ev, rs, precision=prec, tol=1e-5, max_iter=200)
    torch.cuda.synchronize()
    assert rc == q.QE_OK
    ref = np.loadtxt(os.path.join(GOLDEN, "c0_dense_eigs.txt"))[:nb]
    assert np.abs(ev.cpu().numpy() - ref).max() <= 1e-6
    assert rs.cpu().numpy().max() <= 1e-5
    x = _from_t(pt)
    assert np.abs(np.conj(x) @ x.T - np.eye(nb)).max() <= 1e-10


def test_c2_mixed_davidson_fp32_rayleigh_ritz(q, ctx):
    """C2 with the FP32 reduced eigenproblems (QE_RR_FP32) within 1e-6 Ry of the
    oracle's Davidson; the default (FP64 Rayleigh-Ritz) is covered by the C2
    test of test_gpu_davidson.py."""
    c, prob, keep, pt = _device_problem(q, ctx, "C2")
    ev = torch.zeros(c["nbnd"], dtype=torch.float64, device="cuda")
    rc, it = ctx.davidson(prob, pt, ev, None, precision=q.QE_MIXED | q.QE_RR_FP32, tol=1e-4,
                          max_iter=200)
    torch.cuda.synchronize()
    assert rc == q.QE_OK
    ref = np.loadtxt(os.path.join(GOLDEN, "c2_davidson_eigs.txt"))
    assert np.abs(ev.cpu().numpy() - ref).max() <= 1e-6
