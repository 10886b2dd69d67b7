"""GPU parity of H|psi> and of the pseudopotential builders against the FP64
oracle (Sec. 3.3: kinetic, local-potential and pseudopotential contributions;
Sec. 3.2.2 (viii): pseudopotential terms).

Both sides build their own V_loc(r) and beta(G) from the same seeded cell
(qeinputs); the GPU path is called through the C ABI (ctypes binding).
Tolerances: FP64 per band ||Hpsi_gpu - Hpsi_ref|| / ||Hpsi_ref|| <= 1e-12;
mixed (FP32 FFT and FP32 products) <= 2e-5.
"""
import numpy as np
import pytest

import oracle
import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_2104_10502_gb300 as q
    return q


@pytest.fixture(scope="module")
def ctx(q):
    c = q.Context(0)
    yield c
    c.close()


def _cell(name, **over):
    c = dict(qeinputs.config(name))
    c.update(over)
    return c


def _oracle_problem(c):
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    return v, beta, d


def _gpu_problem(q, ctx, c, nb):
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    miller, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    dev = torch.device("cuda", 0)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    nproj = 4 * len(c["widths"]) * len(c["tau"])
    beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
    ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
    d = torch.from_numpy(qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))).to(dev)
    prob = ctx.problem(lat, k, ecut, grid, v, beta, d, nb)
    return prob, (v, beta, d), kin


def _to_t(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.float64).reshape(x.shape + (2,))).cuda()


def _from_t(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _rel_band(got, want):
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


@pytest.mark.parametrize("name", ["SMALL", "C0"])
def test_builders_match_oracle(q, ctx, name):
    c = _cell(name)
    v, beta, _ = _oracle_problem(c)
    _, (vg, bg, _), _ = _gpu_problem(q, ctx, c, 1)
    torch.cuda.synchronize()
    np.testing.assert_allclose(vg.cpu().numpy(), v, rtol=0, atol=1e-14)
    np.testing.assert_allclose(_from_t(bg), beta, rtol=0, atol=1e-14 * np.abs(beta).max())


def test_builders_c1_sampled(q, ctx):
    c = _cell("C1")
    _, (vg, bg, _), kin = _gpu_problem(q, ctx, c, 1)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, n, 200) for n in c["grid"]], axis=1)
    vs = oracle.vloc_gaussian(c["lat"], c["grid"], c["tau"], points=pts)
    gv = vg.cpu().numpy()[pts[:, 2], pts[:, 1], pts[:, 0]]
    np.testing.assert_allclose(gv, vs, rtol=0, atol=1e-14)
    beta = oracle.beta_gaussian(c["lat"], c["k"], c["ecut"], c["tau"][:3], c["widths"])
    np.testing.assert_allclose(_from_t(bg[:beta.shape[0]]), beta, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name,nb", [("SMALL", 7), ("C0", 8), ("SMALL", 1), ("C0", 33)])
def test_hpsi_fp64_matches_oracle(q, ctx, name, nb):
    c = _cell(name)
    v, beta, d = _oracle_problem(c)
    prob, keep, kin = _gpu_problem(q, ctx, c, nb)
    psi = qeinputs.random_vectors(nb, len(kin), seed=7)
    want = oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, psi)
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_FP64)
    torch.cuda.synchronize()
    got = _from_t(ht)
    assert _rel_band(got, want).max() <= 1e-12


@pytest.mark.parametrize("name,grid", [("SMALL", None), ("C0", None), ("C0", (16, 16, 16))])
def test_hpsi_fp64_both_fft_arithmetics(q, ctx, name, grid):
    """The FP64 path's two FFT arithmetics -- float-float pairs (default) and
    float64 on the FP64 pipe (QE_FFT_FP64PIPE) -- each within 1e-12 of the
    oracle, on mixed-radix grids (radix 3 and 5 twiddled stages) and on a grid
    too small for the padding skip (C0's sphere, max |m| = 7, on 16 points:
    4 * 7 >= 16, so the first radix-4 stage takes all four inputs)."""
    c = _cell(name) if grid is None else _cell(name, grid=grid)
    nb = 6
    v, beta, d = _oracle_problem(c)
    prob, keep, kin = _gpu_problem(q, ctx, c, nb)
    psi = qeinputs.random_vectors(nb, len(kin), seed=11)
    want = oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, psi)
    pt = _to_t(psi)
    got = {}
    for lab, prec in (("ff", q.QE_FP64), ("pipe", q.QE_FP64 | q.QE_FFT_FP64PIPE)):
        ht = torch.empty_like(pt)
        ctx.hpsi(prob, pt, ht, prec)
        torch.cuda.synchronize()
        got[lab] = _from_t(ht)
        assert _rel_band(got[lab], want).max() <= 1e-12, lab
    # the flag only selects the FFT arithmetic of QE_FP64: ignored with QE_MIXED
    hm = torch.empty_like(pt)
    hm2 = torch.empty_like(pt)
    ctx.hpsi(prob, pt, hm, q.QE_MIXED)
    ctx.hpsi(prob, pt, hm2, q.QE_MIXED | q.QE_FFT_FP64PIPE)
    torch.cuda.synchronize()
    assert torch.equal(hm, hm2)


def test_hpsi_c1_full_size_fp64(q, ctx):
    c = _cell("C1")
    nb = c["nbnd"]
    v, beta, d = _oracle_problem(c)
    prob, keep, kin = _gpu_problem(q, ctx, c, nb)
    psi = qeinputs.start_bands(kin, nb, c["psi_seed"])
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_FP64)
    torch.cuda.synchronize()
    got = _from_t(ht)
    sel = np.array([0, 1, 63, 64, 126, 127])          # sampled bands, the oracle one by one
    want = oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, psi[sel])
    assert _rel_band(got[sel], want).max() <= 1e-12
    # Hermiticity of the GPU operator on the whole block: <psi_i|H psi_j>
    g = np.conj(psi[:16]) @ got[:16].T
    assert np.abs(g - g.conj().T).max() <= 1e-12 * np.abs(g).max()


def test_hpsi_mixed_matches_oracle(q, ctx):
    c = _cell("C0")
    nb = 8
    v, beta, d = _oracle_problem(c)
    prob, keep, kin = _gpu_problem(q, ctx, c, nb)
    psi = qeinputs.start_bands(kin, nb, 1)
    want = oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, psi)
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_MIXED)
    torch.cuda.synchronize()
    assert _rel_band(_from_t(ht), want).max() <= 2e-5


@pytest.mark.parametrize("prec_name,nb", [("QE_FP64", 5), ("QE_FP64", 19), ("QE_MIXED", 11)])
def test_hpsi_host_memory_matches_device(q, ctx, prec_name, nb):
    """Host buffers (psi uploaded in band chunks beside the FFTs, beta beside
    them too) give bit for bit the device-buffer result."""
    prec = getattr(q, prec_name)
    c = _cell("SMALL")
    prob_d, (vg, bg, dg), kin = _gpu_problem(q, ctx, c, nb)
    psi = qeinputs.random_vectors(nb, len(kin), seed=3)
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob_d, pt, ht, prec)
    torch.cuda.synchronize()
    vh = vg.cpu().numpy().copy()
    bh = bg.cpu().numpy().copy()
    dh = dg.cpu().numpy().copy()
    prob_h = ctx.problem(c["lat"], c["k"], c["ecut"], c["grid"], vh, bh, dh, nb)
    out = np.zeros_like(psi)
    ctx.hpsi(prob_h, np.ascontiguousarray(psi), out, prec)
    assert np.array_equal(out, _from_t(ht))


def test_hpsi_empty_lattice_and_no_projectors(q, ctx):
    c = _cell("SMALL")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    miller, kin = q.gsphere(lat, k, ecut, grid)
    v = torch.zeros((grid[2], grid[1], grid[0]), dtype=torch.float64, device="cuda")
    prob = ctx.problem(lat, k, ecut, grid, v, None, None, 3)
    psi = qeinputs.random_vectors(3, len(kin), seed=4)
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_FP64)
    torch.cuda.synchronize()
    np.testing.assert_allclose(_from_t(ht), kin[None, :] * psi, rtol=0, atol=1e-13)


def test_hpsi_zero_bands_is_a_no_op(q, ctx):
    c = _cell("SMALL")
    prob, keep, kin = _gpu_problem(q, ctx, c, 0)
    ctx.hpsi(prob, None, None, q.QE_FP64)


def test_hpsi_rejects_bad_grids(q, ctx):
    c = _cell("C0")
    v = torch.zeros((14, 32, 32), dtype=torch.float64, device="cuda")
    prob = ctx.problem(c["lat"], c["k"], c["ecut"], (32, 32, 14), v, None, None, 1)
    pt = torch.zeros((1, 1503, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QEError) as e:
        ctx.hpsi(prob, pt, torch.empty_like(pt))
    assert e.value.code == q.QE_EINVAL
    v = torch.zeros((33, 32, 32), dtype=torch.float64, device="cuda")   # 33 = 3 * 11
    prob = ctx.problem(c["lat"], c["k"], c["ecut"], (32, 32, 33), v, None, None, 1)
    with pytest.raises(q.QEError) as e:
        ctx.hpsi(prob, pt, torch.empty_like(pt))
    assert e.value.code == q.QE_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_same_operator_flag_reuses_and_invalidates(q, ctx, prec):
    """QE_SAME_OPERATOR reuses the prepared operator of the previous call (bit
    for bit the same result); another operator prepared in between (a second
    cell, a Davidson solve) makes the flag fall back to rebuilding it."""
    c0 = _cell("C0")
    sm = _cell("SMALL")
    p0, keep0, kin0 = _gpu_problem(q, ctx, c0, 6)
    p1, keep1, kin1 = _gpu_problem(q, ctx, sm, 5)
    x0 = _to_t(qeinputs.random_vectors(6, len(kin0), seed=31))
    x1 = _to_t(qeinputs.random_vectors(5, len(kin1), seed=32))
    ref0, ref1 = torch.empty_like(x0), torch.empty_like(x1)
    ctx.hpsi(p0, x0, ref0, prec)
    ctx.hpsi(p1, x1, ref1, prec)
    out = torch.empty_like(x1)
    ctx.hpsi(p1, x1, out, prec | q.QE_SAME_OPERATOR)          # same as the previous call
    torch.cuda.synchronize()
    assert torch.equal(out, ref1)
    out0 = torch.empty_like(x0)
    ctx.hpsi(p0, x0, out0, prec | q.QE_SAME_OPERATOR)         # another operator: rebuilt
    torch.cuda.synchronize()
    assert torch.equal(out0, ref0)
    ev = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.davidson(p1, x1.clone(), ev, None, precision=prec, tol=1e-5)
    ctx.hpsi(p0, x0, out0, prec | q.QE_SAME_OPERATOR)         # after a solve in between
    torch.cuda.synchronize()
    assert torch.equal(out0, ref0)
