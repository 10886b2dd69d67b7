"""The k = 0 real-band mode (the Gamma-point trick the paper mentions in
Sec. 3.3: at k = 0 the wavefunctions can be taken real in r, c(-G) = conj c(G),
which halves the FFT work): two such bands share one complex FFT, the
projections are real.

Checked through the C ABI against the FP64 oracle (whose H is the plain
definition, no pairing): H|psi> of bands real in r with QE_GAMMA within the
qe_hpsi tolerances (FP64 1e-12 per band, mixed 2e-5), odd band counts, a cell
off k = 0 where the flag must be ignored; Davidson solves with the mode (the
default at k = 0) against the same solves without it (QE_NO_GAMMA) and the
stored dense eigenvalues, and the returned bands real in r (the mode is the
default for solves on grids of at least 48^3 points, mixed ones with
QE_RR_FP32 excepted, else on request).
"""
import os

import numpy as np
import pytest

import oracle
import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def _mirror(miller):
    """Index of -G for every G of the sphere (host, from the Miller indices)."""
    key = {tuple(m): i for i, m in enumerate(miller)}
    return np.array([key[tuple(-m)] for m in miller])


def _real_in_r(psi, mg):
    """(psi + conj psi(-G)) / 2: the real-in-r part of every band."""
    return 0.5 * (psi + np.conj(psi[:, mg]))


def _problem(q, ctx, c, nb):
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
    return ctx.problem(lat, k, ecut, grid, v, beta, d, nb), (v, beta, d), np.asarray(miller), kin


def _oracle_h(c, psi):
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    return oracle.hpsi(lat, k, ecut, grid, v, beta, d, psi)


# prec: 0 = QE_FP64 (float-float FFT), 1 = QE_MIXED, 0x400 = QE_FP64 | QE_FFT_FP64PIPE
@pytest.mark.parametrize("nb,prec,tol", [(8, 0, 1e-12), (7, 0, 1e-12), (1, 0, 1e-12), (9, 1, 2e-5),
                                         (7, 0x400, 1e-12)])
def test_gamma_hpsi_matches_oracle(q, ctx, nb, prec, tol):
    c = qeinputs.config("C0")
    prob, keep, miller, kin = _problem(q, ctx, c, nb)
    psi = _real_in_r(qeinputs.random_vectors(nb, len(kin), seed=11), _mirror(miller))
    want = _oracle_h(c, psi)
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, prec | q.QE_GAMMA)
    torch.cuda.synchronize()
    got = _from_t(ht)
    assert _rel_band(got, want).max() <= tol
    # the paired result is itself real in r
    mg = _mirror(miller)
    assert np.abs(got - np.conj(got[:, mg])).max() <= 10 * tol * np.abs(got).max()


# nb = 7: an odd band count at C1 size, where the FP64 projections take the
# real-output tensor-core product with a ragged last column pair
@pytest.mark.parametrize("nb", [128, 7])
def test_gamma_hpsi_c1_sampled(q, ctx, nb):
    c = qeinputs.config("C1")
    prob, keep, miller, kin = _problem(q, ctx, c, nb)
    psi = _real_in_r(qeinputs.start_bands(kin, nb, c["psi_seed"]), _mirror(miller))
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_FP64 | q.QE_GAMMA)
    torch.cuda.synchronize()
    got = _from_t(ht)
    # both halves of three band pairs; all of the odd block
    sel = np.array([0, 1, 62, 63, 126, 127]) if nb == 128 else np.arange(nb)
    want = _oracle_h(c, psi[sel])
    assert _rel_band(got[sel], want).max() <= 1e-12


def test_gamma_hpsi_c1_unlike_norms(q, ctx):
    """Neighbouring bands of very different norm (1 and 1e-6, as the projected
    corrections of an orthonormalisation pass can be): the real-output
    projection product gives each band its own exponent, so the weak bands
    keep the FP64 tolerance relative to their own norm.  V_loc = 0, because
    bands 2b and 2b+1 also share one FFT, whose rounding is relative to the
    pair (V = 0 makes the local term exactly zero, isolating the kinetic and
    nonlocal terms)."""
    c = qeinputs.config("C1")
    nb = 16
    prob, keep, miller, kin = _problem(q, ctx, c, nb)
    keep[0].zero_()
    psi = _real_in_r(qeinputs.start_bands(kin, nb, c["psi_seed"]), _mirror(miller))
    psi[1::2] *= 1e-6
    pt = _to_t(psi)
    ht = torch.empty_like(pt)
    ctx.hpsi(prob, pt, ht, q.QE_FP64 | q.QE_GAMMA)
    torch.cuda.synchronize()
    got = _from_t(ht)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    want = oracle.hpsi(lat, k, ecut, grid, np.zeros((grid[2], grid[1], grid[0])), beta, d, psi)
    assert _rel_band(got, want).max() <= 1e-12


def test_gamma_flag_is_ignored_off_gamma(q, ctx):
    c = qeinputs.config("SMALL")
    assert np.any(np.asarray(c["k"]) != 0.0)
    nb = 5
    prob, keep, miller, kin = _problem(q, ctx, c, nb)
    psi = qeinputs.random_vectors(nb, len(kin), seed=3)
    pt = _to_t(psi)
    h1, h2 = torch.empty_like(pt), torch.empty_like(pt)
    ctx.hpsi(prob, pt, h1, q.QE_FP64)
    ctx.hpsi(prob, pt, h2, q.QE_FP64 | q.QE_GAMMA)
    torch.cuda.synchronize()
    assert torch.equal(h1, h2)


@pytest.mark.parametrize("prec,tol,etol", [(0, 1e-8, 1e-10), (1, 1e-5, 1e-6)])
def test_davidson_gamma_mode_matches_complex_bands(q, ctx, prec, tol, etol):
    c = qeinputs.config("C0")
    nb = c["nbnd"]
    prob, keep, miller, kin = _problem(q, ctx, c, nb)
    psi0 = qeinputs.start_bands(kin, nb, c["psi_seed"])
    ref = np.loadtxt(os.path.join(GOLDEN, "c0_dense_eigs.txt"))[:nb]
    out = {}
    on = q.QE_GAMMA        # C0 (32^3 grid) is below the size where solves take the mode by default
    for flag in (on, q.QE_NO_GAMMA):
        pt = _to_t(psi0)
        ev = torch.zeros(nb, dtype=torch.float64, device="cuda")
        rs = torch.zeros_like(ev)
        rc, it = ctx.davidson(prob, pt, ev, rs, precision=prec | flag, tol=tol, max_iter=200)
        assert rc == 0
        out[flag] = (ev.cpu().numpy(), _from_t(pt), rs.cpu().numpy())
        assert np.abs(out[flag][0] - ref).max() <= etol
        assert out[flag][2].max() <= tol
    assert np.abs(out[on][0] - out[q.QE_NO_GAMMA][0]).max() <= 2 * etol
    # the k = 0 mode returns bands real in r, orthonormal
    mg = _mirror(miller)
    x = out[on][1]
    assert np.abs(x - np.conj(x[:, mg])).max() <= 1e-12
    g = np.conj(x) @ x.T
    assert np.abs(g - np.eye(nb)).max() <= (1e-10 if prec == 0 else 1e-6)
