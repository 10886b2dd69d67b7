"""GPU band-by-band conjugate-gradient eigensolver (Sec. 3.3: iterative solution
of the Kohn-Sham Hamiltonian with the conjugate-gradient method) through the C
ABI, pinned like the Davidson: the oracle's stored dense-diagonalisation
eigenvalues of C0 and SMALL (1e-10 Ry in FP64, 1e-6 Ry mixed), the empty-lattice
closed form, a constant potential shift, orthonormal bands with residuals
within tol, host and device arrays alike, reported non-convergence."""
import os

import numpy as np
import pytest

import qeinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name))


@pytest.fixture(scope="module")
def q():
    import paper_2104_10502_gb300 as q
    return q


@pytest.fixture(scope="module")
def ctx(q):
    c = q.Context(0)
    yield c
    c.close()


def _setup(q, ctx, name, empty=False, vshift=0.0):
    c = qeinputs.config(name)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    nb = c["nbnd"]
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    dev = torch.device("cuda", 0)
    v = torch.zeros((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    beta = d = None
    if not empty:
        ctx.vloc_gaussian(lat, grid, c["tau"], v)
        v += vshift
        nproj = 4 * len(c["widths"]) * len(c["tau"])
        beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
        ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
        d = torch.from_numpy(qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))).to(dev)
    psi0 = qeinputs.start_bands(kin, nb, c["psi_seed"])
    pt = torch.from_numpy(psi0.view(np.float64).reshape(nb, npw, 2).copy()).to(dev)
    return c, ctx.problem(lat, k, ecut, grid, v, beta, d, nb), pt, (v, beta, d)


def _cg(q, ctx, prob, pt, tol, precision=None, **kw):
    nb = prob.nbnd
    ev = torch.zeros(nb, dtype=torch.float64, device="cuda")
    rs = torch.zeros(nb, dtype=torch.float64, device="cuda")
    rc, it = ctx.cg(prob, pt, ev, rs, precision=q.QE_FP64 if precision is None else precision,
                    tol=tol, **kw)
    torch.cuda.synchronize()
    return rc, it, ev.cpu().numpy(), rs.cpu().numpy()


def _orthonormal(pt, tol):
    p = pt.cpu().numpy()
    p = p[..., 0] + 1j * p[..., 1]
    assert np.abs(np.conj(p) @ p.T - np.eye(p.shape[0])).max() <= tol


def test_c0_fp64_matches_dense_diagonalisation(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "C0")
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-8)
    assert rc == q.QE_OK and it > 0
    assert rs.max() <= 1e-8
    assert np.abs(ev - _golden("c0_dense_eigs.txt")[:c["nbnd"]]).max() <= 1e-10
    _orthonormal(pt, 1e-12)


def test_small_off_gamma_and_constant_shift(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "SMALL")
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-8)
    assert rc == q.QE_OK
    ref = _golden("small_dense_eigs.txt")[:c["nbnd"]]
    assert np.abs(ev - ref).max() <= 1e-10
    c, prob, pt, keep = _setup(q, ctx, "SMALL", vshift=0.37)
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-8)
    assert rc == q.QE_OK
    assert np.abs(ev - (ref + 0.37)).max() <= 1e-10


def test_empty_lattice_closed_form(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "C0", empty=True)
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-8)
    assert rc == q.QE_OK
    assert np.abs(ev - _golden("c0_empty_lattice.txt")).max() <= 1e-10


def test_c0_mixed_within_1e6(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "C0")
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-5, precision=q.QE_MIXED)
    assert rc == q.QE_OK
    assert rs.max() <= 1e-5
    assert np.abs(ev - _golden("c0_dense_eigs.txt")[:c["nbnd"]]).max() <= 1e-6


def test_host_memory_matches_device(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "SMALL")
    v, beta, d = keep
    psi_h = pt.cpu().numpy().copy()
    psi_h = np.ascontiguousarray(psi_h[..., 0] + 1j * psi_h[..., 1])
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-8)
    prob_h = ctx.problem(c["lat"], c["k"], c["ecut"], c["grid"], v.cpu().numpy().copy(),
                         beta.cpu().numpy().copy(), d.cpu().numpy().copy(), c["nbnd"])
    ev_h = np.zeros(c["nbnd"])
    rc_h, it_h = ctx.cg(prob_h, psi_h, ev_h, None, tol=1e-8)
    assert rc_h == q.QE_OK and it_h == it
    assert np.array_equal(ev_h, ev)


def test_nonconvergence_returns_best_bands(q, ctx):
    c, prob, pt, keep = _setup(q, ctx, "C0")
    rc, it, ev, rs = _cg(q, ctx, prob, pt, 1e-12, max_iter=2, max_sweeps=1)
    assert rc == q.QE_ENOCONV
    assert np.all(np.isfinite(ev)) and np.all(rs > 0)
    ref = _golden("c0_dense_eigs.txt")[:c["nbnd"]]
    assert np.all(ev >= ref - 1e-10)          # Ritz values bound the eigenvalues from above
