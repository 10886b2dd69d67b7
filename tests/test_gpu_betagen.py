"""H|psi> with projectors generated on the fly (qe_hpsi_gen; Sec. 3.2.2 item
(viii): calculation of pseudopotential terms) against the FP64 oracle, whose
beta is the stored closed-form transform of the same Gaussian projectors.

The caller describes the projectors by atom positions, angular momenta and
radial tables F_n(|k+G|); the library forms beta from them (structure factor
from per-atom phase tables).  Per band ||Hpsi_gpu - Hpsi_ref|| / ||Hpsi_ref||
<= 1e-12 in FP64, 2e-5 mixed: on the tensor-core path (C1 sampled bands; the
tetragonal cell at a k point off Gamma, where the e^{-ik.R} factor matters) and
on the SIMT path (C0, SMALL with k off Gamma); host arrays give the same bits as
device arrays.
"""
import math

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


def _radial(lat, kin, widths):
    """F_{w,l}(q) of the unit-norm Gaussian projectors: Omega^-1/2 N_l (2 pi)^{3/2}
    w^{2l+3} e^{-w^2 q^2 / 2}, radial functions (w, l = 0), (w, l = 1) per width."""
    omega = abs(np.linalg.det(lat))
    c = (2 * math.pi) ** 1.5 / math.sqrt(omega)
    rows, ls = [], []
    for w in widths:
        g = np.exp(-0.5 * w * w * kin)
        n0 = math.sqrt(4.0 / (math.sqrt(math.pi) * w ** 3))
        n1 = math.sqrt(8.0 / (3.0 * math.sqrt(math.pi) * w ** 5))
        rows += [c * n0 * w ** 3 * g, c * n1 * w ** 5 * g]
        ls += [0, 1]
    return np.ascontiguousarray(rows), np.array(ls, dtype=np.int32)


def _to_t(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.float64).reshape(x.shape + (2,))).cuda()


def _from_t(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _case(q, ctx, lat, k, ecut, grid, tau, widths, nb, seed, sel=None, precision=0):
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device="cuda")
    ctx.vloc_gaussian(lat, grid, tau, v)
    d = qeinputs.d_matrix(len(tau), len(widths))
    rad, ls = _radial(lat, kin, widths)
    prob = ctx.problem_gen(lat, k, ecut, grid, v, torch.from_numpy(d).cuda(), d.shape[0], nb)
    psi = qeinputs.start_bands(kin, nb, seed)
    pt = _to_t(psi)
    ht = torch.full_like(pt, float("nan"))
    ctx.hpsi_gen(prob, tau, ls, torch.from_numpy(rad).cuda(), pt, ht, precision)
    torch.cuda.synchronize()
    got = _from_t(ht)
    sel = np.arange(nb) if sel is None else np.asarray(sel)
    vo = oracle.vloc_gaussian(lat, grid, tau)
    bo = oracle.beta_gaussian(lat, k, ecut, tau, widths)
    want = oracle.hpsi(lat, k, ecut, grid, vo, bo, d, psi[sel])
    rel = np.linalg.norm(got[sel] - want, axis=1) / np.linalg.norm(want, axis=1)
    return float(rel.max()), (prob, tau, ls, rad, psi, got)


@pytest.mark.parametrize("name,prec,tol", [("C0", 0, 1e-12), ("SMALL", 0, 1e-12), ("SMALL", 1, 2e-5)])
def test_simt_path_cells(q, ctx, name, prec, tol):
    c = qeinputs.config(name)
    err, _ = _case(q, ctx, c["lat"], c["k"], c["ecut"], c["grid"], c["tau"], c["widths"], c["nbnd"], 3,
                   precision=prec)
    assert err <= tol


def test_tensor_core_path_c1_sampled(q, ctx):
    c = qeinputs.config("C1")
    err, _ = _case(q, ctx, c["lat"], c["k"], c["ecut"], c["grid"], c["tau"], c["widths"], 128,
                   c["psi_seed"], sel=[0, 1, 64, 127])
    assert err <= 1e-12


def test_tensor_core_path_off_gamma(q, ctx):
    t = qeinputs.config("C3T")
    b = oracle.reciprocal(t["lat"])
    k = 0.25 * b[0] + 0.5 * b[1]
    for prec, tol in ((0, 1e-12), (1, 2e-5)):
        err, _ = _case(q, ctx, t["lat"], k, t["ecut"], t["grid"], t["tau"], t["widths"], 64, 9,
                       sel=[0, 31, 63], precision=prec)
        assert err <= tol


def test_host_arrays_give_the_same_bits(q, ctx):
    c = qeinputs.config("C3T")
    lat, k, ecut, grid = c["lat"], np.zeros(3), c["ecut"], c["grid"]
    _, kin = q.gsphere(lat, k, ecut, grid)
    v = np.zeros((grid[2], grid[1], grid[0]))
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    rad, ls = _radial(lat, kin, c["widths"])
    nb = 40
    psi = qeinputs.start_bands(kin, nb, 4)
    prob_h = ctx.problem_gen(lat, k, ecut, grid, v, d, d.shape[0], nb)
    out_h = np.zeros_like(psi)
    ctx.hpsi_gen(prob_h, c["tau"], ls, rad, np.ascontiguousarray(psi), out_h)
    prob_d = ctx.problem_gen(lat, k, ecut, grid, torch.from_numpy(v).cuda(), torch.from_numpy(d).cuda(),
                             d.shape[0], nb)
    ht = torch.empty(nb, len(kin), 2, dtype=torch.float64, device="cuda")
    ctx.hpsi_gen(prob_d, c["tau"], ls, torch.from_numpy(rad).cuda(), _to_t(psi), ht)
    torch.cuda.synchronize()
    assert np.array_equal(out_h, _from_t(ht))
