"""GPU charge density (Sec. 3.3: charge-density generation) through the C ABI
against the FP64 oracle's definition, rho(r) = (1/Omega) sum_nk w_nk
|psi_nk(r)|^2, element by element on the whole grid:

* FP64 (float-float FFT) within 1e-12 of max |rho|; mixed (FP32 FFT) within 2e-5;
* an odd mixed-radix grid with two k points of different weights (SMALL);
* the k = 0 band pairs (QE_GAMMA) with an odd band count and unequal weights;
* the full C1 size (96^3 grid, 128 bands in two stick chunks);
* the charge (Omega / N) sum rho = sum w ||c||^2, host arrays equal to device
  arrays bit for bit, no k points gives zero density.
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


def _to_t(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.float64).reshape(x.shape + (2,))).cuda()


def _gpu_rho(q, ctx, c, ks, psis, ws, precision):
    grid = c["grid"]
    rho = torch.full((grid[2], grid[1], grid[0]), float("nan"), dtype=torch.float64, device="cuda")
    ctx.density(c["lat"], c["ecut"], grid, np.array(ks), [_to_t(p) for p in psis], ws, rho, precision)
    torch.cuda.synchronize()
    return rho.cpu().numpy()


def _bands(q, c, k, nb, seed):
    _, kin = q.gsphere(c["lat"], k, c["ecut"], c["grid"])
    return qeinputs.start_bands(kin, nb, seed)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_small_two_k_points(q, ctx, prec, tol):
    c = qeinputs.config("SMALL")
    ks = [c["k"], np.zeros(3)]
    psis = [_bands(q, c, ks[0], 7, 1), _bands(q, c, ks[1], 5, 2)]
    ws = [np.linspace(2.0, 0.5, 7), np.array([0.25, 0.5, 0.75, 1.0, 1.25])]
    want = oracle.density(c["lat"], c["ecut"], c["grid"], ks, psis, ws)
    got = _gpu_rho(q, ctx, c, ks, psis, ws, prec)
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_gamma_pairs_odd_count(q, ctx, prec, tol):
    c = qeinputs.config("C0")
    miller, _ = q.gsphere(c["lat"], c["k"], c["ecut"], c["grid"])
    key = {tuple(m): i for i, m in enumerate(np.asarray(miller))}
    mg = np.array([key[tuple(-m)] for m in np.asarray(miller)])
    psi = _bands(q, c, c["k"], 7, 3)
    psi = 0.5 * (psi + np.conj(psi[:, mg]))               # real in r
    w = np.array([2.0, 1.0, 2.0, 0.5, 1.5, 2.0, 0.3])
    want = oracle.density(c["lat"], c["ecut"], c["grid"], [c["k"]], [psi], [w])
    got = _gpu_rho(q, ctx, c, [c["k"]], [psi], [w], prec | q.QE_GAMMA)
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    plain = _gpu_rho(q, ctx, c, [c["k"]], [psi], [w], prec)
    assert np.abs(plain - want).max() <= tol * np.abs(want).max()


def test_c1_full_size(q, ctx):
    c = qeinputs.config("C1")
    nb = c["nbnd"]
    psi = _bands(q, c, c["k"], nb, c["psi_seed"])
    psi /= np.linalg.norm(psi, axis=1)[:, None]
    w = np.full(nb, 2.0)
    want = oracle.density(c["lat"], c["ecut"], c["grid"], [c["k"]], [psi], [w])
    got = _gpu_rho(q, ctx, c, [c["k"]], [psi], [w], q.QE_FP64)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    omega = abs(np.linalg.det(c["lat"]))
    assert abs(got.sum() * omega / got.size - 2.0 * nb) <= 1e-11 * nb


def test_host_arrays_and_no_k_points(q, ctx):
    c = qeinputs.config("SMALL")
    ks = [c["k"]]
    psi = _bands(q, c, ks[0], 4, 5)
    w = [np.array([1.0, 2.0, 1.0, 0.5])]
    dev = _gpu_rho(q, ctx, c, ks, [psi], w, q.QE_FP64)
    grid = c["grid"]
    host = np.zeros((grid[2], grid[1], grid[0]))
    ctx.density(c["lat"], c["ecut"], grid, np.array(ks), [np.ascontiguousarray(psi)], w, host, q.QE_FP64)
    assert np.array_equal(host, dev)
    zero = np.full((grid[2], grid[1], grid[0]), 7.0)
    ctx.density(c["lat"], c["ecut"], grid, np.zeros((0, 3)), [], [], zero, q.QE_FP64)
    assert np.all(zero == 0.0)
