"""One self-consistency step on the GPU (qe_scf_step; Sec. 3.3: electronic
self-consistency, charge-density generation) against the oracle's step:
density, Hartree potential on the density sphere, Slater exchange, linear
mixing.  Element by element on the whole grid: FP64 within 1e-12 of max |V|,
mixed within 2e-5; two k points with an odd mixed-radix grid (SMALL), the
bands of a converged C0 solve, host arrays equal to device arrays bit for bit,
and a grid too small for the density sphere refused."""
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


def _bands(q, c, k, nb, seed):
    _, kin = q.gsphere(c["lat"], k, c["ecut"], c["grid"])
    psi = qeinputs.start_bands(kin, nb, seed)
    return psi / np.linalg.norm(psi, axis=1)[:, None]


def _gpu_step(q, ctx, c, ks, psis, ws, vext, vin, alpha, prec):
    grid = c["grid"]
    shp = (grid[2], grid[1], grid[0])
    vnew = torch.full(shp, float("nan"), dtype=torch.float64, device="cuda")
    rho = torch.full(shp, float("nan"), dtype=torch.float64, device="cuda")
    ctx.scf_step(c["lat"], c["ecut"], grid, np.array(ks), [_to_t(p) for p in psis], ws,
                 torch.from_numpy(vext).cuda(), torch.from_numpy(vin).cuda(), alpha, vnew, rho, prec)
    torch.cuda.synchronize()
    return vnew.cpu().numpy(), rho.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_small_two_k_points(q, ctx, prec, tol):
    c = qeinputs.config("SMALL")
    ks = [c["k"], np.zeros(3)]
    psis = [_bands(q, c, ks[0], 5, 1), _bands(q, c, ks[1], 4, 2)]
    ws = [np.array([2.0, 2.0, 1.0, 1.0, 0.5]), np.array([1.0, 1.0, 0.5, 0.5])]
    vext = oracle.vloc_gaussian(c["lat"], c["grid"], c["tau"])
    vin = 0.8 * vext
    want, rho_w = oracle.scf_step(c["lat"], c["ecut"], c["grid"], ks, psis, ws, vext, vin, 0.3)
    got, rho_g = _gpu_step(q, ctx, c, ks, psis, ws, vext, vin, 0.3, prec)
    assert np.abs(rho_g - rho_w).max() <= tol * np.abs(rho_w).max()
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_step_from_converged_c0_bands(q, ctx):
    c = qeinputs.config("C0")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device="cuda")
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    beta = torch.empty((8, npw, 2), dtype=torch.float64, device="cuda")
    ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
    d = torch.from_numpy(qeinputs.d_matrix(2, 1)).cuda()
    prob = ctx.problem(lat, k, ecut, grid, v, beta, d, 4)
    pt = _to_t(qeinputs.start_bands(kin, 4, 0))
    ev = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc, it = ctx.davidson(prob, pt, ev, None, tol=1e-9)
    assert rc == q.QE_OK
    a = pt.cpu().numpy()
    psi = a[..., 0] + 1j * a[..., 1]
    w = np.full(4, 2.0)
    vext = v.cpu().numpy()
    want, rho = oracle.scf_step(lat, ecut, grid, [k], [psi], [w], vext, vext, 0.5)
    got, rho_g = _gpu_step(q, ctx, c, [k], [psi], [w], vext, vext, 0.5, q.QE_FP64)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    omega = abs(np.linalg.det(lat))
    assert abs(rho_g.sum() * omega / rho_g.size - 8.0) <= 1e-11


def test_host_arrays_and_small_grid(q, ctx):
    c = qeinputs.config("SMALL")
    ks = [c["k"]]
    psi = _bands(q, c, ks[0], 3, 4)
    ws = [np.array([2.0, 1.0, 1.0])]
    vext = oracle.vloc_gaussian(c["lat"], c["grid"], c["tau"])
    dev, rho_d = _gpu_step(q, ctx, c, ks, [psi], ws, vext, vext, 0.25, q.QE_FP64)
    vnew = np.zeros_like(vext)
    rho = np.zeros_like(vext)
    ctx.scf_step(c["lat"], c["ecut"], c["grid"], np.array(ks), [np.ascontiguousarray(psi)], ws,
                 vext, vext.copy(), 0.25, vnew, rho, q.QE_FP64)
    assert np.array_equal(vnew, dev) and np.array_equal(rho, rho_d)
    c0 = qeinputs.config("C0")
    grid = (24, 24, 24)                         # holds the band sphere, not the density sphere
    _, kin = q.gsphere(c0["lat"], c0["k"], c0["ecut"], grid)
    p0 = np.ascontiguousarray(qeinputs.start_bands(kin, 2, 0))
    v0 = np.zeros((24, 24, 24))
    with pytest.raises(q.QEError) as e:
        ctx.scf_step(c0["lat"], c0["ecut"], grid, np.zeros((1, 3)), [p0], [np.ones(2)], v0, v0.copy(),
                     0.5, np.zeros_like(v0))
    assert e.value.code == q.QE_EINVAL
