"""Pins of the oracle's self-consistency step (Sec. 3.3: electronic
self-consistency, charge-density generation):

* a cosine density rho0 + A cos(g.r) (g on the density sphere) has the
  closed-form Hartree potential 8 pi A cos(g.r) / |g|^2 (Cartesian g and r);
* a direct O(N_G N_r) sum of the Hartree definition on a tiny skewed grid;
* V_H has zero mean (the G = 0 term is dropped);
* the Slater exchange formula at a known point and its scaling
  v_x(8 rho) = 2 v_x(rho);
* the mixing end points (alpha = 0 keeps V_in, alpha = 1 gives V_out) and
  linearity in alpha, with the step's density equal to density().
"""
import math

import numpy as np

import oracle
import qeinputs


def _pts(lat, grid):
    n1, n2, n3 = grid
    out = np.zeros((n3, n2, n1, 3))
    for j2 in range(n3):
        for j1 in range(n2):
            for j0 in range(n1):
                out[j2, j1, j0] = j0 / n1 * lat[0] + j1 / n2 * lat[1] + j2 / n3 * lat[2]
    return out


def test_cosine_density_closed_form():
    lat = np.array([[9.0, 0.0, 0.0], [1.0, 10.0, 0.0], [0.5, -0.8, 11.0]])
    grid = (30, 32, 36)
    b = oracle.reciprocal(lat)
    r = _pts(lat, grid)
    for m in [(1, 0, 0), (2, -1, 1), (0, 3, -2)]:
        g = np.array(m) @ b
        rho = 0.05 + 0.01 * np.cos(r @ g)
        vh = oracle.hartree(lat, 40.0, grid, rho)
        want = 8 * math.pi * 0.01 * np.cos(r @ g) / (g @ g)
        np.testing.assert_allclose(vh, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_direct_sum_on_tiny_grid():
    lat = np.array([[5.0, 0.0, 0.0], [1.0, 5.5, 0.0], [0.5, -0.7, 6.0]])
    grid = (9, 10, 11)
    ecut_rho = 6.0
    rng = np.random.default_rng(1)
    rho = rng.random((grid[2], grid[1], grid[0]))
    _, kin, q = oracle.gsphere(lat, np.zeros(3), ecut_rho)
    r = _pts(lat, grid).reshape(-1, 3)
    ph = np.exp(-1j * (r @ q.T))                  # (Nr, NG), G = q at k = 0
    rg = ph.T @ rho.ravel() / r.shape[0]
    vg = np.where(kin > 0, 8 * math.pi * rg / np.where(kin > 0, kin, 1.0), 0.0)
    want = np.real(np.conj(ph) @ vg).reshape(rho.shape)
    got = oracle.hartree(lat, ecut_rho, grid, rho)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert abs(got.mean()) <= 1e-13 * np.abs(got).max()


def test_exchange_formula():
    rho = np.array([0.0, 1.0, 0.01, 0.37])
    v = oracle.exchange(rho)
    assert v[0] == 0.0
    assert abs(v[1] + 2.0 * (3.0 / math.pi) ** (1.0 / 3.0)) <= 1e-15
    np.testing.assert_allclose(oracle.exchange(8.0 * rho), 2.0 * v, rtol=1e-14, atol=0)


def test_mixing_end_points_and_density():
    c = qeinputs.config("SMALL")
    lat, ecut, grid = c["lat"], c["ecut"], c["grid"]
    _, kin, _ = oracle.gsphere(lat, c["k"], ecut)
    psi = qeinputs.start_bands(kin, 3, 2)
    psi /= np.linalg.norm(psi, axis=1)[:, None]
    w = np.array([2.0, 2.0, 1.0])
    vext = oracle.vloc_gaussian(lat, grid, c["tau"])
    vin = 0.5 * vext
    v0, rho = oracle.scf_step(lat, ecut, grid, [c["k"]], [psi], [w], vext, vin, 0.0)
    v1, _ = oracle.scf_step(lat, ecut, grid, [c["k"]], [psi], [w], vext, vin, 1.0)
    vh, _ = oracle.scf_step(lat, ecut, grid, [c["k"]], [psi], [w], vext, vin, 0.3)
    np.testing.assert_array_equal(v0, vin)
    np.testing.assert_allclose(vh, 0.7 * vin + 0.3 * v1, rtol=0, atol=1e-14 * np.abs(v1).max())
    np.testing.assert_array_equal(rho, oracle.density(lat, ecut, grid, [c["k"]], [psi], [w]))
    vout = vext + oracle.hartree(lat, 4 * ecut, grid, rho) + oracle.exchange(rho)
    np.testing.assert_allclose(v1, vout, rtol=0, atol=1e-15 * np.abs(vout).max())
