"""Pins of the oracle's charge density (Sec. 3.3: charge-density generation):

* Parseval: (Omega / N) sum_j rho(r_j) = sum_nk w_nk sum_G |c_nk(G)|^2;
* one plane wave: |psi(r)|^2 = |c|^2 at every grid point;
* two plane waves: |a|^2 + |b|^2 + 2 Re(a conj(b) e^{i (G_a - G_b).r}) in closed form
  (Cartesian G and r, so that a transposed lattice or a swapped axis fails);
* an O(N_G N_r) direct sum over plane waves and grid points on tiny grids (a
  skewed cell, k off Gamma, two k points with different weights);
* translating every band by a grid vector t (c_G -> c_G e^{-iG.t}) rolls rho by t.
"""
import numpy as np
import pytest

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


def test_parseval_charge():
    c = qeinputs.config("SMALL")
    lat, ecut, grid = c["lat"], c["ecut"], c["grid"]
    ks = [c["k"], np.zeros(3)]
    psis, ws = [], []
    for i, k in enumerate(ks):
        m, _, _ = oracle.gsphere(lat, k, ecut)
        psis.append(qeinputs.random_vectors(3, len(m), seed=10 + i))
        ws.append(np.array([2.0, 1.0, 0.5]) * (0.25 + 0.5 * i))
    rho = oracle.density(lat, ecut, grid, ks, psis, ws)
    omega = oracle.volume(lat)
    want = sum(float(np.sum(w * np.sum(np.abs(p) ** 2, axis=1))) for p, w in zip(psis, ws))
    assert abs(rho.sum() * omega / rho.size - want) <= 1e-12 * want
    assert rho.min() >= 0.0


def test_single_and_two_plane_waves():
    lat = np.array([[7.0, 0.0, 0.0], [1.0, 8.0, 0.0], [0.5, -0.7, 9.0]])
    k = np.array([0.05, -0.1, 0.02])
    ecut, grid = 6.0, (20, 21, 24)
    m, _, q = oracle.gsphere(lat, k, ecut)
    omega = oracle.volume(lat)
    c = np.zeros((1, len(m)), dtype=complex)
    c[0, 7] = 0.6 - 0.8j
    rho = oracle.density(lat, ecut, grid, [k], [c], [np.array([1.5])])
    np.testing.assert_allclose(rho, 1.5 / omega, rtol=1e-13, atol=0)
    ia, ib = 3, 40
    a, b = 0.3 + 0.4j, -0.7 + 0.2j
    c = np.zeros((1, len(m)), dtype=complex)
    c[0, ia], c[0, ib] = a, b
    rho = oracle.density(lat, ecut, grid, [k], [c], [np.array([2.0])])
    g = q[ia] - q[ib]                               # G_a - G_b (k cancels)
    r = _pts(lat, grid)
    want = 2.0 / omega * (abs(a) ** 2 + abs(b) ** 2 + 2 * np.real(a * np.conj(b) * np.exp(1j * (r @ g))))
    np.testing.assert_allclose(rho, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_direct_sum_on_tiny_grid():
    lat = np.array([[5.0, 0.0, 0.0], [1.0, 5.5, 0.0], [0.5, -0.7, 6.0]])
    ecut, grid = 3.5, (7, 6, 8)
    ks = [np.array([0.0, 0.13, -0.07]), np.zeros(3)]
    r = _pts(lat, grid).reshape(-1, 3)
    psis, ws, want = [], [], np.zeros(r.shape[0])
    for i, k in enumerate(ks):
        m, _, q = oracle.gsphere(lat, k, ecut)
        oracle.check_grid(m, grid)
        p = qeinputs.random_vectors(2, len(m), seed=30 + i)
        w = np.array([1.0, 0.3]) * (1 + i)
        gk = q - k[None, :]                          # Cartesian G
        for cn, wn in zip(p, w):
            val = np.exp(1j * (r @ gk.T)) @ cn       # sum_G c_G e^{iG.r}
            want += wn * np.abs(val) ** 2
        psis.append(p)
        ws.append(w)
    want = want.reshape(grid[2], grid[1], grid[0]) / oracle.volume(lat)
    got = oracle.density(lat, ecut, grid, ks, psis, ws)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * want.max())


def test_translation_by_a_grid_vector_rolls_the_density():
    c = qeinputs.config("C0")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    m, _, q = oracle.gsphere(lat, k, ecut)
    psi = qeinputs.random_vectors(3, len(m), seed=5)
    w = np.array([2.0, 2.0, 1.0])
    rho = oracle.density(lat, ecut, grid, [k], [psi], [w])
    shift = (3, 5, 2)                                 # grid steps along a1, a2, a3
    t = sum(shift[i] / grid[i] * lat[i] for i in range(3))
    g = q - k[None, :]
    moved = psi * np.exp(-1j * (g @ t))[None, :]
    rho2 = oracle.density(lat, ecut, grid, [k], [moved], [w])
    want = np.roll(rho, shift=(shift[2], shift[1], shift[0]), axis=(0, 1, 2))
    np.testing.assert_allclose(rho2, want, rtol=0, atol=1e-13 * rho.max())
