"""Pins of the oracle's local potential, kinetic term and full H|psi>
(Sec. 3.3: kinetic-energy and local-potential contributions; Sec. 3.2.1: FFTXlib).

* the FFT route against an O(N_G N_r) direct DFT written in Cartesian
  arithmetic on tiny odd / mixed-radix grids, including a skewed cell and k != 0;
* a single plane wave in gives the analytic Fourier coefficients of the
  periodic Gaussian potential out;
* constant potential and empty lattice;
* Hermiticity and agreement with the element-wise dense matrix.
"""
import math

import numpy as np
import pytest

import oracle
import qeinputs


def _direct_local(lat, k, ecut, grid, vloc, psi):
    _, _, q = oracle.gsphere(lat, k, ecut)
    g = q - np.asarray(k)[None, :]                  # Cartesian G
    n1, n2, n3 = grid
    pts = []
    for j2 in range(n3):
        for j1 in range(n2):
            for j0 in range(n1):
                pts.append(j0 / n1 * lat[0] + j1 / n2 * lat[1] + j2 / n3 * lat[2])
    r = np.array(pts)                                # x fastest, matches vloc.ravel()
    ph = np.exp(1j * (r @ g.T))                      # (Nr, NG)
    v = vloc.ravel()
    out = []
    for c in psi:
        pr = ph @ c
        out.append(np.conj(ph).T @ (v * pr) / r.shape[0])
    return np.array(out)


@pytest.mark.parametrize("lat,k,ecut,grid", [
    (np.diag([4.0, 5.0, 6.0]), np.array([0.1, -0.2, 0.05]), 4.0, (5, 6, 9)),
    (np.array([[5.0, 0.0, 0.0], [1.0, 5.5, 0.0], [0.5, -0.7, 6.0]]),
     np.array([0.0, 0.13, -0.07]), 3.5, (7, 6, 8)),
])
def test_fft_route_matches_direct_dft(lat, k, ecut, grid):
    m, _, _ = oracle.gsphere(lat, k, ecut)
    oracle.check_grid(m, grid)
    rng = np.random.default_rng(5)
    vloc = rng.standard_normal((grid[2], grid[1], grid[0]))
    psi = qeinputs.random_vectors(3, len(m), seed=6)
    got = oracle.apply_local(lat, k, ecut, grid, vloc, psi)
    want = _direct_local(lat, k, ecut, grid, vloc, psi)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _vc_analytic(lat, tau, g, amp=-2.0, sigma=1.0):
    """Fourier coefficient of the periodic Gaussian potential:
    (amp / Omega) (2 pi sigma^2)^{3/2} e^{-sigma^2 g^2 / 2} sum_I e^{-i g.R_I}."""
    omega = abs(np.linalg.det(lat))
    g2 = np.sum(g * g, axis=-1)
    s = np.exp(-1j * (g @ np.asarray(tau).T)).sum(axis=-1)
    return amp / omega * (2 * math.pi * sigma ** 2) ** 1.5 * np.exp(-0.5 * sigma ** 2 * g2) * s


def test_single_plane_wave_gives_analytic_gaussian_coefficients():
    c = qeinputs.config("C0")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    m, _, q = oracle.gsphere(lat, k, ecut)
    vloc = oracle.vloc_gaussian(lat, grid, c["tau"])
    for i0 in (0, 5, 40, 700):
        psi = np.zeros((1, len(m)), dtype=complex)
        psi[0, i0] = 1.0
        got = oracle.apply_local(lat, k, ecut, grid, vloc, psi)[0]
        want = _vc_analytic(lat, c["tau"], q - q[i0][None, :])
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_vtilde_matches_analytic_on_orthorhombic_cell():
    lat = np.array([[9.0, 0.0, 0.0], [0.0, 10.0, 0.0], [0.0, 0.0, 11.0]])
    tau = np.array([[1.0, 2.0, 3.0], [6.0, 5.5, 8.0]])
    grid = (30, 32, 36)
    v = oracle.vloc_gaussian(lat, grid, tau)
    vt = oracle.vtilde(v)
    b = oracle.reciprocal(lat)
    for g in [(0, 0, 0), (1, 0, 0), (2, -3, 1), (-4, 4, 5), (3, 3, -3)]:
        gc = np.array(g) @ b
        want = _vc_analytic(lat, tau, gc[None, :])[0]
        got = vt[g[2] % grid[2], g[1] % grid[1], g[0] % grid[0]]
        assert abs(got - want) < 1e-15


@pytest.mark.parametrize("lat", [
    np.array([[10.0, 0.0, 0.0], [2.0, 10.0, 0.0], [1.0, -1.5, 11.0]]),
    np.array([[10.5, 0.7, -0.4], [-1.2, 9.8, 0.9], [0.6, 2.1, 10.2]]),
])
def test_vtilde_matches_analytic_on_skewed_cell(lat):
    """The general (27-image) branch of vloc_gaussian on skewed cells: its
    discrete Fourier coefficients equal the closed-form transform of the
    periodic Gaussian, (amp / Omega) (2 pi sigma^2)^{3/2} e^{-sigma^2 g^2 / 2}
    sum_I e^{-i g.R_I}, at Cartesian g = sum_i m_i b_i.  A lattice used by
    columns instead of rows (r or the images built from lat^T) moves the
    Gaussians and fails here.  Truncation of the image sum (next images at
    >= 9 bohr: e^{-40}) and grid aliasing (e^{-60}) are far below the bound."""
    tau = np.array([[1.0, 2.0, 3.0], [6.0, 5.5, 8.0], [8.5, 0.4, 1.2]])
    grid = (40, 40, 45)
    v = oracle.vloc_gaussian(lat, grid, tau)
    vt = oracle.vtilde(v)
    b = oracle.reciprocal(lat)
    for g in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, -3, 1), (-4, 4, 5), (3, 3, -3),
              (1, -1, 2), (-2, 0, -3)]:
        gc = np.array(g) @ b
        want = _vc_analytic(lat, tau, gc[None, :])[0]
        got = vt[g[2] % grid[2], g[1] % grid[1], g[0] % grid[0]]
        assert abs(got - want) < 1e-15


def test_vloc_general_and_factorised_forms_agree():
    lat = np.diag([8.0, 9.0, 10.0])
    tau = np.array([[0.5, 0.5, 0.5], [7.5, 8.0, 1.0]])
    grid = (16, 18, 20)
    v = oracle.vloc_gaussian(lat, grid, tau)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, n, 50) for n in grid], axis=1)
    vs = oracle.vloc_gaussian(lat, grid, tau, points=pts)
    np.testing.assert_allclose(v[pts[:, 2], pts[:, 1], pts[:, 0]], vs, rtol=1e-14, atol=1e-300)


def test_constant_potential_is_a_shift():
    c = qeinputs.config("SMALL")
    m, kin, _ = oracle.gsphere(c["lat"], c["k"], c["ecut"])
    psi = qeinputs.random_vectors(3, len(m), seed=1)
    v = np.full((c["grid"][2], c["grid"][1], c["grid"][0]), -0.75)
    got = oracle.apply_local(c["lat"], c["k"], c["ecut"], c["grid"], v, psi)
    np.testing.assert_allclose(got, -0.75 * psi, rtol=0, atol=1e-13)


def test_empty_lattice_is_kinetic_only():
    c = qeinputs.config("SMALL")
    m, kin, _ = oracle.gsphere(c["lat"], c["k"], c["ecut"])
    psi = qeinputs.random_vectors(2, len(m), seed=2)
    v = np.zeros((c["grid"][2], c["grid"][1], c["grid"][0]))
    beta = np.zeros((0, len(m)), dtype=complex)
    got = oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, np.zeros((0, 0)), psi)
    np.testing.assert_allclose(got, kin[None, :] * psi, rtol=1e-15, atol=0)


def _small_problem():
    c = qeinputs.config("SMALL")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    return lat, k, ecut, grid, v, beta, d


def test_hermiticity():
    lat, k, ecut, grid, v, beta, d = _small_problem()
    npw = beta.shape[1]
    x = qeinputs.random_vectors(4, npw, seed=3)
    hx = oracle.hpsi(lat, k, ecut, grid, v, beta, d, x)
    g = np.conj(x) @ hx.T                      # <x_i|H x_j>
    np.testing.assert_allclose(g, g.conj().T, rtol=0, atol=1e-13 * np.abs(g).max())


def test_dense_matrix_agrees_with_operator():
    lat, k, ecut, grid, v, beta, d = _small_problem()
    h = oracle.dense_h(lat, k, ecut, grid, v, beta, d)
    np.testing.assert_allclose(h, h.conj().T, rtol=0, atol=1e-14)
    x = qeinputs.random_vectors(3, h.shape[0], seed=4)
    np.testing.assert_allclose(oracle.hpsi(lat, k, ecut, grid, v, beta, d, x), x @ h.T,
                               rtol=0, atol=1e-12)


def test_preconditioner_diagonal_is_the_exact_diagonal_for_diagonal_d():
    """h_G = |k+G|^2 + mean V + sum_i D_ii |B_i(G)|^2 is the exact diagonal of H
    when D is diagonal: the local term's diagonal is V~(0) = mean V and the
    nonlocal one is sum_ij B_i D_ij conj(B_j) at G = G'."""
    lat, k, ecut, grid, v, beta, d = _small_problem()
    assert np.count_nonzero(d - np.diag(np.diag(d))) == 0
    _, kin, _ = oracle.gsphere(lat, k, ecut)
    h = oracle.dense_h(lat, k, ecut, grid, v, beta, d)
    np.testing.assert_allclose(oracle.h_diag(kin, v, beta, d), np.real(np.diag(h)), rtol=0,
                               atol=1e-13 * np.abs(h).max())
