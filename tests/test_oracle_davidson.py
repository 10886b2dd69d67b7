"""Pins of the oracle's Rayleigh-Ritz and block Davidson (Sec. 3.3: Davidson
iterative diagonalisation; Sec. 3.2.1: KS_Solvers and the dense generalized
eigensolver of LAXlib).

* Rayleigh-Ritz against SciPy's generalized Hermitian eigensolver;
* Davidson against the dense diagonalisation (LAPACK) of the C0 cell, against
  the empty-lattice closed form (integer sums of squares), against the rank-1
  secular equation solved by bracketing, and under exact symmetries (a constant
  potential shift; a rigid translation of all atoms by a grid vector).
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle
import qeinputs


def _problem(name, **over):
    c = dict(qeinputs.config(name))
    c.update(over)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    m, kin, _ = oracle.gsphere(lat, k, ecut)
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    return c, kin, v, beta, d


def _solve(c, kin, v, beta, d, tol=None, nb=None):
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    nb = c["nbnd"] if nb is None else nb
    psi0 = qeinputs.start_bands(kin, nb, c["psi_seed"])
    hd = oracle.h_diag(kin, v, beta, d)
    ah = lambda x: oracle.hpsi(lat, k, ecut, grid, v, beta, d, x)
    return oracle.davidson(ah, hd, psi0, c["tol"] if tol is None else tol)


def test_rayleigh_ritz_against_library():
    rng = np.random.default_rng(0)
    n = 24
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = a + a.conj().T
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    s = b @ b.conj().T + n * np.eye(n)
    e, x = oracle.rayleigh_ritz(h, s, 7)
    w = scipy.linalg.eigh(h, s, eigvals_only=True)
    np.testing.assert_allclose(e, w[:7], rtol=0, atol=1e-12)
    np.testing.assert_allclose(x.conj().T @ s @ x, np.eye(7), atol=1e-12)
    np.testing.assert_allclose(h @ x, s @ x * e[None, :], atol=1e-10)


def test_c0_davidson_matches_dense_diagonalisation():
    c, kin, v, beta, d = _problem("C0")
    h = oracle.dense_h(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d)
    w = np.linalg.eigvalsh(h)
    r = _solve(c, kin, v, beta, d)
    assert r["converged"] and np.all(r["resid"] <= c["tol"])
    np.testing.assert_allclose(r["e"], w[:c["nbnd"]], rtol=0, atol=1e-10)


def test_c0_empty_lattice_closed_form():
    c, kin, v, beta, d = _problem("C0")
    r = _solve(c, kin, np.zeros_like(v), beta[:0], d[:0, :0])
    unit = (2 * math.pi / 10.0) ** 2
    want = unit * np.array([0, 1, 1, 1, 1, 1, 1, 2], dtype=float)
    assert r["converged"]
    np.testing.assert_allclose(r["e"], want, rtol=0, atol=1e-10)


def test_constant_shift_of_the_potential():
    c, kin, v, beta, d = _problem("SMALL")
    r0 = _solve(c, kin, v, beta, d)
    r1 = _solve(c, kin, v + 0.37, beta, d)
    np.testing.assert_allclose(r1["e"], r0["e"] + 0.37, rtol=0, atol=1e-10)


def test_rank_one_secular_equation():
    a, ecut, dval = 8.0, 10.0, 0.5
    lat = qeinputs.cubic(a)
    m, kin, _ = oracle.gsphere(lat, np.zeros(3), ecut)
    beta = oracle.beta_gaussian(lat, np.zeros(3), ecut, np.array([[0.0, 0.0, 0.0]]), (1.0,))[:1]
    dm = np.array([[dval]])
    # shells by the integer norm m1^2+m2^2+m3^2 (exact degeneracy)
    n2 = (m ** 2).sum(axis=1)
    shells = np.unique(n2)
    kk = (2 * math.pi / a) ** 2 * shells.astype(float)
    wts = np.array([np.sum(np.abs(beta[0, n2 == s]) ** 2) for s in shells])
    mult = np.array([np.sum(n2 == s) for s in shells])
    f = lambda e: 1.0 - dval * np.sum(wts / (e - kk))
    eig = []
    for j in range(len(shells)):
        eig += [kk[j]] * int(mult[j] - 1)
        hi = kk[j + 1] if j + 1 < len(shells) else kk[j] + 10.0
        lo_b, hi_b = kk[j] + 1e-14 * (1 + kk[j]), hi - 1e-14 * (1 + hi)
        eig.append(scipy.optimize.brentq(f, lo_b, hi_b, xtol=1e-15, rtol=1e-15, maxiter=500))
    eig = np.sort(np.array(eig))
    grid = (16, 16, 16)
    v = np.zeros((16, 16, 16))
    h = oracle.dense_h(lat, np.zeros(3), ecut, grid, v, beta, dm)
    np.testing.assert_allclose(np.linalg.eigvalsh(h)[:20], eig[:20], rtol=0, atol=1e-12)
    ah = lambda x: oracle.hpsi(lat, np.zeros(3), ecut, grid, v, beta, dm, x)
    r = oracle.davidson(ah, oracle.h_diag(kin, v, beta, dm), qeinputs.start_bands(kin, 5, 1), 1e-9)
    assert r["converged"]
    np.testing.assert_allclose(r["e"], eig[:5], rtol=0, atol=1e-10)


def test_translation_by_a_grid_vector_keeps_eigenvalues():
    c, kin, v, beta, d = _problem("SMALL")
    lat, grid = c["lat"], c["grid"]
    shift = 3 * lat[0] / grid[0] - 2 * lat[2] / grid[2]
    c2 = dict(c)
    c2["tau"] = c["tau"] + shift[None, :]
    v2 = oracle.vloc_gaussian(lat, grid, c2["tau"])
    beta2 = oracle.beta_gaussian(lat, c["k"], c["ecut"], c2["tau"], c["widths"])
    h1 = oracle.dense_h(lat, c["k"], c["ecut"], grid, v, beta, d)
    h2 = oracle.dense_h(lat, c["k"], c["ecut"], grid, v2, beta2, d)
    np.testing.assert_allclose(np.linalg.eigvalsh(h1), np.linalg.eigvalsh(h2), rtol=0, atol=1e-12)
    # and the operator is the same up to the diagonal phase e^{-i(k+G).t}
    _, _, q = oracle.gsphere(lat, c["k"], c["ecut"])
    u = np.exp(-1j * (q @ shift))
    np.testing.assert_allclose(h2, u[:, None] * h1 * np.conj(u)[None, :], rtol=0, atol=1e-12)


def test_variational_in_the_cutoff():
    # nested bases at a fixed grid: eigenvalues cannot go up when ecut grows
    c, kin, v, beta, d = _problem("SMALL")
    prev = None
    for ecut in (8.0, 10.0, 12.0):
        b = oracle.beta_gaussian(c["lat"], c["k"], ecut, c["tau"], c["widths"])
        h = oracle.dense_h(c["lat"], c["k"], ecut, c["grid"], v, b, d)
        w = np.linalg.eigvalsh(h)[:6]
        if prev is not None:
            assert np.all(w <= prev + 1e-12)
        prev = w


def test_nonconvergence_is_reported():
    c, kin, v, beta, d = _problem("SMALL")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    ah = lambda x: oracle.hpsi(lat, k, ecut, grid, v, beta, d, x)
    r = oracle.davidson(ah, oracle.h_diag(kin, v, beta, d),
                        qeinputs.start_bands(kin, 4, 0), 1e-12, max_iter=1)
    assert not r["converged"] and r["iters"] == 1
