"""Pins of the oracle's band-by-band conjugate-gradient eigensolver (Sec. 3.3:
iterative solution of the Kohn-Sham Hamiltonian with the conjugate-gradient
method), the same as the Davidson pins: the dense diagonalisation (LAPACK) of
the C0 and SMALL cells, the empty-lattice closed form, a constant potential
shift, orthonormal returned bands with residuals within tol, and reported
non-convergence.  The line minimisation is checked on its own against a dense
scan of the Rayleigh quotient on the great circle it searches."""
import math

import numpy as np

import oracle
import qeinputs


def _problem(name):
    c = qeinputs.config(name)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    _, kin, _ = oracle.gsphere(lat, k, ecut)
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    return c, kin, v, beta, d


def _cg(c, kin, v, beta, d, tol, **kw):
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    ah = lambda x: oracle.hpsi(lat, k, ecut, grid, v, beta, d, x)
    psi0 = qeinputs.start_bands(kin, c["nbnd"], c["psi_seed"])
    return oracle.cg(ah, oracle.h_diag(kin, v, beta, d), psi0, tol, **kw)


def test_c0_cg_matches_dense_diagonalisation():
    c, kin, v, beta, d = _problem("C0")
    h = oracle.dense_h(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d)
    w = np.linalg.eigvalsh(h)[:c["nbnd"]]
    r = _cg(c, kin, v, beta, d, 1e-8)
    assert r["converged"] and np.all(r["resid"] <= 1e-8)
    np.testing.assert_allclose(r["e"], w, rtol=0, atol=1e-10)
    x = r["psi"]
    np.testing.assert_allclose(np.conj(x) @ x.T, np.eye(c["nbnd"]), atol=1e-12)


def test_small_cg_matches_dense_and_constant_shift():
    c, kin, v, beta, d = _problem("SMALL")
    h = oracle.dense_h(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d)
    w = np.linalg.eigvalsh(h)[:c["nbnd"]]
    r0 = _cg(c, kin, v, beta, d, 1e-8)
    assert r0["converged"]
    np.testing.assert_allclose(r0["e"], w, rtol=0, atol=1e-10)
    r1 = _cg(c, kin, v + 0.37, beta, d, 1e-8)
    np.testing.assert_allclose(r1["e"], w + 0.37, rtol=0, atol=1e-10)


def test_empty_lattice_closed_form():
    c, kin, v, beta, d = _problem("C0")
    r = _cg(c, kin, np.zeros_like(v), beta[:0], d[:0, :0], 1e-8)
    unit = (2 * math.pi / 10.0) ** 2
    want = unit * np.array([0, 1, 1, 1, 1, 1, 1, 2], dtype=float)
    assert r["converged"]
    np.testing.assert_allclose(r["e"], want, rtol=0, atol=1e-10)


def test_line_minimisation_angle():
    """t = atan2(-2b, c - a) / 2 minimises E(t) = a cos^2 t + 2 b sin t cos t +
    c sin^2 t over a dense scan of the circle."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, b, c = rng.standard_normal(3)
        t = 0.5 * math.atan2(-2 * b, c - a)
        e = lambda s: a * np.cos(s) ** 2 + 2 * b * np.sin(s) * np.cos(s) + c * np.sin(s) ** 2
        scan = np.linspace(-math.pi, math.pi, 200001)
        assert e(t) <= e(scan).min() + 1e-9


def test_nonconvergence_is_reported():
    c, kin, v, beta, d = _problem("SMALL")
    r = _cg(c, kin, v, beta, d, 1e-12, max_iter=2, max_sweeps=1)
    assert not r["converged"] and r["sweeps"] == 1
