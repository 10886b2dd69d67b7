"""Pins of the oracle's projector coefficients and nonlocal term (Sec. 3.2.2
item (viii), pseudopotential terms; Sec. 3.3, pseudopotential contribution).

* B_i(G) against a direct real-space quadrature of <k+G|beta_i> written from
  the real-space definition of the projector (catches phase, (-i)^l, axis and
  normalisation mistakes);
* Parseval: sum_G |B_i(G)|^2 = ||beta_i||^2 = 1 once the cut-off tail and the
  overlap with periodic images are below double precision;
* orthogonality of s and p projectors on one atom.
"""
import math

import numpy as np
import pytest

import oracle
import qeinputs


def _beta_real(r, w, l, ax):
    r2 = np.sum(r * r, axis=-1)
    g = np.exp(-r2 / (2 * w * w))
    if l == 0:
        n0 = math.sqrt(4.0 / (math.sqrt(math.pi) * w ** 3))
        return n0 / (2 * math.sqrt(math.pi)) * g
    n1 = math.sqrt(8.0 / (3.0 * math.sqrt(math.pi) * w ** 5))
    return n1 * math.sqrt(3 / (4 * math.pi)) * r[..., ax] * g


def test_coefficients_match_real_space_quadrature():
    lat = np.diag([9.0, 10.0, 11.0])
    k = np.array([0.07, -0.05, 0.11])
    tau = np.array([[2.0, 3.0, 4.5]])
    widths = (1.0, 0.7)
    beta = oracle.beta_gaussian(lat, k, 8.0, tau, widths)
    _, _, q = oracle.gsphere(lat, k, 8.0)
    omega = abs(np.linalg.det(lat))
    h = 0.14
    x = np.arange(-7.0, 7.0 + 1e-9, h)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    rel = np.stack([X, Y, Z], axis=-1)            # r - R
    for gi in (0, 3, 17, 60, len(q) - 1):
        qq = q[gi]
        ph = np.exp(-1j * (rel @ qq)) * np.exp(-1j * (qq @ tau[0]))
        col = 0
        for w in widths:
            for l, ax in ((0, 0), (1, 0), (1, 1), (1, 2)):
                f = _beta_real(rel, w, l, ax)
                want = (f * ph).sum() * h ** 3 / math.sqrt(omega)
                assert abs(beta[col, gi] - want) < 1e-11, (gi, col)
                col += 1


@pytest.mark.parametrize("w,ecut", [(1.0, 45.0), (0.7, 90.0)])
def test_parseval_unit_norm(w, ecut):
    lat = qeinputs.cubic(14.0)
    tau = np.array([[3.0, 4.0, 5.0]])
    beta = oracle.beta_gaussian(lat, np.zeros(3), ecut, tau, (w,))
    norms = np.sum(np.abs(beta) ** 2, axis=1)
    np.testing.assert_allclose(norms, np.ones(4), rtol=0, atol=1e-13)
    gram = np.conj(beta) @ beta.T
    np.testing.assert_allclose(gram, np.eye(4), rtol=0, atol=1e-13)


def test_parseval_with_gaussian_tail():
    # s projector: the missing weight beyond the cut-off is the closed-form
    # radial tail of |beta~(q)|^2 ~ exp(-w^2 q^2):
    #   1 - tail = erf(w Q) - (2/sqrt(pi)) w Q exp(-w^2 Q^2),  Q = sqrt(ecut)
    lat = qeinputs.cubic(14.0)
    w, ecut = 1.0, 12.0
    beta = oracle.beta_gaussian(lat, np.zeros(3), ecut, np.array([[1.0, 2.0, 3.0]]), (w,))
    got = np.sum(np.abs(beta[0]) ** 2)
    Q = math.sqrt(ecut)
    want = math.erf(w * Q) - 2 / math.sqrt(math.pi) * w * Q * math.exp(-(w * Q) ** 2)
    # the lattice sum over a truncated sphere differs from the integral by a
    # boundary term of the size of the integrand at the cut-off
    tail = 1.0 - want
    assert tail > 1e-5 and abs(got - want) < 0.1 * tail


def test_nonlocal_rank_structure():
    c = qeinputs.config("SMALL")
    beta = oracle.beta_gaussian(c["lat"], c["k"], c["ecut"], c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    psi = qeinputs.random_vectors(3, beta.shape[1], seed=9)
    got = oracle.apply_nonlocal(beta, d, psi)
    # the explicit triple sum of the definition, band by band
    want = np.zeros_like(psi)
    for n in range(psi.shape[0]):
        for i in range(beta.shape[0]):
            for j in range(beta.shape[0]):
                if d[i, j] != 0.0:
                    want[n] += beta[i] * d[i, j] * np.vdot(beta[j], psi[n])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
