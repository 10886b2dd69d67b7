"""Rayleigh-Ritz and the block Davidson eigensolver.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper names the Davidson method as one of the iterative Kohn-Sham solvers
(Sec. 3.3; KS_Solvers in Sec. 3.2.1) and the dense generalized eigenproblem
of the reduced matrices (LAXlib, Sec. 3.2.1), without writing either down.  The
steps below are the textbook block Davidson (Davidson 1975; Liu 1978):

1. Start from the given bands (any full-rank block: S_r handles a
   non-orthonormal start); after the first Rayleigh-Ritz the basis V is the
   set of Ritz vectors, which is orthonormal.
2. Rayleigh-Ritz on span(V): H_r = V^+ H V, S_r = V^+ V; Cholesky S_r = L L^+;
   eigen-decomposition of L^-1 H_r L^-+; X = L^-+ Y; keep the nb lowest pairs;
   Ritz vectors Psi = V X, H Psi = (HV) X.
3. Residuals r_n = H psi_n - e_n psi_n (||psi_n|| = 1); band n is converged when
   ||r_n||_2 <= tol.  Stop when every band is converged (or after max_iter).
4. Corrections for unconverged bands: delta_n(G) = r_n(G) / p(h_G - e_n) with
   the positive preconditioner p(x) = sqrt(x^2 + pmin^2), pmin = 0.1 Ry.  (A
   sign-keeping p(x) = x for |x| >= pmin is the exact inverse of H - e on a
   diagonal H, so on the empty lattice it returns the Ritz vector itself and the
   basis stops growing.)
5. If dim(V) + #corrections > max_dim, V collapses to the current Ritz vectors.
6. The corrections are orthonormalised against V and among themselves
   (Gram-Schmidt, two passes); one left with norm below ``drop`` is dropped.
   Without this step a preconditioner that is exact on the diagonal (the empty
   lattice) returns corrections inside span(V) and S_r turns singular.
   Append the corrections (and their H products) to V and go to 2.  If no
   correction survives, the basis cannot grow: stop (not converged).

Parity: pinned (Rayleigh-Ritz against library generalized eigensolvers on
random Hermitian / HPD pairs; Davidson against the dense diagonalisation and
against the closed forms of the empty lattice and the rank-1 secular equation).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def rayleigh_ritz(hred: np.ndarray, sred: np.ndarray, nev: int):
    """Lowest ``nev`` eigenpairs of the pencil (hred, sred): returns (e, X) with
    X^+ sred X = I, columns of X the eigenvectors."""
    L = scipy.linalg.cholesky(sred, lower=True)
    z = scipy.linalg.solve_triangular(L, hred, lower=True)                  # L^-1 H
    a = scipy.linalg.solve_triangular(L, z.conj().T, lower=True).conj().T   # L^-1 H L^-+
    a = 0.5 * (a + a.conj().T)
    w, y = np.linalg.eigh(a)
    x = scipy.linalg.solve_triangular(L.conj().T, y[:, :nev], lower=False)
    return w[:nev], x


def precondition(resid: np.ndarray, hdiag: np.ndarray, e: np.ndarray, pmin: float):
    """delta_n(G) = r_n(G) / sqrt((h_G - e_n)^2 + pmin^2)."""
    x = hdiag[None, :] - e[:, None]
    return resid / np.sqrt(x * x + pmin * pmin)


def orthonormalize_against(v: np.ndarray, delta: np.ndarray, drop: float) -> np.ndarray:
    """Classical Gram-Schmidt, each vector projected twice: normalise delta_j,
    remove its components along the rows of ``v`` (orthonormal) and along the
    corrections already accepted, renormalise; a correction whose norm after
    projection is below ``drop`` adds no new direction and is dropped."""
    out = []
    for d in delta:
        d = d / np.linalg.norm(d)
        for _ in range(2):
            d = d - (np.conj(v) @ d) @ v
            for a in out:
                d = d - np.vdot(a, d) * a
        nrm = np.linalg.norm(d)
        if nrm > drop:
            out.append(d / nrm)
    return np.array(out, dtype=np.complex128).reshape(-1, delta.shape[1])


def davidson(apply_h, hdiag: np.ndarray, psi0: np.ndarray, tol: float,
             max_iter: int = 100, max_dim: int | None = None, pmin: float = 0.1,
             drop: float = 1e-10):
    """Block Davidson.  ``apply_h`` maps a block (m, npw) to H times it.

    Returns a dict: e (nb,), psi (nb, npw), resid (nb,), iters, converged.
    """
    psi0 = np.atleast_2d(np.asarray(psi0, dtype=np.complex128))
    nb = psi0.shape[0]
    max_dim = 4 * nb if max_dim is None else max_dim
    v = psi0.copy()
    hv = apply_h(v)
    it = 0
    first = True
    while True:
        sred = np.conj(v) @ v.T
        hred = np.conj(v) @ hv.T
        e, x = rayleigh_ritz(hred, sred, nb)
        psi = x.T @ v
        hpsi = x.T @ hv
        if it == 0 and first:
            # the Ritz vectors of the start block become the (orthonormal) basis
            v, hv, first = psi, hpsi, False
        r = hpsi - e[:, None] * psi
        rn = np.linalg.norm(r, axis=1)
        conv = rn <= tol
        if conv.all() or it >= max_iter:
            break
        it += 1
        unc = np.nonzero(~conv)[0]
        delta = precondition(r[unc], hdiag, e[unc], pmin)
        if v.shape[0] + delta.shape[0] > max_dim:
            v, hv = psi, hpsi
        delta = orthonormalize_against(v, delta, drop)
        if delta.shape[0] == 0:
            break
        v = np.vstack([v, delta])
        hv = np.vstack([hv, apply_h(delta)])
    return dict(e=e, psi=psi, resid=rn, iters=it, converged=bool(conv.all()))
