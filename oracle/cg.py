"""Band-by-band conjugate-gradient eigensolver.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper names the conjugate-gradient method beside Davidson as the iterative
solvers of the Kohn-Sham Hamiltonian that run on the GPU (Sec. 3.3) without
writing it down.  The steps below are the textbook band-by-band scheme of
direct minimisation (Teter, Payne and Allan 1989; Payne et al., Rev. Mod. Phys.
64, 1045 (1992), Sec. V): each band minimises the Rayleigh quotient in the
complement of the bands below it, along preconditioned conjugate directions,
with an exact line minimisation on the unit sphere.

1. Start: Rayleigh-Ritz of the start block; its Ritz vectors are orthonormal.
2. For n = 0 .. nb-1, from psi = psi_n made orthogonal to the current
   psi_0..n-1 (the bands below moved in their own minimisations) and
   normalised, H psi updated by the same combination of the stored H psi_m:
   a. e = <psi|H|psi>, gradient g = H psi - e psi; stop this band when ||g|| <= tol
      or after max_iter iterations of this sweep;
   b. preconditioned gradient z = g / sqrt((h_G - e)^2 + pmin^2) (the Davidson
      preconditioner of eigen.py), projected out of span(psi_0..n-1, psi);
   c. direction d = z + beta d_prev with the Polak-Ribiere coefficient
      beta = max(0, <z, g - g_prev> / <z_prev, g_prev>) (restart when negative),
      then projected out of span(psi_0..n-1, psi) and normalised: d^;
   d. exact minimum of E(t) = <p(t)|H|p(t)>, p(t) = cos t psi + sin t d^:
      with a = e, b = Re<psi|H d^>, c = <d^|H|d^>, t = atan2(-2b, c - a) / 2;
   e. psi <- cos t psi + sin t d^, H psi <- cos t H psi + sin t H d^.
3. Rayleigh-Ritz of span(psi_0..nb-1) (a subspace rotation): eigenvalues,
   rotated bands, residual norms ||H psi_n - e_n psi_n||.
4. Repeat 2-3 (a sweep) until every residual is <= tol, or max_sweeps.

Parity: pinned (dense diagonalisation of C0 and SMALL, empty lattice in closed
form, constant potential shift; see tests/test_oracle_cg.py).
"""
from __future__ import annotations

import math

import numpy as np

from .eigen import rayleigh_ritz, precondition


def _project_out(x, lower, p):
    """x minus its components along the orthonormal rows of `lower` and along p."""
    if lower.shape[0]:
        x = x - (np.conj(lower) @ x) @ lower
    return x - np.vdot(p, x) * p


def cg(apply_h, hdiag: np.ndarray, psi0: np.ndarray, tol: float, max_iter: int = 100,
       max_sweeps: int = 20, pmin: float = 0.1):
    """Band-by-band CG.  ``apply_h`` maps a block (m, npw) to H times it.

    Returns a dict: e (nb,), psi (nb, npw), resid (nb,), iters (CG iterations,
    i.e. H applications to search directions, summed over bands and sweeps),
    sweeps, converged."""
    psi0 = np.atleast_2d(np.asarray(psi0, dtype=np.complex128))
    nb = psi0.shape[0]
    hv = apply_h(psi0)
    e, x = rayleigh_ritz(np.conj(psi0) @ hv.T, np.conj(psi0) @ psi0.T, nb)
    psi = x.T @ psi0
    hpsi = x.T @ hv
    iters = 0
    sweeps = 0
    while True:
        r = hpsi - e[:, None] * psi
        rn = np.linalg.norm(r, axis=1)
        if (rn <= tol).all() or sweeps >= max_sweeps:
            break
        sweeps += 1
        for n in range(nb):
            lower = psi[:n]
            p, hp = psi[n].copy(), hpsi[n].copy()
            if n:
                coef = np.conj(lower) @ p
                p = p - coef @ lower
                hp = hp - coef @ hpsi[:n]
                nrm = np.linalg.norm(p)
                p, hp = p / nrm, hp / nrm
            d_prev = g_prev = z_prev = None
            for _ in range(max_iter):
                en = float(np.real(np.vdot(p, hp)))
                g = hp - en * p
                if np.linalg.norm(g) <= tol:
                    break
                z = _project_out(precondition(g[None, :], hdiag, np.array([en]), pmin)[0], lower, p)
                if d_prev is None:
                    d = z
                else:
                    beta = float(np.real(np.vdot(z, g - g_prev)) / np.real(np.vdot(z_prev, g_prev)))
                    d = z + max(beta, 0.0) * d_prev
                d = _project_out(d, lower, p)
                dn = d / np.linalg.norm(d)
                hd = apply_h(dn[None, :])[0]
                iters += 1
                b = float(np.real(np.vdot(p, hd)))
                c = float(np.real(np.vdot(dn, hd)))
                t = 0.5 * math.atan2(-2.0 * b, c - en)
                ct, st = math.cos(t), math.sin(t)
                p = ct * p + st * dn
                hp = ct * hp + st * hd
                d_prev, g_prev, z_prev = d, g, z
            psi[n], hpsi[n] = p, hp
        e, x = rayleigh_ritz(np.conj(psi) @ hpsi.T, np.conj(psi) @ psi.T, nb)
        psi = x.T @ psi
        hpsi = x.T @ hpsi
    return dict(e=e, psi=psi, resid=rn, iters=iters, sweeps=sweeps, converged=bool((rn <= tol).all()))
