"""The Kohn-Sham operator H = T + V_loc + V_NL on a block of bands.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper lists the kinetic-energy, local-potential and pseudopotential
contributions to the Hamiltonian among the GPU kernels (Sec. 3.3) and the
3D FFT library that the local term uses (Sec. 3.2.1, FFTXlib).  Definitions
(Rydberg units, plane-wave coefficients c_G in the order of ``pw.gsphere``):

* kinetic:   (T c)_G = |k+G|^2 c_G
* local:     psi(r_j) = sum_G c_G e^{i G.r_j}  (unnormalised inverse DFT on the grid),
             (V c)_G  = (1/N) sum_j e^{-i G.r_j} V(r_j) psi(r_j),  N = N1 N2 N3
             equivalently V_{GG'} = Vt((G - G') mod grid), Vt(g) = (1/N) sum_j V(r_j) e^{-i g.r_j}
* nonlocal:  (V_NL c)_G = sum_{ij} B_i(G) D_ij sum_G' conj(B_j(G')) c_G'

Blocks are arrays (nbnd, npw) complex128, one band per row.

Parity: pinned (empty lattice, constant potential, single plane wave against the
analytic Gaussian transform, direct DFT on tiny grids, Hermiticity, dense H).
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from .pw import gsphere, grid_slots, check_grid


def _slots(lat, k, ecut, grid):
    miller, kin, _ = gsphere(lat, k, ecut)
    check_grid(miller, grid)
    s0, s1, s2 = grid_slots(miller, grid)
    return kin, (s2, s1, s0)   # array index order [z][y][x]


def apply_kinetic(kin: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return kin[None, :] * psi


def apply_local(lat, k, ecut, grid, vloc: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(V_loc psi) through full-grid FFTs, one band at a time."""
    _, idx = _slots(lat, k, ecut, grid)
    n1, n2, n3 = grid
    ntot = n1 * n2 * n3
    out = np.empty_like(psi)
    for b in range(psi.shape[0]):
        a = np.zeros((n3, n2, n1), dtype=np.complex128)
        a[idx] = psi[b]
        # numpy's inverse transform carries 1/N; multiply it back out to get the
        # plain sum_G c_G e^{+iG.r}
        pr = scipy.fft.ifftn(a, workers=-1) * ntot
        f = scipy.fft.fftn(vloc * pr, workers=-1)
        out[b] = f[idx] / ntot
    return out


def apply_nonlocal(beta: np.ndarray, dmat: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """V_NL psi = B^T D (conj(B) psi^T) in the (band, G) layout."""
    if beta.shape[0] == 0:
        return np.zeros_like(psi)
    p = np.conj(beta) @ psi.T          # (nproj, nbnd): <beta_i|psi_n>
    q = dmat @ p                        # (nproj, nbnd)
    return (beta.T @ q).T               # (nbnd, npw)


def hpsi(lat, k, ecut, grid, vloc, beta, dmat, psi) -> np.ndarray:
    """H psi for a block psi (nbnd, npw)."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    kin, _ = _slots(lat, k, ecut, grid)
    return (apply_kinetic(kin, psi) + apply_local(lat, k, ecut, grid, vloc, psi)
            + apply_nonlocal(beta, dmat, psi))


def vtilde(vloc: np.ndarray) -> np.ndarray:
    """Vt(g) = (1/N) sum_j V(r_j) e^{-i g.r_j} on the grid, array [g2][g1][g0]."""
    return scipy.fft.fftn(vloc, workers=-1) / vloc.size


def dense_h(lat, k, ecut, grid, vloc, beta, dmat) -> np.ndarray:
    """The full Hermitian matrix H_{GG'} (npw, npw), built element-wise from the
    definition (no FFT of wavefunctions)."""
    miller, kin, _ = gsphere(lat, k, ecut)
    check_grid(miller, grid)
    vt = vtilde(vloc)
    d = miller[:, None, :] - miller[None, :, :]
    h = vt[np.mod(d[..., 2], grid[2]), np.mod(d[..., 1], grid[1]), np.mod(d[..., 0], grid[0])]
    h = h + np.diag(kin)
    if beta.shape[0]:
        h = h + beta.T @ dmat @ np.conj(beta)
    return h


def h_diag(kin: np.ndarray, vloc: np.ndarray, beta: np.ndarray, dmat: np.ndarray) -> np.ndarray:
    """Diagonal estimate used by the Davidson preconditioner:
    h_G = |k+G|^2 + mean(V) + sum_i D_ii |B_i(G)|^2."""
    h = kin + float(np.mean(vloc))
    if beta.shape[0]:
        h = h + np.einsum("i,ig->g", np.diag(dmat), np.abs(beta) ** 2)
    return h
