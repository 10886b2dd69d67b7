"""Charge density of a set of bands over k points.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper lists charge-density generation among the kernels ported to the GPU
(Sec. 3.3) and electronic self-consistency among the accelerated
functionalities; it does not write the density down.  The standard plane-wave
definition (Rydberg units, bands normalised to sum_G |c_G|^2 = 1, so that the
Bloch function is Omega^{-1/2} sum_G c_G e^{i(k+G).r}):

    rho(r_j) = (1 / Omega) sum_k sum_n w_nk |psi_nk(r_j)|^2,
    psi_nk(r_j) = sum_G c_nk(G) e^{i G.r_j}        (the e^{ik.r} factor has modulus 1)

on the FFT grid r_j = sum_i (j_i / N_i) a_i, array [N3][N2][N1] (x fastest);
w_nk is the occupation times the k-point weight of band n at k.  Its integral
(Omega / N) sum_j rho(r_j) = sum_nk w_nk sum_G |c_nk(G)|^2 (Parseval), the
electron count for normalised bands.

Parity: pinned (Parseval charge, single and two plane waves in closed form,
direct O(N_G N_r) sum on tiny grids, translation by a grid vector).
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from .pw import gsphere, grid_slots, check_grid, volume


def band_in_r(lat, k, ecut, grid, c: np.ndarray) -> np.ndarray:
    """psi(r_j) = sum_G c_G e^{iG.r_j} on the grid, complex (N3, N2, N1)."""
    miller, _, _ = gsphere(lat, k, ecut)
    check_grid(miller, grid)
    s0, s1, s2 = grid_slots(miller, grid)
    n1, n2, n3 = grid
    a = np.zeros((n3, n2, n1), dtype=np.complex128)
    a[s2, s1, s0] = c
    # numpy's inverse transform carries 1/N: multiply it back out
    return scipy.fft.ifftn(a, workers=-1) * (n1 * n2 * n3)


def density(lat, ecut, grid, kpts, psis, weights) -> np.ndarray:
    """rho(r_j), float64 (N3, N2, N1).  kpts: (nk, 3) Cartesian; psis[i]: the
    bands (nb_i, npw_i) of k point i in its sphere's order; weights[i]: (nb_i,)."""
    n1, n2, n3 = grid
    rho = np.zeros((n3, n2, n1))
    for k, psi, w in zip(kpts, psis, weights):
        psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
        for c, wn in zip(psi, np.asarray(w, dtype=np.float64)):
            p = band_in_r(lat, k, ecut, grid, c)
            rho += wn * (p.real * p.real + p.imag * p.imag)
    return rho / volume(lat)
