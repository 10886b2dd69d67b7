"""One self-consistency step of the local potential from the bands.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper lists electronic self-consistency and charge-density generation among
the GPU-accelerated functionalities (Sec. 3.3) without writing them down.  The
step below is the textbook density-mixing update of a local potential
(Rydberg units, e^2 = 2):

1. rho(r) from the bands (density.py);
2. Hartree potential on the density sphere |G|^2 <= 4 ecutwfc (the sphere on
   which a density built from bands of cut-off ecutwfc has its coefficients):
       rho~(G) = (1/N) sum_j rho(r_j) e^{-iG.r_j},
       V_H(r_j) = sum_{G != 0} 8 pi rho~(G) / |G|^2 e^{iG.r_j}   (G = 0 dropped:
       the neutralising background);
3. exchange of the homogeneous electron gas (Slater, LDA):
       v_x(r) = -2 (3 rho(r) / pi)^{1/3};
4. V_out = V_ext + V_H + v_x and the linear mixing
       V_new = (1 - alpha) V_in + alpha V_out.

Parity: pinned (a cosine density has the closed-form Hartree potential
8 pi A cos(g.r) / |g|^2; a direct O(N_G N_r) sum on a tiny grid; the exchange
formula's scaling v_x(8 rho) = 2 v_x(rho); the mixing end points; the zero mean
of V_H).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

from .pw import gsphere, grid_slots, check_grid
from .density import density


def hartree(lat, ecut_rho, grid, rho: np.ndarray) -> np.ndarray:
    """V_H(r_j) of the density on the sphere |G|^2 <= ecut_rho, float64 (N3, N2, N1)."""
    miller, kin, _ = gsphere(lat, np.zeros(3), ecut_rho)
    check_grid(miller, grid)
    s0, s1, s2 = grid_slots(miller, grid)
    n = rho.size
    rg = scipy.fft.fftn(rho, workers=-1)[s2, s1, s0] / n        # rho~(G) on the sphere
    vg = np.zeros_like(rg)
    nz = kin > 0.0
    vg[nz] = 8.0 * math.pi * rg[nz] / kin[nz]
    a = np.zeros(rho.shape, dtype=np.complex128)
    a[s2, s1, s0] = vg
    return np.real(scipy.fft.ifftn(a, workers=-1) * n)


def exchange(rho: np.ndarray) -> np.ndarray:
    """v_x(r) = -2 (3 rho / pi)^{1/3} (Ry), rho >= 0."""
    return -2.0 * np.cbrt(3.0 * np.maximum(rho, 0.0) / math.pi)


def scf_step(lat, ecut, grid, kpts, psis, weights, vext, vin, alpha: float):
    """(V_new, rho) of one step from the bands of the k points (see the header)."""
    rho = density(lat, ecut, grid, kpts, psis, weights)
    vout = vext + hartree(lat, 4.0 * ecut, grid, rho) + exchange(rho)
    return (1.0 - alpha) * vin + alpha * vout, rho
