"""Plane-wave set-up: lattices, the G-sphere, grid slots, V_loc(r), beta(G).

TEST INFRASTRUCTURE ONLY (see the package header).

Follows Sec. 3.2.2 of the paper ("Modules"): (iii) Bravais and reciprocal
lattices, (vi) generation of plane waves and of their mapping to FFT grids,
(viii) calculation of pseudopotential terms.  The paper names these steps but
does not write them down; the definitions used are the standard ones:

* reciprocal vectors b_i = 2 pi (a_j x a_k) / Omega, Omega = a_1 . (a_2 x a_3)
* sphere S_k = { m in Z^3 : |k + G_m|^2 <= ecut }, G_m = sum_i m_i b_i (Ry units)
* grid point r_j = sum_i (j_i / N_i) a_i, Miller index m sits at slot m_i mod N_i
* V_loc(r) = AMP * sum_I sum_{T in {-1,0,1}^3} exp(-|r - R_I - T.lat|^2 / (2 sigma^2))
* beta_{I,n,l,m}(r) = N_{n,l} S_lm(r - R_I) exp(-|r - R_I|^2 / (2 w_n^2)), with
  S_lm the real solid harmonics (Y_00, and sqrt(3/4pi) (x, y, z)), unit L2 norm;
  its plane-wave coefficient is the closed-form Fourier transform
  <k+G|beta> = Omega^-1/2 e^{-i q.R} N (-i)^l (2pi)^{3/2} w^{2l+3} S_lm(q) e^{-w^2 q^2/2}.

Plane-wave order (a reading: the paper does not fix one): ascending |k+G|^2,
ties by (m1, m2, m3) lexicographically.  Because the order is decided by a
floating-point value, the value is defined by this exact float64 evaluation
with every operation rounded separately (no fused multiply-add):
    q_c = ((k_c + m1*b1_c) + m2*b2_c) + m3*b3_c,   |q|^2 = (qx*qx + qy*qy) + qz*qz
and the sphere test is |q|^2 <= ecut * (1 + 1e-12).

Parity: pinned (sphere counts by brute force and symmetry; beta by quadrature and
Parseval; V_loc through the analytic Fourier transform of the Gaussian).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _cross(u, v):
    return (u[1] * v[2] - u[2] * v[1],
            u[2] * v[0] - u[0] * v[2],
            u[0] * v[1] - u[1] * v[0])


def volume(lat) -> float:
    """Omega = |a1 . (a2 x a3)| (bohr^3)."""
    a = [[float(x) for x in row] for row in np.asarray(lat)]
    c = _cross(a[1], a[2])
    return abs((a[0][0] * c[0] + a[0][1] * c[1]) + a[0][2] * c[2])


def reciprocal(lat) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij, b1 = (a2 x a3) * (2 pi / vol)."""
    a = [[float(x) for x in row] for row in np.asarray(lat)]
    c1 = _cross(a[1], a[2])
    c2 = _cross(a[2], a[0])
    c3 = _cross(a[0], a[1])
    vol = (a[0][0] * c1[0] + a[0][1] * c1[1]) + a[0][2] * c1[2]
    fac = TWO_PI / vol
    return np.array([[x * fac for x in c] for c in (c1, c2, c3)], dtype=np.float64)


def _kin_of(miller: np.ndarray, k, b: np.ndarray):
    m1 = miller[:, 0].astype(np.float64)
    m2 = miller[:, 1].astype(np.float64)
    m3 = miller[:, 2].astype(np.float64)
    q = []
    for c in range(3):
        q.append(((float(k[c]) + m1 * b[0, c]) + m2 * b[1, c]) + m3 * b[2, c])
    kin = (q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]
    return np.stack(q, axis=1), kin


def gsphere(lat, k, ecut: float):
    """Return (miller int64 (npw,3), kin float64 (npw,), q float64 (npw,3)).

    Brute-force enumeration over a box that contains the sphere, then the
    order described in the module header.
    """
    lat = np.asarray(lat, dtype=np.float64)
    b = reciprocal(lat)
    kn = float(np.linalg.norm(np.asarray(k, dtype=np.float64)))
    gmax = math.sqrt(ecut) + kn
    lim = [int(math.floor(gmax * float(np.linalg.norm(lat[i])) / TWO_PI)) + 1
           for i in range(3)]
    r = [np.arange(-l, l + 1) for l in lim]
    mm = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    q, kin = _kin_of(mm, k, b)
    inside = kin <= ecut * (1.0 + 1e-12)
    mm, kin, q = mm[inside], kin[inside], q[inside]
    order = np.lexsort((mm[:, 2], mm[:, 1], mm[:, 0], kin))
    return mm[order].astype(np.int64), kin[order], q[order]


def check_grid(miller: np.ndarray, grid) -> None:
    """Raise ValueError unless N_i >= 2 max|m_i| + 1 for every axis (the sphere
    must not wrap onto itself on the grid)."""
    for i in range(3):
        need = 2 * int(np.abs(miller[:, i]).max(initial=0)) + 1
        if grid[i] < need:
            raise ValueError(f"grid axis {i}: {grid[i]} < {need}")


def grid_slots(miller: np.ndarray, grid):
    """Slot (i0, i1, i2) = (m_i mod N_i) of every plane wave on the FFT grid."""
    return tuple(np.mod(miller[:, i], grid[i]) for i in range(3))


def grid_points(lat, grid) -> np.ndarray:
    """Cartesian r_j, array (N3, N2, N1, 3), x (axis 0 of the grid) fastest."""
    lat = np.asarray(lat, dtype=np.float64)
    n1, n2, n3 = grid
    f0 = np.arange(n1) / n1
    f1 = np.arange(n2) / n2
    f2 = np.arange(n3) / n3
    F2, F1, F0 = np.meshgrid(f2, f1, f0, indexing="ij")
    return (F0[..., None] * lat[0] + F1[..., None] * lat[1] + F2[..., None] * lat[2])


def vloc_gaussian(lat, grid, tau, amp: float = -2.0, sigma: float = 1.0,
                  points: np.ndarray | None = None) -> np.ndarray:
    """V_loc sampled on the grid, float64 (N3, N2, N1), Ry.

    Sum over atoms and the 27 nearest periodic images of a Gaussian.  With
    ``points`` (an int array (n, 3) of grid indices (j0, j1, j2)), only those
    samples are returned, as a 1-D array.
    """
    lat = np.asarray(lat, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64).reshape(-1, 3)
    if points is None:
        r = grid_points(lat, grid)
    else:
        p = np.asarray(points)
        f = p / np.asarray(grid, dtype=np.float64)[None, :]
        r = f[:, 0:1] * lat[0] + f[:, 1:2] * lat[1] + f[:, 2:3] * lat[2]
    diag = np.allclose(lat, np.diag(np.diag(lat)))
    if diag and points is None:
        # Orthogonal axes: the 27-image sum of a Gaussian factorises exactly
        # into three 1-D three-term sums along the axes.
        n1, n2, n3 = grid
        L = np.diag(lat)
        axes = [np.arange(n) / n * L[i] for i, n in enumerate((n1, n2, n3))]
        v = np.zeros((n3, n2, n1))
        for R in tau:
            g = []
            for i in range(3):
                s = np.zeros_like(axes[i])
                for t in (-1, 0, 1):
                    d = axes[i] - R[i] - t * L[i]
                    s = s + np.exp(-(d * d) / (2.0 * sigma * sigma))
                g.append(s)
            v += g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
        return amp * v
    v = np.zeros(r.shape[:-1])
    for R in tau:
        for T in itertools.product((-1, 0, 1), repeat=3):
            shift = R + T[0] * lat[0] + T[1] * lat[1] + T[2] * lat[2]
            d = r - shift
            v += np.exp(-np.sum(d * d, axis=-1) / (2.0 * sigma * sigma))
    return amp * v


def beta_gaussian(lat, k, ecut: float, tau, widths) -> np.ndarray:
    """Projector coefficients B[i, G] = <k+G|beta_i>, complex128 (nproj, npw).

    Order: atom-major; per atom, per radial width w_n: [s, p_x, p_y, p_z].
    """
    lat = np.asarray(lat, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64).reshape(-1, 3)
    omega = volume(lat)
    _, _, q = gsphere(lat, k, ecut)
    q2 = np.sum(q * q, axis=1)
    y00 = 1.0 / (2.0 * math.sqrt(math.pi))
    y1 = math.sqrt(3.0 / (4.0 * math.pi))
    rows = []
    for R in tau:
        phase = np.exp(-1j * (q @ R))
        for w in widths:
            n0 = math.sqrt(4.0 / (math.sqrt(math.pi) * w ** 3))
            n1 = math.sqrt(8.0 / (3.0 * math.sqrt(math.pi) * w ** 5))
            g = np.exp(-0.5 * w * w * q2)
            c = (2.0 * math.pi) ** 1.5 / math.sqrt(omega)
            rows.append(phase * (c * n0 * w ** 3 * y00) * g)
            for ax in range(3):
                rows.append(phase * (-1j) * (c * n1 * w ** 5 * y1) * q[:, ax] * g)
    return np.array(rows, dtype=np.complex128).reshape(-1, q.shape[0])
