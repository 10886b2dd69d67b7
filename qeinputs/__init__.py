"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module holds no arithmetic of the method (no plane-wave sphere, no
potential, no projector, no Hamiltonian, no eigensolver).  It only fixes the
synthetic workloads — cells, atom positions, projector widths, D values,
band counts — and draws the random numbers those workloads need, so that the
FP64 oracle and the CUDA path start from identical inputs.

The paper's benchmark structures (16 COD crystals with SSSP pseudopotentials,
Sec. 3.3) are not available; the cells below stand in for them with the
paper's shapes: tens of atoms, 250-1000 A^3 cells (Sec. 3.3).

Units: bohr, Rydberg.
"""
from __future__ import annotations

import numpy as np

# Gaussian local potential V(r) = AMP * sum_I exp(-|r-R_I|^2 / (2 SIGMA^2)).
VLOC_AMP_RY = -2.0
VLOC_SIGMA = 1.0
# Diagonal D values of the Kleinman-Bylander projectors, per angular channel.
D_S_RY = 0.5
D_P_RY = -0.3
# Number of projectors per radial function: one s plus three p (x, y, z).
PROJ_PER_RADIAL = 4


def cubic(a: float) -> np.ndarray:
    """Simple cubic lattice, rows are a1, a2, a3 (bohr)."""
    return np.diag([float(a)] * 3)


def tetragonal(a: float, c: float) -> np.ndarray:
    """Tetragonal lattice a x a x c (bohr), rows are a1, a2, a3."""
    return np.diag([float(a), float(a), float(c)])


def random_atoms(lat: np.ndarray, natom: int, min_sep: float, seed: int,
                 max_tries: int = 1_000_000) -> np.ndarray:
    """Cartesian positions (natom, 3) drawn uniformly in the cell by rejection.

    A candidate is accepted when its periodic minimum-image distance to every
    accepted atom is at least ``min_sep`` bohr.  Raises RuntimeError when
    ``max_tries`` candidates do not suffice.
    """
    rng = np.random.default_rng(seed)
    lat = np.asarray(lat, dtype=np.float64)
    frac = []
    tries = 0
    while len(frac) < natom:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_atoms: could not place atoms")
        f = rng.random(3)
        ok = True
        for g in frac:
            d = f - g
            d -= np.round(d)
            if np.linalg.norm(d @ lat) < min_sep:
                ok = False
                break
        if ok:
            frac.append(f)
    return np.array(frac).reshape(-1, 3) @ lat


def d_matrix(natom: int, nrad: int) -> np.ndarray:
    """Block-diagonal D (Ry), projector order atom-major, then per radial
    function [s, p_x, p_y, p_z]."""
    per_atom = np.array(([D_S_RY] + [D_P_RY] * 3) * nrad, dtype=np.float64)
    return np.diag(np.tile(per_atom, natom))


def start_bands(kin: np.ndarray, nbnd: int, seed: int) -> np.ndarray:
    """Random starting bands (nbnd, npw) complex128: (u + i v) / (1 + |k+G|^2),
    u, v ~ N(0, 1) from ``numpy.random.default_rng(seed)``.  ``kin`` is the
    caller's |k+G|^2 array in plane-wave order."""
    rng = np.random.default_rng(seed)
    npw = int(np.asarray(kin).shape[0])
    u = rng.standard_normal((nbnd, npw))
    v = rng.standard_normal((nbnd, npw))
    return (u + 1j * v) / (1.0 + np.asarray(kin, dtype=np.float64))[None, :]


def random_vectors(nbnd: int, npw: int, seed: int) -> np.ndarray:
    """Plain complex Gaussian block (nbnd, npw) complex128 for operator tests."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nbnd, npw)) + 1j * rng.standard_normal((nbnd, npw))


def mp_kpoints_frac(n1: int, n2: int, n3: int) -> np.ndarray:
    """Gamma-centred Monkhorst-Pack grid in fractional reciprocal coordinates
    (i/n1, j/n2, l/n3), all points kept (no symmetry reduction)."""
    return np.array([[i / n1, j / n2, l / n3]
                     for i in range(n1) for j in range(n2) for l in range(n3)],
                    dtype=np.float64)


def config(name: str) -> dict:
    """The synthetic workloads.

    C0  plain FP64 Davidson: cubic a=10, 2 atoms, 20 Ry, grid 32^3, 8 bands.
    C1  H|psi> throughput: cubic a=20, 64 random atoms, 40 Ry, grid 96^3,
        8 projectors/atom (512), 128 bands.
    C2  mixed precision: the C1 cell with 256 bands.
    C3T tetragonal 12x12x24, 24 atoms, 30 Ry, grid 48x48x96, 4x4x1 k grid, 64 bands.
    SMALL  a small odd-grid cell for fast parity tests (two radial sets).
    """
    if name == "C0":
        lat = cubic(10.0)
        return dict(name=name, lat=lat, k=np.zeros(3), ecut=20.0, grid=(32, 32, 32),
                    tau=np.array([[0.0, 0.0, 0.0], [5.0, 5.0, 5.0]]),
                    widths=(1.0,), nbnd=8, tol=1e-8, psi_seed=0)
    if name in ("C1", "C2"):
        lat = cubic(20.0)
        tau = random_atoms(lat, 64, 2.5, seed=1)
        nb = 128 if name == "C1" else 256
        return dict(name=name, lat=lat, k=np.zeros(3), ecut=40.0, grid=(96, 96, 96),
                    tau=tau, widths=(1.0, 0.7), nbnd=nb, tol=1e-6,
                    psi_seed=2 if name == "C1" else 3)
    if name == "C3T":
        lat = tetragonal(12.0, 24.0)
        tau = random_atoms(lat, 24, 2.5, seed=4)
        return dict(name=name, lat=lat, k=np.zeros(3), ecut=30.0, grid=(48, 48, 96),
                    tau=tau, widths=(1.0,), nbnd=64, tol=1e-6, psi_seed=4,
                    kfrac=mp_kpoints_frac(4, 4, 1))
    if name == "SMALL":
        # odd, mixed-radix grid; k off Gamma; several sticks and a ragged tail
        lat = np.array([[7.0, 0.0, 0.0], [0.0, 8.0, 0.0], [0.0, 0.0, 9.0]])
        tau = np.array([[0.5, 1.0, 1.5], [4.0, 3.5, 6.0], [2.0, 6.5, 2.5]])
        return dict(name=name, lat=lat, k=np.array([0.11, -0.07, 0.05]), ecut=12.0,
                    grid=(24, 27, 30), tau=tau, widths=(1.0, 0.7), nbnd=7,
                    tol=1e-8, psi_seed=11)
    raise KeyError(name)


def smooth235(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    m = max(1, int(n))
    while True:
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            return m
        m += 1


def c3_problems() -> list:
    """The batched workload: the C3T cell at its 16 Gamma-centred k points
    (k = (i/4) b1 + (j/4) b2, i, j = 0..3), then 32 cubic cells with
    a in U{8..16} bohr, 2..24 atoms (fewer in the smallest cells, so that
    rejection sampling at 2.5 bohr separation stays quick: at most a^3/24),
    nb in U{16..96}, 30 Ry, 4 projectors per atom (w = 1 bohr) and each grid
    dimension the smallest 2,3,5-smooth N >= 2 floor(a sqrt(ecut) / 2 pi) + 1
    (the no-wrap bound on a cubic cell at Gamma).  Draws from
    default_rng(5); start-band seeds 100 + index."""
    t = config("C3T")
    lat = t["lat"]
    if np.count_nonzero(lat - np.diag(np.diag(lat))):
        raise ValueError("c3_problems: orthogonal cell expected")
    bdiag = 2.0 * np.pi / np.diag(lat)          # b_i of an orthogonal cell
    out = []
    for i, kf in enumerate(t["kfrac"]):
        out.append(dict(lat=lat, k=kf * bdiag, ecut=t["ecut"], grid=t["grid"], tau=t["tau"],
                        widths=t["widths"], nbnd=t["nbnd"], psi_seed=100 + i, tol=t["tol"]))
    rng = np.random.default_rng(5)
    for j in range(32):
        a = int(rng.integers(8, 17))
        natom = int(rng.integers(2, 25))
        natom = max(2, min(natom, (a ** 3) // 24))
        nb = int(rng.integers(16, 97))
        aseed = int(rng.integers(0, 2 ** 31))
        lat_c = cubic(float(a))
        mmax = int(np.floor(a * np.sqrt(30.0) / (2.0 * np.pi)))
        n = smooth235(2 * mmax + 1)
        out.append(dict(lat=lat_c, k=np.zeros(3), ecut=30.0, grid=(n, n, n),
                        tau=random_atoms(lat_c, natom, 2.5, seed=aseed), widths=(1.0,),
                        nbnd=nb, psi_seed=100 + len(out), tol=t["tol"]))
    return out
