"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Calls only ``oracle`` and ``qeinputs``.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import qeinputs  # noqa: E402


def dense_eigs(name, nev):
    c = qeinputs.config(name)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    h = oracle.dense_h(lat, k, ecut, grid, v, beta, d)
    return np.linalg.eigvalsh(h)[:nev]


def write(fname, header, values):
    with open(os.path.join(HERE, fname), "w") as f:
        for line in header:
            f.write("# " + line + "\n")
        for x in values:
            f.write(f"{x:.17e}\n")


def davidson_eigs(name, tol):
    c = qeinputs.config(name)
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    _, kin, _ = oracle.gsphere(lat, k, ecut)
    psi0 = qeinputs.start_bands(kin, c["nbnd"], c["psi_seed"])
    r = oracle.davidson(lambda x: oracle.hpsi(lat, k, ecut, grid, v, beta, d, x),
                        oracle.h_diag(kin, v, beta, d), psi0, tol)
    if not r["converged"]:
        raise RuntimeError(f"{name}: oracle Davidson did not converge")
    return r["e"], r["iters"]


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "c2":
    e, it = davidson_eigs("C2", 1e-7)
    write("c2_davidson_eigs.txt",
          ["Lowest 256 eigenvalues (Ry) of the C2 workload (the C1 cell: cubic a=20 bohr,",
           "64 seeded atoms, 512 projectors, 40 Ry, grid 96^3) from the FP64 oracle's block",
           f"Davidson at residual 1e-7 ({it} iterations).  The mixed-precision GPU path of",
           "the paper's Davidson solver (Sec. 3.3) must match these to 1e-6 Ry."],
          e)
    sys.exit(0)

if __name__ == "__main__":
    write("c0_dense_eigs.txt",
          ["Lowest 16 eigenvalues (Ry) of the dense H of the C0 cell (cubic a=10 bohr,",
           "2 atoms, 20 Ry, grid 32^3, Gaussian V_loc, 4 projectors/atom), by LAPACK",
           "eigvalsh of the oracle's element-wise dense matrix.  Davidson of the paper",
           "(Sec. 3.3) must reproduce the lowest 8 to 1e-10 Ry."],
          dense_eigs("C0", 16))
    write("small_dense_eigs.txt",
          ["Lowest 16 eigenvalues (Ry) of the dense H of the SMALL cell (7x8x9 bohr,",
           "k off Gamma, 12 Ry, grid 24x27x30, two projector widths), LAPACK eigvalsh."],
          dense_eigs("SMALL", 16))
    unit = (2 * math.pi / 10.0) ** 2
    write("c0_empty_lattice.txt",
          ["Empty lattice, cubic a=10 bohr at Gamma: eigenvalues (2pi/a)^2 n, n the",
           "sums of three squares in increasing order (0, 1 x6, 2 x12); lowest 8."],
          [unit * n for n in (0, 1, 1, 1, 1, 1, 1, 2)])
