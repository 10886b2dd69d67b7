"""FP64 CPU oracle for the plane-wave H|psi> and the block-Davidson eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library and does not import it.

It is a plain, slow, obviously correct restatement of the operations the paper
names (Sec. 3.2.2 items (iii), (vi), (viii); Sec. 3.2.1; Sec. 3.3) in the
standard norm-conserving plane-wave formalism, in float64/complex128 with
NumPy/SciPy library primitives (FFT, GEMM, Cholesky, Hermitian eigensolver).

Parity status of each function is listed in its module header; every function
here is pinned by a ``-m "not gpu"`` test against a closed form, a brute-force
computation or a library routine on a special case.
"""
from .pw import (reciprocal, volume, gsphere, grid_slots, vloc_gaussian,
                 beta_gaussian, check_grid)
from .hamiltonian import (apply_local, apply_nonlocal, apply_kinetic, hpsi,
                          dense_h, h_diag, vtilde)
from .eigen import rayleigh_ritz, davidson
from .density import band_in_r, density
from .cg import cg
from .scf import hartree, exchange, scf_step

__all__ = [
    "reciprocal", "volume", "gsphere", "grid_slots", "vloc_gaussian",
    "beta_gaussian", "check_grid", "apply_local", "apply_nonlocal",
    "apply_kinetic", "hpsi", "dense_h", "h_diag", "vtilde", "rayleigh_ritz",
    "davidson", "band_in_r", "density", "cg", "hartree", "exchange", "scf_step",
]
