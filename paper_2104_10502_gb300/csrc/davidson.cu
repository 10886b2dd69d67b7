// Block Davidson on the device (Sec. 3.3 of the paper: Davidson iterative
// diagonalisation of the Kohn-Sham Hamiltonian).
#include "ctx.h"

extern "C" int qe_davidson(qe_ctx* ctx, const qe_problem* prob, int precision, double tol,
                           int max_iter, int max_dim, double* psi_inout, double* evals,
                           double* resid, int* iters, void* stream) {
  qe::set_error("qe_davidson: not available in this build");
  return QE_EINVAL;
}
