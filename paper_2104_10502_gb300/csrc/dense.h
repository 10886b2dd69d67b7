// FP64 dense linear algebra on the device (see dense.cu).
#pragma once

#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "plan.h"

namespace qe {

constexpr int kMaxDense = 4096;   // largest reduced problem handled

// State of the grid-wide barrier of the cooperative kernels (zeroed by the host
// before each launch); err is the shared error word (1 = a barrier timed out).
struct GridBar {
  unsigned int* count = nullptr;   // count[0] arrivals, count[1] generation
  unsigned int* gen = nullptr;     // == count + 1
  int* err = nullptr;
};

struct DenseWork {
  cx<double>* tau = nullptr;   // [n] Householder scalars
  cx<double>* p = nullptr;     // [n] tridiagonalisation work vector
  cx<double>* vbuf = nullptr;  // [n] reflector of the current step, contiguous
  cx<double>* refl = nullptr;  // [n][n] reflector j in row j (coalesced back-transformation)
  double* d = nullptr;         // [n] diagonal of T
  double* e = nullptr;         // [n] off-diagonal of T
  double* y = nullptr;         // [nev][n] eigenvectors of T
  double* piv = nullptr;       // [n] Cholesky pivots
  int* status = nullptr;       // device status word (0 = ok)
  GridBar bar;                 // barrier state (3 words, next to status)
  double ctol_rel = 1e-10;     // cluster width relative to the spread of T
};

// Lower Cholesky in place (upper part zeroed).  allow_drop: a column whose
// remaining pivot^2 is <= drop2 is dropped (zero column, piv = 0); otherwise a
// non-positive pivot sets *status = 1 + column.
int cholesky(cx<double>* A, int n, int lda, double drop2, bool allow_drop, double* piv,
             int* status, GridBar bar, cudaStream_t st);
int trsm_lower(const cx<double>* L, int n, int ldl, cx<double>* B, int ldb, int ncols,
               cudaStream_t st);
int trsm_upper_h(const cx<double>* L, int n, int ldl, cx<double>* B, int ldb, int ncols,
                 cudaStream_t st);
int conj_transpose(const cx<double>* src, int lds, cx<double>* dst, int ldd, int rows, int cols,
                   cudaStream_t st);
int hermitize(cx<double>* A, int n, int lda, cudaStream_t st);
// Lowest nev eigenpairs of Hermitian A (destroyed): w[nev] ascending, X [n][ldx]
// with eigenvector k in column k.
int heev_lowest(cx<double>* A, int n, int lda, int nev, double* w, cx<double>* X, int ldx,
                DenseWork& wk, cudaStream_t st, Prof* pf);

}  // namespace qe
