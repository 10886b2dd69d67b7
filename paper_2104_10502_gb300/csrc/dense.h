// FP64 dense linear algebra on the device (see dense.cu).
#pragma once

#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "plan.h"

namespace qe {

constexpr int kMaxDense = 4096;   // largest reduced problem handled
constexpr int kSmallDense = 64;   // largest one solved by the single-CTA shared-memory path

// State of the grid-wide barrier of the cooperative kernels (zeroed by the host
// before each launch); err is the shared error word (1 = a barrier timed out).
// wait_ns bounds every wait (2 s); stall (0 normally) is the number of extra
// arrivals a barrier waits for: a count that no CTA supplies, so that every
// barrier runs out (the test hook qe_test_grid_wait).
struct GridBar {
  unsigned int* count = nullptr;   // count[0] arrivals, count[1] generation
  unsigned int* gen = nullptr;     // == count + 1
  int* err = nullptr;
  unsigned long long wait_ns = 2000000000ull;
  unsigned int stall = 0;
};

// Precision-dependent constants of the dense kernels (machine epsilon, the
// smallest magnitude treated as nonzero, Sturm-interval margins, the relative
// width of an eigenvalue cluster for re-orthogonalisation).
template <typename R> struct RealT;
template <> struct RealT<double> {
  using vec2 = double2;
  static constexpr double eps = 2.2e-16, tiny = 1e-300, tiny_rel = 1e-30, margin = 1e-14;
  static constexpr double ctol = 1e-10;
};
template <> struct RealT<float> {
  using vec2 = float2;
  static constexpr float eps = 1.2e-7f, tiny = 1e-30f, tiny_rel = 1e-20f, margin = 1e-6f;
  static constexpr float ctol = 1e-5f;
};

template <typename R>
struct DenseWorkT {
  cx<R>* tau = nullptr;        // [n] Householder scalars
  cx<R>* p = nullptr;          // [n] tridiagonalisation work vector
  cx<R>* vbuf = nullptr;       // [n] reflector of the current step, contiguous
  cx<R>* refl = nullptr;       // [n][n] reflector j in row j (coalesced back-transformation)
  cx<R>* wyt = nullptr;        // [ceil((n-1)/8)][8][8] compact-WY T of each block of 8 reflectors
  R* d = nullptr;              // [n] diagonal of T
  R* e = nullptr;              // [n] off-diagonal of T
  R* y = nullptr;              // [nev][n] eigenvectors of T
  R* piv = nullptr;            // [n] Cholesky pivots
  int* status = nullptr;       // device status word (0 = ok)
  GridBar bar;                 // barrier state (3 words, next to status)
  R ctol_rel = RealT<R>::ctol; // cluster width relative to the spread of T
};
using DenseWork = DenseWorkT<double>;

// Lower Cholesky in place (upper part zeroed).  allow_drop: a column whose
// remaining pivot^2 is <= drop2 is dropped (zero column, piv = 0); otherwise a
// non-positive pivot sets *status = 1 + column.
// real_sym: A real (zero imaginary parts), factored in real arithmetic.
int cholesky(cx<double>* A, int n, int lda, double drop2, bool allow_drop, double* piv,
             int* status, GridBar bar, cudaStream_t st, bool real_sym = false);
// L X = B with L given as its transpose LT (LT[i][r] = L[r][i]).
int trsm_lower_t(const cx<double>* LT, int n, int ldt, cx<double>* B, int ldb, int ncols,
                 cudaStream_t st);
// dst = src^T (rows x cols -> cols x rows)
int transpose(const cx<double>* src, int lds, cx<double>* dst, int ldd, int rows, int cols,
              cudaStream_t st);
// L^+ X = B (L lower with real positive diagonal); real_sym: L and B real.
int trsm_upper_h(const cx<double>* L, int n, int ldl, cx<double>* B, int ldb, int ncols,
                 cudaStream_t st, bool real_sym = false);
int conj_transpose(const cx<double>* src, int lds, cx<double>* dst, int ldd, int rows, int cols,
                   cudaStream_t st);
int hermitize(cx<double>* A, int n, int lda, cudaStream_t st);
// Lowest nev eigenpairs of Hermitian A (destroyed): w[nev] ascending, X [n][ldx]
// with eigenvector k in column k.  real_sym: A is real (zero imaginary parts;
// the k = 0 reduced problems), reduced by the real form of the kernel.
int heev_lowest(cx<double>* A, int n, int lda, int nev, double* w, cx<double>* X, int ldx,
                DenseWork& wk, cudaStream_t st, Prof* pf, bool real_sym = false);
// Generalised lowest eigenpairs for n <= kSmallDense in one CTA: S = L L^+
// (L -> L, n x n; a non-positive pivot sets wk.status[0] = 1 + column), then
// the standard problem of L^-1 H L^-+ -> w[nev], Y in X (ld ldx); the caller
// applies X = L^-+ Y.  H, S: n x n with leading dimension ld.
int rr_small_fits(int n);
int rr_small(const cx<double>* H, const cx<double>* S, int ld, int n, int nev, cx<double>* L,
             double* w, cx<double>* X, int ldx, DenseWork& wk, cudaStream_t st, Prof* pf);

}  // namespace qe

// The same routines in single precision (dense_f32.cu).
namespace qe::f32 {
// Lower Cholesky in place (upper part zeroed).  allow_drop: a column whose
// remaining pivot^2 is <= drop2 is dropped (zero column, piv = 0); otherwise a
// non-positive pivot sets *status = 1 + column.
// real_sym: A real (zero imaginary parts), factored in real arithmetic.
int cholesky(cx<float>* A, int n, int lda, float drop2, bool allow_drop, float* piv,
             int* status, GridBar bar, cudaStream_t st, bool real_sym = false);
// L X = B with L given as its transpose LT (LT[i][r] = L[r][i]).
int trsm_lower_t(const cx<float>* LT, int n, int ldt, cx<float>* B, int ldb, int ncols,
                 cudaStream_t st);
// dst = src^T (rows x cols -> cols x rows)
int transpose(const cx<float>* src, int lds, cx<float>* dst, int ldd, int rows, int cols,
              cudaStream_t st);
// L^+ X = B (L lower with real positive diagonal); real_sym: L and B real.
int trsm_upper_h(const cx<float>* L, int n, int ldl, cx<float>* B, int ldb, int ncols,
                 cudaStream_t st, bool real_sym = false);
int conj_transpose(const cx<float>* src, int lds, cx<float>* dst, int ldd, int rows, int cols,
                   cudaStream_t st);
int hermitize(cx<float>* A, int n, int lda, cudaStream_t st);
// Lowest nev eigenpairs of Hermitian A (destroyed): w[nev] ascending, X [n][ldx]
// with eigenvector k in column k.
int heev_lowest(cx<float>* A, int n, int lda, int nev, float* w, cx<float>* X, int ldx,
                DenseWorkT<float>& wk, cudaStream_t st, Prof* pf, bool real_sym = false);
// Generalised lowest eigenpairs for n <= kSmallDense in one CTA: S = L L^+
// (L -> L, n x n; a non-positive pivot sets wk.status[0] = 1 + column), then
// the standard problem of L^-1 H L^-+ -> w[nev], Y in X (ld ldx); the caller
// applies X = L^-+ Y.  H, S: n x n with leading dimension ld.
int rr_small_fits(int n);
int rr_small(const cx<float>* H, const cx<float>* S, int ld, int n, int nev, cx<float>* L,
             float* w, cx<float>* X, int ldx, DenseWorkT<float>& wk, cudaStream_t st, Prof* pf);

}  // namespace qe::f32
