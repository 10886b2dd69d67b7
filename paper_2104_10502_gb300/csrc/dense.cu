// Complex dense linear algebra of the Rayleigh-Ritz step and of the Cholesky
// orthonormalisation (Sec. 3.2.1 of the paper: LAXlib, parallel dense linear
// algebra and diagonalisation; Sec. 3.3: generalized eigenproblems), FP64
// instantiation of dense_impl.cuh (dense_f32.cu is the FP32 one).
//
// Matrices are row-major complex (interleaved reals), A[i][j] at i*lda + j.
//   cholesky      right-looking, one launch per column, optional dropping of
//                 columns whose remaining pivot is below a threshold (this is
//                 Gram-Schmidt with dropping, expressed on the Gram matrix);
//   trsm_lower    L X = B, column-parallel forward substitution;
//   trsm_upper_h  L^+ X = B, column-parallel back substitution;
//   heev_lowest   lowest eigenpairs of a Hermitian matrix: Householder
//                 tridiagonalisation (real off-diagonal), Sturm bisection,
//                 inverse iteration with re-orthogonalisation inside clusters
//                 of (nearly) equal eigenvalues, back-transformation.
//   rr_small      the whole generalised reduction for n <= 64 in one CTA.
// The multi-CTA kernels are cooperative launches with a bounded grid barrier.
// In this instantiation (QE_DENSE_FP64) the tridiagonalisation, the last
// bisection rounds, inverse iteration, back-transformation and rr_small run in
// float-float arithmetic on the FP32 pipes (the *_ff kernels of dense_impl.cuh).
#define QE_DENSE_R double
#define QE_DENSE_NS qe
#define QE_DENSE_FP64 1
#include "dense_impl.cuh"
