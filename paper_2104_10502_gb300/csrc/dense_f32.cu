// The dense linear algebra of dense.cu in single precision (namespace qe::f32):
// the mixed path solves its Rayleigh-Ritz problems, whose reduced matrices are
// FP32-accurate anyway, in FP32 (GB300 runs FP32 ~60x faster than FP64) and
// restores FP64 accuracy with a final FP64 Rayleigh-Ritz.
#define QE_DENSE_R float
#define QE_DENSE_NS qe::f32
#include "dense_impl.cuh"
