// Complex matrix products of the nonlocal (pseudopotential) term and of the
// Davidson subspace (Sec. 3.3: pseudopotential contribution to the
// Hamiltonian; Sec. 3.2.1: LAXlib dense linear algebra):
//
//   gemm_inner  P[m][n] = sum_k conj(A[m][k]) B[n][k]   (projections <beta|psi>,
//               overlap and Hamiltonian matrices of the subspace); K is the long
//               plane-wave axis, so K is split over CTAs and the partial sums are
//               added in a fixed order (deterministic, independent of timing);
//   gemm_outer  C[n][m] (+)= sum_k A[k][m] B[k][n]    (beta (D P), rotations V X);
//   dmul        Q = D P with a real D.
// These are SIMT kernels: FP64 has no tcgen05 kind on sm_103a (and DMMA runs
// no faster than DFMA on GB300), so they use the three-multiplication complex
// product to cut the multiply-adds by a quarter, and the FP64 instantiation
// computes in float-float arithmetic on the FP32 pipes (ff.cuh: 48-bit
// significands, ~1e-14 relative, the FP64 rate being 1/64 of the FP32 one on
// GB300); operands arrive and results leave in double.
#include <algorithm>
#include <type_traits>

#include "fft_device.cuh"
#include "plan.h"

namespace qe {

static int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

// Arithmetic of the kernels behind an instantiation (float-float for double) and
// the type of their split-K partials (double for float-float).
template <typename T>
using CompT = std::conditional_t<std::is_same<T, double>::value, ff, T>;
template <typename C>
using PartT = std::conditional_t<std::is_same<C, ff>::value, double, C>;

constexpr int IBM = 32, IBN = 32, IBK = 16;

// grid: (ceil(N/32), ceil(M/32), nsplit); block 256 = 16 x 16, 2 x 2 outputs each.
// Complex products by the three-multiplication form (3 real FMAs per complex
// multiply-add instead of 4): for conj(a) b,
//   t1 = ar br, t2 = ai bi, t3 = (ar - ai)(br + bi);  Re = t1 + t2, Im = t3 - t1 + t2.
template <typename T>
__global__ void __launch_bounds__(256)
k_gemm_inner(const double2* __restrict__ A, int lda, const double2* __restrict__ B, int ldb,
             int M, int N, int K, int kchunk, cx<PartT<T>>* __restrict__ part) {
  using P = PartT<T>;
  __shared__ T Ar[IBK][IBM + 1], Ai[IBK][IBM + 1], As[IBK][IBM + 1];
  __shared__ T Br[IBK][IBN + 1], Bi[IBK][IBN + 1], Bs[IBK][IBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.x * IBN, m0 = blockIdx.y * IBM;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  T t1[2][2] = {}, t2[2][2] = {}, t3[2][2] = {};
  for (int k0 = kb; k0 < ke; k0 += IBK) {
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int idx = tid + rep * 256;
      const int r = idx >> 4, kk = idx & 15;
      const int gk = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (gk < ke) {
        if (m0 + r < M) a = A[(size_t)(m0 + r) * lda + gk];
        if (n0 + r < N) b = B[(size_t)(n0 + r) * ldb + gk];
      }
      Ar[kk][r] = T(a.x);
      Ai[kk][r] = T(a.y);
      As[kk][r] = T(a.x) - T(a.y);
      Br[kk][r] = T(b.x);
      Bi[kk][r] = T(b.y);
      Bs[kk][r] = T(b.x) + T(b.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < IBK; ++kk) {
      T ar[2], ai[2], as[2], br[2], bi[2], bs[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        ar[i] = Ar[kk][ty * 2 + i]; ai[i] = Ai[kk][ty * 2 + i]; as[i] = As[kk][ty * 2 + i];
        br[i] = Br[kk][tx * 2 + i]; bi[i] = Bi[kk][tx * 2 + i]; bs[i] = Bs[kk][tx * 2 + i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }
  cx<P>* out = part + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
      if (m < M && n < N)
        out[(size_t)m * N + n] = {P(t1[i][j] + t2[i][j]), P(t3[i][j] - t1[i][j] + t2[i][j])};
    }
}

// Narrow variant for N <= 8 (one new band block against the basis, a small
// Gram matrix): tile 32 x 8, one output per thread (tm = tid % 32, tn = tid / 32),
// same three-multiplication products and split-K partials as k_gemm_inner.
// grid: (1, ceil(M/32), nsplit).
template <typename T>
__global__ void __launch_bounds__(256)
k_gemm_inner_n8(const double2* __restrict__ A, int lda, const double2* __restrict__ B, int ldb,
                int M, int N, int K, int kchunk, cx<PartT<T>>* __restrict__ part) {
  using P = PartT<T>;
  __shared__ T Ar[IBK][IBM + 1], Ai[IBK][IBM + 1], As[IBK][IBM + 1];
  __shared__ T Br[IBK][9], Bi[IBK][9], Bs[IBK][9];
  const int tid = threadIdx.x;
  const int tm = tid & 31, tn = tid >> 5;
  const int m0 = blockIdx.y * IBM;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  T t1 = T(0), t2 = T(0), t3 = T(0);
  for (int k0 = kb; k0 < ke; k0 += IBK) {
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int idx = tid + rep * 256;
      const int r = idx >> 4, kk = idx & 15;
      const int gk = k0 + kk;
      double2 a = make_double2(0.0, 0.0);
      if (gk < ke && m0 + r < M) a = A[(size_t)(m0 + r) * lda + gk];
      Ar[kk][r] = T(a.x);
      Ai[kk][r] = T(a.y);
      As[kk][r] = T(a.x) - T(a.y);
    }
    if (tid < 8 * IBK) {
      const int r = tid >> 4, kk = tid & 15;
      const int gk = k0 + kk;
      double2 b = make_double2(0.0, 0.0);
      if (gk < ke && r < N) b = B[(size_t)r * ldb + gk];
      Br[kk][r] = T(b.x);
      Bi[kk][r] = T(b.y);
      Bs[kk][r] = T(b.x) + T(b.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < IBK; ++kk) {
      t1 = fma(Ar[kk][tm], Br[kk][tn], t1);
      t2 = fma(Ai[kk][tm], Bi[kk][tn], t2);
      t3 = fma(As[kk][tm], Bs[kk][tn], t3);
    }
    __syncthreads();
  }
  const int m = m0 + tm, n = tn;
  if (m < M && n < N)
    part[(size_t)blockIdx.z * M * N + (size_t)m * N + n] = {P(t1 + t2), P(t3 - t1 + t2)};
}

// C = sum over splits of the partials, in split order.  Eight threads per
// output: thread q of an output adds splits q, q + 8, ... (two loads in
// flight), then the eight sums are combined in lane order; the total is the
// same for every launch (fixed order), independent of timing.
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_split(const cx<T>* __restrict__ part, int nsplit,
                                                      int M, int N, double2* __restrict__ C,
                                                      int ldc, int real_out) {
  const size_t total = (size_t)M * N;
  const int q = threadIdx.x & 7;
  const size_t o0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 3;
  const size_t ostride = ((size_t)gridDim.x * blockDim.x) >> 3;
  for (size_t i = o0; i < (total + ostride - 1) / ostride * ostride; i += ostride) {
    const bool valid = i < total;
    double sx = 0.0, sy = 0.0;
    if (valid) {
      int s = q;
      for (; s + 8 < nsplit; s += 16) {
        const cx<T> p0 = part[(size_t)s * total + i], p1 = part[(size_t)(s + 8) * total + i];
        sx += (double)p0.x; sy += (double)p0.y;
        sx += (double)p1.x; sy += (double)p1.y;
      }
      if (s < nsplit) {
        const cx<T> p0 = part[(size_t)s * total + i];
        sx += (double)p0.x; sy += (double)p0.y;
      }
    }
    for (int o = 1; o < 8; o <<= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (valid && q == 0) {
      const size_t m = i / N, n = i - m * N;
      C[m * ldc + n] = make_double2(sx, real_out ? 0.0 : sy);
    }
  }
}

static int reduce_blocks(size_t total) {
  return (int)std::max<size_t>(1, std::min<size_t>((total * 8 + 255) / 256, 152 * 8));
}

static int inner_split(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 1;
  const int tiles = ((M + IBM - 1) / IBM) * (N <= 8 ? 1 : (N + IBN - 1) / IBN);
  int ns = (2 * 152 * 4 + tiles - 1) / tiles;  // aim for ~4 CTAs per SM
  const int maxs = std::max(1, K / 32);         // at least 32 k per split
  ns = std::max(1, std::min(ns, maxs));
  return ns;
}

template <typename T>
static void launch_inner(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                         int kchunk, int nsplit, void* part, cudaStream_t st) {
  using C = CompT<T>;
  if (N <= 8) {
    dim3 g(1, (M + IBM - 1) / IBM, nsplit);
    k_gemm_inner_n8<C><<<g, 256, 0, st>>>(reinterpret_cast<const double2*>(A), lda,
                                           reinterpret_cast<const double2*>(B), ldb, M, N, K, kchunk,
                                           reinterpret_cast<cx<PartT<C>>*>(part));
  } else {
    dim3 g((N + IBN - 1) / IBN, (M + IBM - 1) / IBM, nsplit);
    k_gemm_inner<C><<<g, 256, 0, st>>>(reinterpret_cast<const double2*>(A), lda,
                                        reinterpret_cast<const double2*>(B), ldb, M, N, K, kchunk,
                                        reinterpret_cast<cx<PartT<C>>*>(part));
  }
}

size_t gemm_inner_scratch(int M, int N, int K, size_t elem_bytes) {
  if (M <= 0 || N <= 0) return 0;
  return (size_t)inner_split(M, N, K) * M * N * 2 * elem_bytes;
}

template <typename T>
int gemm_inner(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
               int ldc, void* part, size_t part_bytes, cudaStream_t st, Prof* pf, bool real_out) {
  if (M <= 0 || N <= 0) return QE_OK;
  const int ns = inner_split(M, N, K);
  if ((size_t)ns * M * N * sizeof(cx<PartT<CompT<T>>>) > part_bytes) {
    set_error("gemm_inner: scratch too small");
    return QE_EINVAL;
  }
  int kchunk = (K + ns - 1) / ns;
  kchunk = (kchunk + IBK - 1) / IBK * IBK;
  const int nsplit = std::max(1, (K + kchunk - 1) / kchunk);
  int rc;
  {
  ProfScope ps(pf, "k_gemm_inner", st);
  launch_inner<T>(A, lda, B, ldb, M, N, K, kchunk, nsplit, part, st);
  rc = check_launch("k_gemm_inner");
  }
  if (rc) return rc;
  ProfScope ps(pf, "k_reduce_split", st);
  const size_t total = (size_t)M * N;
  const int blocks = reduce_blocks(total);
  using P = PartT<CompT<T>>;
  k_reduce_split<P><<<blocks, 256, 0, st>>>(reinterpret_cast<const cx<P>*>(part), nsplit, M, N,
                                            reinterpret_cast<double2*>(C), ldc,
                                            real_out ? 1 : 0);
  return check_launch("k_reduce_split");
}

// As gemm_inner, but with as many K splits as fit in `part_bytes` (at least one),
// for callers whose scratch is a fixed-size region.
template <typename T>
int gemm_inner_bounded(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                       double* C, int ldc, void* part, size_t part_bytes, cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  const size_t one = (size_t)M * N * sizeof(cx<PartT<CompT<T>>>);
  if (one > part_bytes) {
    set_error("gemm_inner_bounded: scratch holds no split");
    return QE_EINVAL;
  }
  const int ns = std::max(1, std::min(inner_split(M, N, K), (int)(part_bytes / one)));
  int kchunk = (K + ns - 1) / ns;
  kchunk = (kchunk + IBK - 1) / IBK * IBK;
  const int nsplit = std::max(1, (K + kchunk - 1) / kchunk);
  int rc;
  {
  ProfScope ps(pf, "k_gemm_inner", st);
  launch_inner<T>(A, lda, B, ldb, M, N, K, kchunk, nsplit, part, st);
  rc = check_launch("k_gemm_inner");
  }
  if (rc) return rc;
  ProfScope ps(pf, "k_reduce_split", st);
  const size_t total = (size_t)M * N;
  const int blocks = reduce_blocks(total);
  using P = PartT<CompT<T>>;
  k_reduce_split<P><<<blocks, 256, 0, st>>>(reinterpret_cast<const cx<P>*>(part), nsplit, M, N,
                                            reinterpret_cast<double2*>(C), ldc, 0);
  return check_launch("k_reduce_split");
}

template int gemm_inner_bounded<double>(const double*, int, const double*, int, int, int, int,
                                        double*, int, void*, size_t, cudaStream_t, Prof*);
template int gemm_inner_bounded<float>(const double*, int, const double*, int, int, int, int,
                                       double*, int, void*, size_t, cudaStream_t, Prof*);

constexpr int OBM = 64, OBN = 32, OBK = 16;

// grid: (ceil(M/64), ceil(N/32)); block 256; thread (tm = tid % 16, tn = tid / 16)
// owns m = m0 + tm + 16 i (i < 4) and n = n0 + 2 tn + j (j < 2).  Three-
// multiplication complex products: t1 = ar br, t2 = ai bi,
// t3 = (ar + ai)(br + bi);  Re = t1 - t2, Im = t3 - t1 - t2.
template <typename T>
__global__ void __launch_bounds__(256)
k_gemm_outer(const double2* __restrict__ A, int lda, const double2* __restrict__ B, int ldb,
             int M, int N, int K, double2* __restrict__ C, int ldc, int alpha_neg, int beta) {
  __shared__ T Ar[OBK][OBM], Ai[OBK][OBM], As[OBK][OBM];
  __shared__ T Br[OBK][OBN + 1], Bi[OBK][OBN + 1], Bs[OBK][OBN + 1];
  const int tid = threadIdx.x;
  const int tm = tid & 15, tn = tid >> 4;
  const int m0 = blockIdx.x * OBM, n0 = blockIdx.y * OBN;
  T t1[4][2] = {}, t2[4][2] = {}, t3[4][2] = {};
  for (int k0 = 0; k0 < K; k0 += OBK) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      const int idx = tid + rep * 256;
      const int kk = idx >> 6, mm = idx & 63;
      double2 a = make_double2(0.0, 0.0);
      if (k0 + kk < K && m0 + mm < M) a = A[(size_t)(k0 + kk) * lda + m0 + mm];
      Ar[kk][mm] = T(a.x);
      Ai[kk][mm] = T(a.y);
      As[kk][mm] = T(a.x) + T(a.y);
    }
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int idx = tid + rep * 256;
      const int kk = idx >> 5, nn = idx & 31;
      double2 b = make_double2(0.0, 0.0);
      if (k0 + kk < K && n0 + nn < N) b = B[(size_t)(k0 + kk) * ldb + n0 + nn];
      Br[kk][nn] = T(b.x);
      Bi[kk][nn] = T(b.y);
      Bs[kk][nn] = T(b.x) + T(b.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < OBK; ++kk) {
      T ar[4], ai[4], as[4], br[2], bi[2], bs[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = Ar[kk][tm + 16 * i]; ai[i] = Ai[kk][tm + 16 * i]; as[i] = As[kk][tm + 16 * i];
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        br[j] = Br[kk][2 * tn + j]; bi[j] = Bi[kk][2 * tn + j]; bs[j] = Bs[kk][2 * tn + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int n = n0 + 2 * tn + j;
    if (n >= N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + tm + 16 * i;
      if (m >= M) continue;
      double2* c = C + (size_t)n * ldc + m;
      double2 v = make_double2((double)(t1[i][j] - t2[i][j]), (double)(t3[i][j] - t1[i][j] - t2[i][j]));
      if (alpha_neg) { v.x = -v.x; v.y = -v.y; }
      if (beta) { const double2 o = *c; v.x += o.x; v.y += o.y; }
      *c = v;
    }
  }
}

// Narrow variant for N <= 8: tile 32 x 8, one output per thread (tm = tid % 32,
// tn = tid / 32), so that a band block of a small problem still spreads over
// ceil(M/32) CTAs.  grid: (ceil(M/32), 1).
template <typename T>
__global__ void __launch_bounds__(256)
k_gemm_outer_n8(const double2* __restrict__ A, int lda, const double2* __restrict__ B, int ldb,
                int M, int N, int K, double2* __restrict__ C, int ldc, int alpha_neg, int beta) {
  __shared__ T Ar[OBK][32], Ai[OBK][32], As[OBK][32];
  __shared__ T Br[OBK][9], Bi[OBK][9], Bs[OBK][9];
  const int tid = threadIdx.x;
  const int tm = tid & 31, tn = tid >> 5;
  const int m0 = blockIdx.x * 32;
  T t1 = T(0), t2 = T(0), t3 = T(0);
  for (int k0 = 0; k0 < K; k0 += OBK) {
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int idx = tid + rep * 256;
      const int kk = idx >> 5, mm = idx & 31;
      double2 a = make_double2(0.0, 0.0);
      if (k0 + kk < K && m0 + mm < M) a = A[(size_t)(k0 + kk) * lda + m0 + mm];
      Ar[kk][mm] = T(a.x);
      Ai[kk][mm] = T(a.y);
      As[kk][mm] = T(a.x) + T(a.y);
    }
    if (tid < OBK * 8) {
      const int kk = tid >> 3, nn = tid & 7;
      double2 b = make_double2(0.0, 0.0);
      if (k0 + kk < K && nn < N) b = B[(size_t)(k0 + kk) * ldb + nn];
      Br[kk][nn] = T(b.x);
      Bi[kk][nn] = T(b.y);
      Bs[kk][nn] = T(b.x) + T(b.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < OBK; ++kk) {
      t1 = fma(Ar[kk][tm], Br[kk][tn], t1);
      t2 = fma(Ai[kk][tm], Bi[kk][tn], t2);
      t3 = fma(As[kk][tm], Bs[kk][tn], t3);
    }
    __syncthreads();
  }
  const int m = m0 + tm, n = tn;
  if (m >= M || n >= N) return;
  double2* c = C + (size_t)n * ldc + m;
  double2 v = make_double2((double)(t1 - t2), (double)(t3 - t1 - t2));
  if (alpha_neg) { v.x = -v.x; v.y = -v.y; }
  if (beta) { const double2 o = *c; v.x += o.x; v.y += o.y; }
  *c = v;
}

template <typename T>
int gemm_outer_ab(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                  double* C, int ldc, int alpha_neg, int beta, cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (K <= 0) {
    set_error("gemm_outer: K must be positive");
    return QE_EINVAL;
  }
  ProfScope ps(pf, "k_gemm_outer", st);
  if (N <= 8) {
    k_gemm_outer_n8<CompT<T>><<<(M + 31) / 32, 256, 0, st>>>(reinterpret_cast<const double2*>(A), lda,
                                                       reinterpret_cast<const double2*>(B), ldb, M, N,
                                                       K, reinterpret_cast<double2*>(C), ldc,
                                                       alpha_neg, beta);
    return check_launch("k_gemm_outer");
  }
  dim3 g((M + OBM - 1) / OBM, (N + OBN - 1) / OBN);
  k_gemm_outer<CompT<T>><<<g, 256, 0, st>>>(reinterpret_cast<const double2*>(A), lda,
                                      reinterpret_cast<const double2*>(B), ldb, M, N, K,
                                      reinterpret_cast<double2*>(C), ldc, alpha_neg, beta);
  return check_launch("k_gemm_outer");
}

template <typename T>
int gemm_outer(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
               int ldc, int beta, cudaStream_t st, Prof* pf) {
  return gemm_outer_ab<T>(A, lda, B, ldb, M, N, K, C, ldc, 0, beta, st, pf);
}

// One CTA per row i of D: the nonzero entries of the row are compacted in
// shared memory in column order (a block-wide scan, so the summation order is
// fixed), then each thread sums them for its columns n of P.
__global__ void __launch_bounds__(128) k_dmul(const double* __restrict__ D,
                                              const double2* __restrict__ P,
                                              double2* __restrict__ Q, int np, int nb,
                                              int real_p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* val = reinterpret_cast<double*>(smem_raw);
  int* col = reinterpret_cast<int*>(val + np);
  __shared__ int wcount[4];
  __shared__ int base;
  const int i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const double* d = D + (size_t)i * np;
  for (int j0 = 0; j0 < np; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const double v = j < np ? d[j] : 0.0;
    const bool nz = v != 0.0;
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int w = 0; w < warp; ++w) off += wcount[w];
    if (nz) {
      const int pos = off + __popc(bal & ((1u << lane) - 1u));
      val[pos] = v;
      col[pos] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += wcount[0] + wcount[1] + wcount[2] + wcount[3];
    __syncthreads();
  }
  const int cnt = base;
  for (int n = threadIdx.x; n < nb; n += blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < cnt; ++q) {
      const double2 pv = P[(size_t)col[q] * nb + n];
      sx = fma(val[q], pv.x, sx);
      sy = fma(val[q], pv.y, sy);
    }
    Q[(size_t)i * nb + n] = make_double2(sx, real_p ? 0.0 : sy);
  }
}

int dmul(const double* D, const double* P, double* Q, int np, int nb, cudaStream_t st, Prof* pf,
         bool real_p) {
  if (np <= 0 || nb <= 0) return QE_OK;
  ProfScope ps(pf, "k_dmul", st);
  const size_t sm = (size_t)np * (sizeof(double) + sizeof(int));
  set_max_dynamic_smem(k_dmul);
  k_dmul<<<np, 128, sm, st>>>(D, reinterpret_cast<const double2*>(P), reinterpret_cast<double2*>(Q),
                              np, nb, real_p ? 1 : 0);
  return check_launch("k_dmul");
}

template int gemm_inner<double>(const double*, int, const double*, int, int, int, int, double*, int,
                                void*, size_t, cudaStream_t, Prof*, bool);
template int gemm_inner<float>(const double*, int, const double*, int, int, int, int, double*, int,
                               void*, size_t, cudaStream_t, Prof*, bool);
template int gemm_outer_ab<double>(const double*, int, const double*, int, int, int, int, double*,
                                   int, int, int, cudaStream_t, Prof*);
template int gemm_outer_ab<float>(const double*, int, const double*, int, int, int, int, double*,
                                  int, int, int, cudaStream_t, Prof*);
template int gemm_outer<double>(const double*, int, const double*, int, int, int, int, double*, int,
                                int, cudaStream_t, Prof*);
template int gemm_outer<float>(const double*, int, const double*, int, int, int, int, double*, int,
                               int, cudaStream_t, Prof*);

}  // namespace qe
