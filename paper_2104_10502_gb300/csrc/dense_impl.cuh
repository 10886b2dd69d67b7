// Implementation of the complex dense linear algebra for one real type R
// (double: the FP64 kernels; float: the mixed path's reduced problems), included
// by dense.cu with QE_DENSE_R = double and by dense_f32.cu with float.
// Matrices are row-major complex (interleaved R), A[i][j] at i*lda + j.
#include <algorithm>
#include <cmath>

#include "dense.h"
#include "plan.h"
#include "fft_device.cuh"

namespace QE_DENSE_NS {

using namespace ::qe;
using R = QE_DENSE_R;
using z = cx<R>;



static int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

__device__ __forceinline__ z zconj(z a) { return {a.x, -a.y}; }
__device__ __forceinline__ R zabs2(z a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// acc + a b and a - (x conj(y) + u conj(t)) as explicit FMA chains (4 and 8 FMAs;
// left to contraction the products and sums take 6 and 12 FP64 instructions)
__device__ __forceinline__ z zfma(z a, z b, z acc) {
  acc.x = fmar(a.x, b.x, acc.x);
  acc.x = fmar(-a.y, b.y, acc.x);
  acc.y = fmar(a.x, b.y, acc.y);
  acc.y = fmar(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ z zrank2(z a, z x, z y, z u, z t) {
  a.x = fmar(-x.x, y.x, a.x);
  a.x = fmar(-x.y, y.y, a.x);
  a.x = fmar(-u.x, t.x, a.x);
  a.x = fmar(-u.y, t.y, a.x);
  a.y = fmar(-x.y, y.x, a.y);
  a.y = fmar(x.x, y.y, a.y);
  a.y = fmar(-u.y, t.x, a.y);
  a.y = fmar(u.x, t.y, a.y);
  return a;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024).  Every thread gets the result.
__device__ R block_sum(R v, R* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  R t = R(0);
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? sh[threadIdx.x] : R(0);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ---- persistent (cooperative) kernels -------------------------------------------
// Loads of data that other CTAs wrote earlier in the same kernel go through L2
// (ld.global.cg): L1 is not coherent across SMs.
__device__ __forceinline__ z ldz(const z* p) {
  const typename RealT<R>::vec2 v = __ldcg(reinterpret_cast<const typename RealT<R>::vec2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ R ldd(const R* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Every wait
// is bounded (b.wait_ns, 2 s); on time-out the error word is set, the waiting
// CTAs see it within 1024 polls, return false and leave the kernel.
__device__ bool grid_sync(const GridBar& b) {
  __shared__ int s_ok;
  __syncthreads();
  // one CTA: the block barrier above already orders its global accesses
  if (gridDim.x == 1) return true;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_gpu(b.gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(b.count, 1u) + 1u;
    if (arrived == gridDim.x + b.stall) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      // acquire-poll the generation word; the clock and the error word are read
      // only every 1024 polls (each read is an L2 round trip on the critical path)
      unsigned long long t0 = 0;
      for (int it = 0;; ++it) {
        if (ld_acquire_gpu(b.gen) != g) break;
        if ((it & 1023) == 1023) {
          const unsigned long long t = gtime_ns();
          if (t0 == 0) t0 = t;
          else if (t - t0 > b.wait_ns) { atomicExch(b.err, 1); ok = 0; break; }
          if (*(volatile int*)b.err) { ok = 0; break; }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid-wide barrier on a monotonic arrival counter (count zeroed by the host
// before the launch; a launch uses either this or grid_sync): the k-th barrier
// of the launch returns once count reaches k * gridDim.x.  Arrival is one
// fence and one reduction without a return value, the wait one acquire poll
// of the same word: fewer L2 round trips than the generation barrier.  Bounded
// (b.wait_ns) like grid_sync.
__device__ bool grid_sync_mono(const GridBar& b, unsigned k) {
  __shared__ int s_ok;
  __syncthreads();
  if (gridDim.x == 1) return true;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(b.count, 1u);
    const unsigned target = k * gridDim.x + b.stall;
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
      if (ld_acquire_gpu(b.count) >= target) break;
      if ((it & 1023) == 1023) {
        const unsigned long long t = gtime_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > b.wait_ns) { atomicExch(b.err, 1); ok = 0; break; }
        if (*(volatile int*)b.err) { ok = 0; break; }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sums of two values over the block (at most 8 warps) with one barrier: warp
// partials go to rb[par] and every thread adds them in the same order.  The
// caller alternates par between consecutive calls, so a call never overwrites
// partials that threads may still be reading from the previous one.
__device__ __forceinline__ void block_sum2_1b(R& a, R& b, R (*rb)[2][8], int par) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { rb[par][0][threadIdx.x >> 5] = a; rb[par][1][threadIdx.x >> 5] = b; }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  a = R(0);
  b = R(0);
  for (int w = 0; w < nw; ++w) { a += rb[par][0][w]; b += rb[par][1][w]; }
}

// Cholesky of the lower triangle with dropping: a pivot above drop2 (above 0
// without dropping) is kept, else its column is dropped (zero in L, pivot 0; a
// zero pivot without dropping sets *status = 1 + column), which is Gram-Schmidt
// with dropping expressed on the Gram matrix.  Blocked: panels of kCholB columns
// with two grid barriers each instead of one per column.  Per panel every CTA
// loads the diagonal block and factors it in shared memory (right-looking, the
// update of each step spread over the CTA); the rows below are solved against
// it one row per warp (L21 = A21 L11^-+, forward substitution across the
// lanes); after the barrier CTA 0 writes L11 and the pivots, and every warp
// takes (row, 32 columns) units of the trailing update A22 -= L21 L21^+; a
// second barrier closes the panel.
// The arithmetic is FP64 (R), spread over the grid for the trailing update,
// whose FP64 work dominates; REAL: zero imaginary parts (the k = 0 Gram
// matrices), a quarter of it.  The upper triangle is zeroed at the end.
constexpr int kCholB = 32;

template <bool REAL>
__global__ void __launch_bounds__(256) k_chol_blocked(z* A, int n, int lda, R drop2, int allow_drop,
                                                      R* piv, int* status, GridBar bar) {
  __shared__ z D[kCholB][kCholB + 1];   // diagonal block -> L11 (lower)
  __shared__ R sd[kCholB], sdi[kCholB];  // its pivots (0: dropped) and their reciprocals
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int gw = c * nwarp + warp, nw = G * nwarp;
  unsigned nbar = 0;
  for (int j0 = 0; j0 < n; j0 += kCholB) {
    const int b = min(kCholB, n - j0), j1 = j0 + b, m = n - j1;
    for (int t = tid; t < b * b; t += nt) {
      const int r = t / b, q = t % b;
      D[r][q] = q <= r ? ldz(&A[(size_t)(j0 + r) * lda + j0 + q]) : z{R(0), R(0)};
    }
    __syncthreads();
    // the diagonal block, right-looking: one thread forms the pivot and its
    // reciprocal, the CTA updates the rest of the block from the unscaled column
    // (l_q l_k^+ = a_qj conj(a_kj) / d), then scales the column
    for (int j = 0; j < b; ++j) {
      if (tid == 0) {
        const R d = D[j][j].x;
        const bool keep = allow_drop ? (d > drop2) : (d > R(0));
        const R p = keep ? sqrt(d) : R(0);
        D[j][j] = {p, R(0)};
        sd[j] = p;
        sdi[j] = keep ? R(1) / p : R(0);
      }
      __syncthreads();
      const R inv = sdi[j];
      const int m = b - j - 1;
      if (inv > R(0)) {
        for (int t = tid; t < m * m; t += nt) {
          const int q = j + 1 + t / m, k = j + 1 + t % m;
          if (k > q) continue;
          const z aq = D[q][j], ak = D[k][j];
          const R i2 = inv * inv;
          z& a = D[q][k];
          if (REAL) {
            a.x = fmar(-aq.x * i2, ak.x, a.x);
          } else {   // a -= aq conj(ak) / d
            const z lq = {aq.x * i2, aq.y * i2};
            a.x = fmar(-lq.x, ak.x, fmar(-lq.y, ak.y, a.x));
            a.y = fmar(-lq.y, ak.x, fmar(lq.x, ak.y, a.y));
          }
        }
      }
      __syncthreads();
      for (int q = j + 1 + tid; q < b; q += nt) {
        const z a = D[q][j];
        D[q][j] = inv > R(0) ? z{a.x * inv, REAL ? R(0) : a.y * inv} : z{R(0), R(0)};
      }
    }
    __syncthreads();
    // L21: row r solves l_r L11^+ = a_r; lane q carries column j0 + q
    for (int r = j1 + gw; r < n; r += nw) {
      z a = lane < b ? ldz(&A[(size_t)r * lda + j0 + lane]) : z{R(0), R(0)};
      for (int j = 0; j < b; ++j) {
        const R p = sd[j], inv = sdi[j];
        const z aj = {__shfl_sync(0xffffffffu, a.x, j), REAL ? R(0) : __shfl_sync(0xffffffffu, a.y, j)};
        const z lj = p > R(0) ? z{aj.x * inv, REAL ? R(0) : aj.y * inv} : z{R(0), R(0)};
        if (lane == j) a = lj;
        if (lane > j && lane < b && p > R(0)) {   // a_q -= l_j conj(L11[q][j])
          const z lq = D[lane][j];
          if (REAL) {
            a.x = fmar(-lj.x, lq.x, a.x);
          } else {
            a.x = fmar(-lj.x, lq.x, fmar(-lj.y, lq.y, a.x));
            a.y = fmar(-lj.y, lq.x, fmar(lj.x, lq.y, a.y));
          }
        }
      }
      if (lane < b) A[(size_t)r * lda + j0 + lane] = a;
    }
    if (!grid_sync_mono(bar, ++nbar)) return;
    if (c == 0) {
      for (int t = tid; t < b * b; t += nt) {
        const int r = t / b, q = t % b;
        if (q <= r) A[(size_t)(j0 + r) * lda + j0 + q] = D[r][q];
      }
      for (int j = tid; j < b; j += nt) {
        piv[j0 + j] = sd[j];
        const bool keep = sd[j] > R(0);
        if (!keep && !allow_drop) *status = 1 + j0 + j;
      }
    }
    // trailing update: unit (row r, columns q0 .. q0 + 31) of the lower triangle
    const int nch = (m + 31) / 32;
    for (int u = gw; u < m * nch; u += nw) {   // uniform per warp
      const int r = j1 + u / nch, q0 = j1 + 32 * (u % nch);
      if (q0 > r) continue;
      const int q = q0 + lane;
      const bool act = q <= r;
      const z lr = lane < b ? ldz(&A[(size_t)r * lda + j0 + lane]) : z{R(0), R(0)};
      const z* lqp = A + (size_t)(act ? q : r) * lda + j0;
      // the lane's row of L21, all loads issued before the first use
      z lq[kCholB];
#pragma unroll
      for (int k = 0; k < kCholB; ++k) lq[k] = (act && k < b) ? ldz(lqp + k) : z{R(0), R(0)};
      z acc = {R(0), R(0)};
#pragma unroll
      for (int k = 0; k < kCholB; ++k) {   // acc = sum_k l_rk conj(l_qk)
        const R rx = __shfl_sync(0xffffffffu, lr.x, k);
        const R ry = REAL ? R(0) : __shfl_sync(0xffffffffu, lr.y, k);
        if (REAL) {
          acc.x = fmar(rx, lq[k].x, acc.x);
        } else {
          acc.x = fmar(rx, lq[k].x, fmar(ry, lq[k].y, acc.x));
          acc.y = fmar(ry, lq[k].x, fmar(-rx, lq[k].y, acc.y));
        }
      }
      if (act) {
        z* a = &A[(size_t)r * lda + q];
        const z av = ldz(a);
        *a = {av.x - acc.x, REAL ? R(0) : av.y - acc.y};
      }
    }
    if (!grid_sync_mono(bar, ++nbar)) return;
  }
  const size_t total = (size_t)n * n;
  const size_t nthr = (size_t)G * nt, gtid = (size_t)c * nt + tid;
  for (size_t t = gtid; t < total; t += nthr) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j > i) A[(size_t)i * lda + j] = {R(0), R(0)};
  }
}

// ---- Cholesky ------------------------------------------------------------------
static int coop_blocks(const void* f, size_t work_items, size_t smem = 0) {
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, 256, smem);
  // one CTA per SM at most: fewer arrivals per grid barrier
  const int cap = std::max(1, nsm * std::max(1, std::min(occ, 1)));
  const int want = (int)std::max<size_t>(1, (work_items + 4095) / 4096);
  return std::min(cap, want);
}

static int launch_coop(const void* f, int blocks, void** args, cudaStream_t st, const char* what,
                       size_t smem = 0, int threads = 256) {
  cudaError_t e = cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(threads), args, smem, st);
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

int cholesky(z* A, int n, int lda, R drop2, bool allow_drop, R* piv, int* status,
             GridBar bar, cudaStream_t st, bool real_sym) {
  if (n <= 0) return QE_OK;
  if (cudaMemsetAsync(bar.count, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
    set_error("cholesky: memset failed");
    return QE_ECUDA;
  }
  int allow = allow_drop ? 1 : 0;
  void* args[] = {&A, &n, &lda, &drop2, &allow, &piv, &status, &bar};
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM at most; ~256 elements of the lower triangle per CTA, so that
  // the FP64 work of the trailing updates spreads over the SMs
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>(nsm, ((size_t)n * n / 2 + 255) / 256));
  const void* f = real_sym ? (const void*)k_chol_blocked<true> : (const void*)k_chol_blocked<false>;
  return launch_coop(f, blocks, args, st, "k_chol_blocked");
}

// ---- triangular solves ---------------------------------------------------------
constexpr int TCOLS = 4;

// L X = B, L lower with real positive diagonal, given as its transpose LT
// (LT[i][r] = L[r][i], so that column i of L is a contiguous row); B [n][ldb],
// columns c0.. of this CTA.
__global__ void __launch_bounds__(256) k_trsm_lower_t(const z* LT, int n, int ldt, z* B, int ldb,
                                                      int ncols) {
  const int c0 = blockIdx.x * TCOLS;
  const int nc = min(TCOLS, ncols - c0);
  for (int i = 0; i < n; ++i) {
    const z* lcol = LT + (size_t)i * ldt;
    if (threadIdx.x < nc) {
      const R inv = R(1) / lcol[i].x;
      z& b = B[(size_t)i * ldb + c0 + threadIdx.x];
      b = {b.x * inv, b.y * inv};
    }
    __syncthreads();
    const int rows = n - i - 1;
    for (int t = threadIdx.x; t < rows * nc; t += blockDim.x) {
      const int r = i + 1 + t / nc, c = c0 + t % nc;
      const z l = lcol[r], x = B[(size_t)i * ldb + c];
      z& b = B[(size_t)r * ldb + c];
      b.x -= l.x * x.x - l.y * x.y;
      b.y -= l.x * x.y + l.y * x.x;
    }
    __syncthreads();
  }
}

// L^+ X = B (back substitution with the conjugate transpose of lower L).
__global__ void __launch_bounds__(256) k_trsm_upper_h(const z* L, int n, int ldl, z* B, int ldb,
                                                      int ncols) {
  const int c0 = blockIdx.x * TCOLS;
  const int nc = min(TCOLS, ncols - c0);
  for (int i = n - 1; i >= 0; --i) {
    if (threadIdx.x < nc) {
      const R inv = R(1) / L[(size_t)i * ldl + i].x;
      z& b = B[(size_t)i * ldb + c0 + threadIdx.x];
      b = {b.x * inv, b.y * inv};
    }
    __syncthreads();
    for (int t = threadIdx.x; t < i * nc; t += blockDim.x) {
      const int r = t / nc, c = c0 + t % nc;
      // (L^+)[r][i] = conj(L[i][r])
      const z l = L[(size_t)i * ldl + r], x = B[(size_t)i * ldb + c];
      z& b = B[(size_t)r * ldb + c];
      b.x -= l.x * x.x + l.y * x.y;
      b.y -= l.x * x.y - l.y * x.x;
    }
    __syncthreads();
  }
}

// L^+ X = B for one column of B per CTA (n <= kTrsmRows * 256): the column lives
// in registers (row r in thread r mod 256), x_i goes through shared memory, and
// each thread prefetches its entries of the next row of L during a step, so a
// step is one block barrier, not an L2 round trip.  REAL: zero imaginary parts.
constexpr int kTrsmRows = 4;

template <bool REAL>
__global__ void __launch_bounds__(256) k_trsm_upper_h_col(const z* L, int n, int ldl, z* B, int ldb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* sx = reinterpret_cast<z*>(smem_raw);   // x_i, n
  const int col = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  z b[kTrsmRows], lcur[kTrsmRows];
#pragma unroll
  for (int k = 0; k < kTrsmRows; ++k) {
    const int r = tid + k * nt;
    b[k] = r < n ? B[(size_t)r * ldb + col] : z{R(0), R(0)};
    lcur[k] = r < n ? ldz(&L[(size_t)(n - 1) * ldl + r]) : z{R(0), R(0)};
  }
  for (int i = n - 1; i >= 0; --i) {
    z lnx[kTrsmRows];
#pragma unroll
    for (int k = 0; k < kTrsmRows; ++k) {   // L[i-1][r], r <= i - 1
      const int r = tid + k * nt;
      lnx[k] = (i > 0 && r < i) ? ldz(&L[(size_t)(i - 1) * ldl + r]) : z{R(0), R(0)};
    }
#pragma unroll
    for (int k = 0; k < kTrsmRows; ++k)
      if (tid + k * nt == i) {   // the owner of row i: x_i = b_i / L_ii
        const R inv = R(1) / lcur[k].x;
        b[k] = {b[k].x * inv, REAL ? R(0) : b[k].y * inv};
        sx[i] = b[k];
      }
    __syncthreads();
    const z x = sx[i];
#pragma unroll
    for (int k = 0; k < kTrsmRows; ++k) {
      if (tid + k * nt < i) {   // b_r -= conj(L[i][r]) x_i
        const z l = lcur[k];
        if (REAL) {
          b[k].x = fmar(-l.x, x.x, b[k].x);
        } else {
          b[k].x = fmar(-l.x, x.x, fmar(-l.y, x.y, b[k].x));
          b[k].y = fmar(-l.x, x.y, fmar(l.y, x.x, b[k].y));
        }
      }
      lcur[k] = lnx[k];
    }
  }
#pragma unroll
  for (int k = 0; k < kTrsmRows; ++k) {
    const int r = tid + k * nt;
    if (r < n) B[(size_t)r * ldb + col] = b[k];
  }
}

int trsm_lower_t(const z* LT, int n, int ldt, z* B, int ldb, int ncols, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return QE_OK;
  k_trsm_lower_t<<<(ncols + TCOLS - 1) / TCOLS, 256, 0, st>>>(LT, n, ldt, B, ldb, ncols);
  return check_launch("k_trsm_lower_t");
}

int trsm_upper_h(const z* L, int n, int ldl, z* B, int ldb, int ncols, cudaStream_t st,
                 bool real_sym) {
  if (n <= 0 || ncols <= 0) return QE_OK;
  if (n <= kTrsmRows * 256) {
    const size_t sm = (size_t)n * sizeof(z);
    if (real_sym)
      k_trsm_upper_h_col<true><<<ncols, 256, sm, st>>>(L, n, ldl, B, ldb);
    else
      k_trsm_upper_h_col<false><<<ncols, 256, sm, st>>>(L, n, ldl, B, ldb);
    return check_launch("k_trsm_upper_h_col");
  }
  k_trsm_upper_h<<<(ncols + TCOLS - 1) / TCOLS, 256, 0, st>>>(L, n, ldl, B, ldb, ncols);
  return check_launch("k_trsm_upper_h");
}

// ---- element-wise helpers ------------------------------------------------------
// dst[i][j] = src[j][i]
__global__ void k_transpose(const z* src, int lds, z* dst, int ldd, int rows, int cols) {
  __shared__ z tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    if (i < rows && j < cols) tile[r][threadIdx.x] = src[(size_t)i * lds + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = c0 + r, i = r0 + threadIdx.x;
    if (i < rows && j < cols) dst[(size_t)j * ldd + i] = tile[threadIdx.x][r];
  }
}

int transpose(const z* src, int lds, z* dst, int ldd, int rows, int cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return QE_OK;
  dim3 g((cols + 31) / 32, (rows + 31) / 32);
  k_transpose<<<g, dim3(32, 8), 0, st>>>(src, lds, dst, ldd, rows, cols);
  return check_launch("k_transpose");
}

// dst[i][j] = conj(src[j][i])
__global__ void k_conj_transpose(const z* src, int lds, z* dst, int ldd, int rows, int cols) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / cols), j = (int)(t % cols);   // dst row i, col j
    dst[(size_t)i * ldd + j] = zconj(src[(size_t)j * lds + i]);
  }
}

// A = (A + A^+) / 2 in place
__global__ void k_hermitize(z* A, int n, int lda) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j < i) continue;
    const z a = A[(size_t)i * lda + j], b = A[(size_t)j * lda + i];
    const z m = {R(0.5) * (a.x + b.x), R(0.5) * (a.y - b.y)};
    A[(size_t)i * lda + j] = m;
    A[(size_t)j * lda + i] = zconj(m);
  }
}

int conj_transpose(const z* src, int lds, z* dst, int ldd, int rows, int cols, cudaStream_t st) {
  const size_t total = (size_t)rows * cols;
  if (!total) return QE_OK;
  k_conj_transpose<<<(int)std::min<size_t>((total + 255) / 256, 152 * 8), 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
  return check_launch("k_conj_transpose");
}

int hermitize(z* A, int n, int lda, cudaStream_t st) {
  const size_t total = (size_t)n * n;
  if (!total) return QE_OK;
  k_hermitize<<<(int)std::min<size_t>((total + 255) / 256, 152 * 8), 256, 0, st>>>(A, n, lda);
  return check_launch("k_hermitize");
}

// ---- Householder reflectors ----------------------------------------------------------
// Step j: H = I - tau v v^+, v_0 = 1, H^+ x = beta e_1 with beta real, where x is
// column j below the diagonal; v_1.. are stored in A[j+2 ..][j] and, for the
// back-transformation, in row j of refl; A[j+1][j] = beta.
// Reflector of step j from the updated column j (rows j+1 ..), computed by one
// CTA: v_1.. to A[j+2 ..][j] and vbuf[1 ..], beta to A[j+1][j] and e[j], tau[j].
__device__ void house_step(z* A, int n, int lda, int j, z* tau, R* e, z* vbuf, z* refl,
                           R* sh) {
  const int m = n - j - 1;
  const z alpha = ldz(&A[(size_t)(j + 1) * lda + j]);
  R s = R(0);
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) s += zabs2(ldz(&A[(size_t)(j + 1 + i) * lda + j]));
  const R sigma = block_sum(s, sh);
  if (sigma == R(0) && alpha.y == R(0)) {
    if (threadIdx.x == 0) { tau[j] = {R(0), R(0)}; e[j] = alpha.x; }
    return;
  }
  const R nu = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + sigma);
  const R beta = alpha.x >= R(0) ? -nu : nu;
  const z am = {alpha.x - beta, alpha.y};
  const R den = am.x * am.x + am.y * am.y;
  const z sc = {am.x / den, -am.y / den};
  z* rrow = refl + (size_t)j * n + (j + 1);
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
    z* x = &A[(size_t)(j + 1 + i) * lda + j];
    const z v = cmul(ldz(x), sc);
    *x = v;
    vbuf[i] = v;
    rrow[i] = v;
  }
  if (threadIdx.x == 0) {
    tau[j] = {(beta - alpha.x) / beta, -alpha.y / beta};
    e[j] = beta;
    A[(size_t)(j + 1) * lda + j] = {beta, R(0)};
    vbuf[0] = {R(1), R(0)};
    rrow[0] = {R(1), R(0)};
  }
}

// Householder tridiagonalisation, all steps in one launch, two barriers per
// step: (matvec p = tau A v) | (rank-2 update A -= v w^+ + w v^+, and, in CTA 0,
// the update of the next column followed by the next reflector).  The
// reflector is also kept contiguous in vbuf; every CTA stages v and w of the
// step in shared memory, so the two phases stream only the trailing block of A.
// Dynamic shared memory: 2 n complex.
__global__ void __launch_bounds__(256) k_tridiag_coop(z* A, int n, int lda, z* tau, R* e, z* p,
                                                      R* dg, z* vbuf, z* refl, GridBar bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* sv = reinterpret_cast<z*>(smem_raw);
  z* sw = sv + n;
  __shared__ R sh[33];
  const size_t nthr = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nwarp = (int)(nthr >> 5), gwarp = (int)(gtid >> 5), lane = threadIdx.x & 31;
  if (n >= 2 && blockIdx.x == 0) house_step(A, n, lda, 0, tau, e, vbuf, refl, sh);
  if (!grid_sync(bar)) return;
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;
    const z t = ldz(&tau[j]);
    const bool active = t.x != R(0) || t.y != R(0);
    if (active) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = ldz(&vbuf[i]);
      __syncthreads();
      // p = tau A v over the trailing block (one warp per row; four loads in
      // flight per lane: the row is read from L2, latency-bound otherwise)
      for (int w = gwarp; w < m; w += nwarp) {
        const z* row = A + (size_t)(j + 1 + w) * lda + (j + 1);
        z acc = {R(0), R(0)}, acc1 = {R(0), R(0)};
        int c = lane;
        for (; c + 96 < m; c += 128) {
          const z a0 = ldz(row + c), a1 = ldz(row + c + 32), a2 = ldz(row + c + 64), a3 = ldz(row + c + 96);
          acc = cadd(acc, cmul(a0, sv[c]));
          acc1 = cadd(acc1, cmul(a1, sv[c + 32]));
          acc = cadd(acc, cmul(a2, sv[c + 64]));
          acc1 = cadd(acc1, cmul(a3, sv[c + 96]));
        }
        for (; c < m; c += 32) acc = cadd(acc, cmul(ldz(row + c), sv[c]));
        acc = cadd(acc, acc1);
        for (int o = 16; o > 0; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) p[j + 1 + w] = cmul(t, acc);
      }
    }
    if (!grid_sync(bar)) return;
    if (active) {
      // w = p - (1/2) conj(tau) (v^+ p) v
      R sr = R(0), si = R(0);
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const z v = sv[i], pr = ldz(&p[j + 1 + i]);
        sw[i] = pr;
        sr += v.x * pr.x + v.y * pr.y;
        si += v.x * pr.y - v.y * pr.x;
      }
      const R vpr = block_sum(sr, sh);
      const R vpi = block_sum(si, sh);
      const z coef = {R(0.5) * (t.x * vpr + t.y * vpi), R(0.5) * (t.x * vpi - t.y * vpr)};
      for (int i = threadIdx.x; i < m; i += blockDim.x) sw[i] = csub(sw[i], cmul(coef, sv[i]));
      __syncthreads();
      // all columns but the first of the trailing block, one warp per row, by the
      // CTAs other than 0 (CTA 0 meanwhile updates that first column and builds
      // the next reflector, the critical path of the step)
      if (m > 1 && (gridDim.x == 1 || blockIdx.x > 0)) {
        const int wpb = (int)(blockDim.x >> 5);
        const int bw = gridDim.x == 1 ? gwarp : gwarp - wpb;
        const int nbw = gridDim.x == 1 ? nwarp : nwarp - wpb;
        for (int r = bw; r < m; r += nbw) {
          const z vr = sv[r], wr = sw[r];
          z* arow = A + (size_t)(j + 1 + r) * lda + (j + 1);
          int c = 1 + lane;
          for (; c + 32 < m; c += 64) {
            const z a0 = ldz(arow + c), a1 = ldz(arow + c + 32);
            const z d0 = cadd(cmul(vr, zconj(sw[c])), cmul(wr, zconj(sv[c])));
            const z d1 = cadd(cmul(vr, zconj(sw[c + 32])), cmul(wr, zconj(sv[c + 32])));
            arow[c] = csub(a0, d0);
            arow[c + 32] = csub(a1, d1);
          }
          for (; c < m; c += 32) {
            const z dlt = cadd(cmul(vr, zconj(sw[c])), cmul(wr, zconj(sv[c])));
            arow[c] = csub(ldz(arow + c), dlt);
          }
        }
      }
    }
    if (blockIdx.x == 0 && j + 1 < n - 1) {
      if (active) {
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          const z dlt = cadd(cmul(sv[r], zconj(sw[0])), cmul(sw[r], zconj(sv[0])));
          z* a = &A[(size_t)(j + 1 + r) * lda + (j + 1)];
          *a = csub(ldz(a), dlt);
        }
        __syncthreads();
      }
      house_step(A, n, lda, j + 1, tau, e, vbuf, refl, sh);
    } else if (blockIdx.x == 0 && active) {
      // last step: only the 1 x 1 trailing element remains
      for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const z dlt = cadd(cmul(sv[r], zconj(sw[0])), cmul(sw[r], zconj(sv[0])));
        z* a = &A[(size_t)(j + 1 + r) * lda + (j + 1)];
        *a = csub(ldz(a), dlt);
      }
    }
    if (!grid_sync(bar)) return;
  }
  for (size_t i = gtid; i < (size_t)n; i += nthr) dg[i] = ldz(&A[i * lda + i]).x;
}

// Householder tridiagonalisation (the same reflectors as k_tridiag_coop) with the
// matrix held in the CTAs' shared memory: CTA c owns rows c, c + G, c + 2G, ...
// (cyclic, so the shrinking trailing block stays evenly spread).  Every CTA
// forms each reflector itself from the published column, so a step needs one
// grid barrier: before it, the owners publish p_r = tau (A v)_r of their rows
// and their entries of the next column; after it, every CTA reads both, forms
// w = p - (1/2) conj(tau) (v^+ p) v, applies A -= v w^+ + w v^+ to its own rows
// and to the next column, and builds the next reflector from that column.  All
// CTAs reach bit-identical reflectors (same inputs, same reduction order).
// Global A is read once at the start; its rows 0..3 then hold the exchange
// vectors (p and the column, two parities).  Needs n >= 4 and at most
// kTridRows rows per CTA.  Dynamic shared memory: (ceil(n / G) + 3) n complex.
constexpr int kTridRows = 8;

#if !defined(QE_DENSE_FP64)   // FP64: k_tridiag_rows_ff below
__global__ void __launch_bounds__(256) k_tridiag_rows(z* A, int n, int lda, z* tau, R* e, R* dg,
                                                      z* refl, GridBar bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int nrmax = (n + G - 1) / G;
  const int nr = c < n ? (n - 1 - c) / G + 1 : 0;   // rows owned: c + q G, q < nr
  z* rows = reinterpret_cast<z*>(smem_raw);          // nrmax x n
  z* sv = rows + (size_t)nrmax * n;                  // reflector v (index i <-> row j+1+i)
  z* sw = sv + n;                                    // p, then w
  z* sx = sw + n;                                    // column to reduce (index i <-> row j+1+i)
  __shared__ R rb[2][2][8];
  __shared__ z spart[8][kTridRows];
  for (int q = 0; q < nr; ++q) {
    const z* src = A + (size_t)(c + q * G) * lda;
    for (int k = tid; k < n; k += nt) rows[(size_t)q * n + k] = ldz(src + k);
  }
  for (int i = tid; i < n - 1; i += nt) sx[i] = ldz(&A[(size_t)(1 + i) * lda]);
  if (c == 0 && tid == 0) dg[0] = ldz(&A[0]).x;
  // every CTA has read A: its rows 0..3 become the exchange vectors
  if (!grid_sync_mono(bar, 1)) return;
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - 1 - j, par = j & 1;
    z* xp = A + (size_t)(2 * par) * lda;       // p_r at [r]
    z* xc = A + (size_t)(2 * par + 1) * lda;   // A[r][j+1] at [r], r >= j+2
    // reflector of step j from sx[0..m)
    const z alpha = sx[0];
    R s = R(0);
    for (int i = 1 + tid; i < m; i += nt) s = fmar(sx[i].x, sx[i].x, fmar(sx[i].y, sx[i].y, s));
    R sigma = s, unused = R(0);
    block_sum2_1b(sigma, unused, rb, 0);
    z t;
    R beta;
    if (sigma == R(0) && alpha.y == R(0)) {
      t = {R(0), R(0)};
      beta = alpha.x;
      for (int i = tid; i < m; i += nt) sv[i] = {i == 0 ? R(1) : R(0), R(0)};
    } else {
      const R nu = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + sigma);
      beta = alpha.x >= R(0) ? -nu : nu;
      const z am = {alpha.x - beta, alpha.y};
      const R rden = R(1) / (am.x * am.x + am.y * am.y), rbeta = R(1) / beta;
      const z sc = {am.x * rden, -am.y * rden};
      t = {(beta - alpha.x) * rbeta, -alpha.y * rbeta};
      for (int i = tid; i < m; i += nt) sv[i] = i == 0 ? z{R(1), R(0)} : cmul(sx[i], sc);
    }
    __syncthreads();
    if (c == 0) {
      z* rrow = refl + (size_t)j * n + (j + 1);
      for (int i = tid; i < m; i += nt) rrow[i] = sv[i];
      if (tid == 0) { tau[j] = t; e[j] = beta; }
    }
    // p = tau A v on the owned rows of the trailing block (r >= j+1): every warp
    // takes 32-column chunks of all those rows, partial sums meet in spart
    const int q0 = c >= j + 1 ? 0 : (j + 1 - c + G - 1) / G;
    const int nq = nr - q0;
    if (nq > 0) {
      z acc[kTridRows];
#pragma unroll
      for (int q = 0; q < kTridRows; ++q) acc[q] = {R(0), R(0)};
      for (int k = warp * 32 + lane; k < m; k += nwarp * 32) {
        const z vk = sv[k];
        const z* base = rows + (size_t)q0 * n + (j + 1) + k;
#pragma unroll
        for (int q = 0; q < kTridRows; ++q)
          if (q < nq) acc[q] = zfma(base[(size_t)q * n], vk, acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kTridRows; ++q) {
        if (q < nq) {
          z a = acc[q];
          for (int o = 16; o > 0; o >>= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
          }
          if (lane == 0) spart[warp][q] = a;
        }
      }
    }
    __syncthreads();
    if (tid < nq) {
      z a = {R(0), R(0)};
      for (int w = 0; w < nwarp; ++w) a = cadd(a, spart[w][tid]);
      const int q = q0 + tid, r = c + q * G;
      xp[r] = cmul(t, a);
      if (r >= j + 2) xc[r] = rows[(size_t)q * n + (j + 1)];
    }
    if (!grid_sync_mono(bar, (unsigned)j + 2)) return;
    // w = p - (1/2) conj(tau) (v^+ p) v; the next column (rows j+2 ..)
    R sr = R(0), si = R(0);
    for (int i = tid; i < m; i += nt) {
      const z v = sv[i], pr = ldz(&xp[j + 1 + i]);
      sw[i] = pr;
      sr = fmar(v.x, pr.x, fmar(v.y, pr.y, sr));
      si = fmar(v.x, pr.y, fmar(-v.y, pr.x, si));
    }
    for (int i = tid; i < m - 1; i += nt) sx[i] = ldz(&xc[j + 2 + i]);
    block_sum2_1b(sr, si, rb, 1);
    const z coef = {R(0.5) * (t.x * sr + t.y * si), R(0.5) * (t.x * si - t.y * sr)};
    const z ncoef = {-coef.x, -coef.y};
    for (int i = tid; i < m; i += nt) sw[i] = zfma(ncoef, sv[i], sw[i]);
    __syncthreads();
    // A -= v w^+ + w v^+ on the owned rows, and on the next column
    for (int q = q0; q < nr; ++q) {
      const int kr = c + q * G - (j + 1);
      const z vr = sv[kr], wr = sw[kr];
      z* arow = rows + (size_t)q * n + (j + 1);
      for (int k = tid; k < m; k += nt) {
        const z a = zrank2(arow[k], vr, sw[k], wr, sv[k]);
        arow[k] = a;
        if (kr == 0 && k == 0) dg[j + 1] = a.x;
      }
    }
    {
      // v_0 = 1: x_i - v_{i+1} conj(w_0) - w_{i+1}
      const z w0 = sw[0];
      for (int i = tid; i < m - 1; i += nt) {
        const z v = sv[i + 1], w = sw[i + 1];
        z x = {sx[i].x - w.x, sx[i].y - w.y};
        x.x = fmar(-v.x, w0.x, x.x);
        x.x = fmar(-v.y, w0.y, x.x);
        x.y = fmar(-v.y, w0.x, x.y);
        x.y = fmar(v.x, w0.y, x.y);
        sx[i] = x;
      }
    }
    __syncthreads();   // the next reflector reads all of sx
  }
}
#endif


// ---- tridiagonal eigenvalues: Sturm bisection, one thread per eigenvalue --------
// Number of eigenvalues of T below x (Sturm sequence in the ratio form, e2 the
// squared off-diagonal); a zero pivot counts as -tiny.
template <typename F>
__device__ int sturm_count(const F* d, const F* e2, int n, F x, F tiny) {
  int cnt = 0;
  F q = d[0] - x;
  if (q == F(0)) q = -tiny;
  if (q < F(0)) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (q == F(0)) q = -tiny;
    if (q < F(0)) ++cnt;
  }
  return cnt;
}

// Multisection rounds on [lo, hi] for the (k+1)-th eigenvalue until the bracket
// is below `width` (or stops shrinking): the 32 lanes count at 32 interior
// points and the bracket shrinks to the sub-interval holding it (a factor 33
// per round instead of 2 for bisection).
template <typename F>
__device__ void multisect(const F* d, const F* e2, int n, int k, F tiny, F& lo, F& hi,
                          F rel, F width) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= width || hi - lo <= rel * fmax(fabs(lo), fabs(hi))) break;
    const F step = (hi - lo) / F(33);
    const F x = lo + step * (lane + 1);
    const int c = (x > lo && x < hi) ? sturm_count(d, e2, n, x, tiny) : (x <= lo ? 0 : n);
    // lanes whose point has more than k eigenvalues below it bound from above
    const unsigned above = __ballot_sync(0xffffffffu, c > k);
    const int first = above ? __ffs(above) - 1 : 32;    // first lane with count > k
    const F nlo = first == 0 ? lo : lo + step * first;
    const F nhi = first == 32 ? hi : lo + step * (first + 1);
    if (!(nhi < hi || nlo > lo)) break;                 // no progress at this resolution
    lo = nlo;
    hi = nhi;
  }
}

// ---- float-float Sturm counts (the FP64 bisection's final rounds) ---------------------
// GB300 runs FP64 at 1/64 of its FP32 rate and the Sturm recurrence is a chain of
// dependent divisions, so its FP64 rounds are latency-bound at the FP64 pipe's
// pace.  Float-float (ff.cuh: hi + lo floats, 48-bit significand, normalised
// here) counts with a backward error of a few units of 2^-47 ||T||, resolving
// eigenvalues to ~1e-14 ||T||; the division takes an approximate quotient of the
// high parts and one correction from the exact remainder (~2^-44 relative).
__device__ __forceinline__ ff ffs_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return ff(h, __fsub_rn(e, __fsub_rn(h, s)));
}
// a - b (Knuth's two-sum of a.hi and -b.hi, then the low parts)
__device__ __forceinline__ ff ffs_sub(ff a, ff b) {
  const float s = __fsub_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fadd_rn(b.hi, v));
  return ffs_norm(s, __fadd_rn(e, __fsub_rn(a.lo, b.lo)));
}
// a / b
__device__ __forceinline__ ff ffs_div(ff a, ff b) {
  const float r = __fdividef(a.hi, b.hi);
  const float p = __fmul_rn(r, b.hi);
  const float pe = __fmaf_rn(r, b.lo, __fmaf_rn(r, b.hi, -p));   // r b = p + pe
  const ff d = ffs_sub(a, ff(p, pe));                              // the remainder a - r b
  return ffs_norm(r, __fdividef(d.hi, b.hi));
}
__device__ int sturm_count_ff(const ff* d, const ff* e2, int n, ff x, float tiny) {
  int cnt = 0;
  ff q = ffs_sub(d[0], x);
  if (q.hi == 0.f) q = ff(-tiny, 0.f);
  if (q.hi < 0.f) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = ffs_sub(ffs_sub(d[i], x), ffs_div(e2[i - 1], q));
    if (q.hi == 0.f) q = ff(-tiny, 0.f);
    if (q.hi < 0.f) ++cnt;
  }
  return cnt;
}
// multisect with float-float counts on a double bracket, down to `width`
__device__ void multisect_ff(const ff* d, const ff* e2, int n, int k, float tiny, double& lo,
                             double& hi, double width) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= width) break;
    const double step = (hi - lo) / 33.0;
    const double x = lo + step * (lane + 1);
    const int c = (x > lo && x < hi) ? sturm_count_ff(d, e2, n, ff(x), tiny) : (x <= lo ? 0 : n);
    const unsigned above = __ballot_sync(0xffffffffu, c > k);
    const int first = above ? __ffs(above) - 1 : 32;
    const double nlo = first == 0 ? lo : lo + step * first;
    const double nhi = first == 32 ? hi : lo + step * (first + 1);
    if (!(nhi < hi || nlo > lo)) break;
    lo = nlo;
    hi = nhi;
  }
}

#if defined(QE_DENSE_FP64)
// ---- the FP64 tridiagonalisation in float-float arithmetic ---------------------------
// k_tridiag_rows with every value a packed float-float complex number (ff.cuh:
// lanes (re, im), hi and lo pairs; 48-bit significands) instead of complex
// double: the same rows, exchange vectors, barriers and reflectors, with the
// FP64 pipe's work (12 FMAs per element and step) moved to the FP32 pipes.  The
// reduction's backward error is a few units of 2^-46 ||A|| instead of 2^-53,
// ~1e-14 ||A||, far below the 1e-10 eigenvalue tolerance of the FP64 solves;
// d, e and tau leave in double, the reflector rows packed float-float (for
// k_wy_t_ff and k_backtransform_ff, the back-transformation in the same
// arithmetic).
// exchange vectors written by other CTAs: read through L2 (as ldz)
__device__ __forceinline__ ff2 pk_load(const z* p) {
  const ulonglong2 u = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  return {{u.x}, {u.y}};
}
__device__ __forceinline__ void pk_store(z* p, ff2 a) { *reinterpret_cast<cx<ff>*>(p) = of2(a); }
__device__ __forceinline__ ff2 pk_re(ff2 a) {   // (re, re)
  float rh, ih, rl, il;
  f2_split(a.hi, rh, ih);
  f2_split(a.lo, rl, il);
  return {f2_of(rh, rh), f2_of(rl, rl)};
}
__device__ __forceinline__ ff2 pk_im(ff2 a) {   // (im, im)
  float rh, ih, rl, il;
  f2_split(a.hi, rh, ih);
  f2_split(a.lo, rl, il);
  return {f2_of(ih, ih), f2_of(il, il)};
}
__device__ __forceinline__ ff2 pk_i(ff2 a) { return {neg2_0(swap2(a.hi)), neg2_0(swap2(a.lo))}; }   // i a
__device__ __forceinline__ ff2 pk_conj(ff2 a) { return {neg2_1(a.hi), neg2_1(a.lo)}; }
__device__ __forceinline__ ff2 pk_neg(ff2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ ff2 pk_zero() { return {f2_of(0.f, 0.f), f2_of(0.f, 0.f)}; }
// acc + a b (complex): re(a) b + im(a) (i b) + acc
__device__ __forceinline__ ff2 pk_fma(ff2 a, ff2 b, ff2 acc) {
  return fma(pk_im(a), pk_i(b), fma(pk_re(a), b, acc));
}
__device__ __forceinline__ ff2 pk_mul(ff2 a, ff2 b) { return fma(pk_im(a), pk_i(b), pk_re(a) * b); }
__device__ __forceinline__ ff2 pk_shfl_xor(ff2 a, int o) {
  return {{__shfl_xor_sync(0xffffffffu, a.hi.v, o)}, {__shfl_xor_sync(0xffffffffu, a.lo.v, o)}};
}
// block sum (all threads get it; fixed order, so every CTA forms the same value)
__device__ __forceinline__ ff2 pk_block_sum(ff2 a, cx<ff> (*buf)[8], int par) {
  for (int o = 16; o > 0; o >>= 1) a = a + pk_shfl_xor(a, o);   // two-sums exact: same in every lane
  if ((threadIdx.x & 31) == 0) buf[par][threadIdx.x >> 5] = of2(ff2_settle(a));
  __syncthreads();
  ff2 t = as2(buf[par][0]);
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = t + as2(buf[par][w]);
  return ff2_settle(t);
}
// scalar parts and float-float scalar arithmetic (normalised)
__device__ __forceinline__ ff pk_get_re(ff2 a) {
  float rh, ih, rl, il;
  f2_split(a.hi, rh, ih);
  f2_split(a.lo, rl, il);
  return ff(rh, rl);
}
__device__ __forceinline__ ff pk_get_im(ff2 a) {
  float rh, ih, rl, il;
  f2_split(a.hi, rh, ih);
  f2_split(a.lo, rl, il);
  return ff(ih, il);
}
__device__ __forceinline__ ff2 pk_make(ff re, ff im) { return {f2_of(re.hi, im.hi), f2_of(re.lo, im.lo)}; }
__device__ __forceinline__ ff ffs_neg(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff ffs_add(ff a, ff b) { return ffs_sub(a, ffs_neg(b)); }
__device__ __forceinline__ ff ffs_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ffs_norm(p, e);
}
// sqrt(a), a >= 0: float root and one correction from the exact remainder
__device__ __forceinline__ ff ffs_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff(0.f, 0.f);
  const float r = sqrtf(a.hi);
  const float p = __fmul_rn(r, r);
  const float pe = __fmaf_rn(r, r, -p);
  const ff d = ffs_sub(a, ff(p, pe));
  return ffs_norm(r, __fdividef(d.hi, __fmul_rn(2.f, r)));
}
__device__ __forceinline__ double ffs_to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ z pk_to_z(ff2 a) {
  const ff r = pk_get_re(a), i = pk_get_im(a);
  return {ffs_to_d(r), ffs_to_d(i)};
}

__global__ void __launch_bounds__(256) k_tridiag_rows_ff(z* A, int n, int lda, z* tau, R* e,
                                                         R* dg, z* refl, GridBar bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int nrmax = (n + G - 1) / G;
  const int nr = c < n ? (n - 1 - c) / G + 1 : 0;   // rows owned: c + q G, q < nr
  cx<ff>* rows = reinterpret_cast<cx<ff>*>(smem_raw);   // nrmax x n
  cx<ff>* sv = rows + (size_t)nrmax * n;               // reflector v (index i <-> row j+1+i)
  cx<ff>* sw = sv + n;                                 // p, then w
  cx<ff>* sx = sw + n;                                 // column to reduce
  __shared__ cx<ff> rb[2][8];
  __shared__ cx<ff> spart[8][kTridRows];
  for (int q = 0; q < nr; ++q) {
    const z* src = A + (size_t)(c + q * G) * lda;
    for (int k = tid; k < n; k += nt) {
      const z a = ldz(src + k);
      rows[(size_t)q * n + k] = cx_from<ff>(a.x, a.y);
    }
  }
  for (int i = tid; i < n - 1; i += nt) {
    const z a = ldz(&A[(size_t)(1 + i) * lda]);
    sx[i] = cx_from<ff>(a.x, a.y);
  }
  if (c == 0 && tid == 0) dg[0] = ldz(&A[0]).x;
  // every CTA has read A: its rows 0..3 become the exchange vectors
  if (!grid_sync_mono(bar, 1)) return;
  const ff2 one = {f2_of(1.f, 0.f), f2_of(0.f, 0.f)};
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - 1 - j, par = j & 1;
    z* xp = A + (size_t)(2 * par) * lda;       // p_r at [r]
    z* xc = A + (size_t)(2 * par + 1) * lda;   // A[r][j+1] at [r], r >= j+2
    // reflector of step j from sx[0..m)
    const ff2 alpha = as2(sx[0]);
    ff2 ss = pk_zero();
    for (int i = 1 + tid; i < m; i += nt) {
      const ff2 x = as2(sx[i]);
      ss = x * x + ss;
    }
    const ff2 s2 = pk_block_sum(ss, rb, 0);
    const ff sigma = ffs_add(pk_get_re(s2), pk_get_im(s2));
    const ff ar = pk_get_re(alpha), ai = pk_get_im(alpha);
    ff2 t;
    ff beta;
    if (sigma.hi == 0.f && ai.hi == 0.f) {
      t = pk_zero();
      beta = ar;
      for (int i = tid; i < m; i += nt) sv[i] = of2(i == 0 ? one : pk_zero());
    } else {
      const ff nu = ffs_sqrt(ffs_add(ffs_add(ffs_mul(ar, ar), ffs_mul(ai, ai)), sigma));
      beta = ar.hi >= 0.f ? ffs_neg(nu) : nu;
      const ff amr = ffs_sub(ar, beta);
      const ff rden = ffs_div(ff(1.f, 0.f), ffs_add(ffs_mul(amr, amr), ffs_mul(ai, ai)));
      const ff2 sc = pk_make(ffs_mul(amr, rden), ffs_neg(ffs_mul(ai, rden)));
      t = pk_make(ffs_div(ffs_sub(beta, ar), beta), ffs_neg(ffs_div(ai, beta)));
      for (int i = tid; i < m; i += nt) sv[i] = of2(i == 0 ? one : ff2_settle(pk_mul(as2(sx[i]), sc)));
    }
    __syncthreads();
    if (c == 0) {
      z* rrow = refl + (size_t)j * n + (j + 1);
      // reflector rows stay packed float-float (k_wy_t_ff, k_backtransform_ff read them)
      for (int i = tid; i < m; i += nt) *reinterpret_cast<cx<ff>*>(&rrow[i]) = sv[i];
      if (tid == 0) { tau[j] = pk_to_z(t); e[j] = ffs_to_d(beta); }
    }
    // p = tau A v on the owned rows of the trailing block (r >= j+1)
    const int q0 = c >= j + 1 ? 0 : (j + 1 - c + G - 1) / G;
    const int nq = nr - q0;
    if (nq > 0) {
      ff2 acc[kTridRows];
#pragma unroll
      for (int q = 0; q < kTridRows; ++q) acc[q] = pk_zero();
      for (int k = warp * 32 + lane; k < m; k += nwarp * 32) {
        const ff2 vk = as2(sv[k]), ivk = pk_i(vk);
        const cx<ff>* base = rows + (size_t)q0 * n + (j + 1) + k;
#pragma unroll
        for (int q = 0; q < kTridRows; ++q)
          if (q < nq) {
            const ff2 a = as2(base[(size_t)q * n]);
            acc[q] = fma(pk_im(a), ivk, fma(pk_re(a), vk, acc[q]));
          }
      }
#pragma unroll
      for (int q = 0; q < kTridRows; ++q) {
        if (q < nq) {
          ff2 a = ff2_settle(acc[q]);
          for (int o = 16; o > 0; o >>= 1) a = a + pk_shfl_xor(a, o);
          if (lane == 0) spart[warp][q] = of2(ff2_settle(a));
        }
      }
    }
    __syncthreads();
    if (tid < nq) {
      ff2 a = as2(spart[0][tid]);
      for (int w = 1; w < nwarp; ++w) a = a + as2(spart[w][tid]);
      const int q = q0 + tid, r = c + q * G;
      pk_store(&xp[r], ff2_settle(pk_mul(t, ff2_settle(a))));
      if (r >= j + 2) pk_store(&xc[r], as2(rows[(size_t)q * n + (j + 1)]));
    }
    if (!grid_sync_mono(bar, (unsigned)j + 2)) return;
    // w = p - (1/2) conj(tau) (v^+ p) v; the next column (rows j+2 ..)
    ff2 sp = pk_zero();
    for (int i = tid; i < m; i += nt) {
      const ff2 v = as2(sv[i]), pr = pk_load(&xp[j + 1 + i]);
      sw[i] = of2(pr);
      sp = pk_fma(pk_conj(v), pr, sp);
    }
    for (int i = tid; i < m - 1; i += nt) sx[i] = of2(pk_load(&xc[j + 2 + i]));
    const ff2 vp = pk_block_sum(ff2_settle(sp), rb, 1);
    const ff2 half = {f2_of(0.5f, 0.5f), f2_of(0.5f, 0.5f)};
    const ff2 cf = ff2_settle(pk_mul(pk_conj(t), vp));
    const ff2 ncoef = pk_neg(ff2{mul2(cf.hi, half.hi), mul2(cf.lo, half.lo)});
    for (int i = tid; i < m; i += nt) sw[i] = of2(ff2_settle(pk_fma(ncoef, as2(sv[i]), as2(sw[i]))));
    __syncthreads();
    // A -= v w^+ + w v^+ on the owned rows, and on the next column
    for (int q = q0; q < nr; ++q) {
      const int kr = c + q * G - (j + 1);
      const ff2 nvr = pk_neg(as2(sv[kr])), nwr = pk_neg(as2(sw[kr]));
      const ff2 nvr_re = pk_re(nvr), nvr_im = pk_im(nvr), nwr_re = pk_re(nwr), nwr_im = pk_im(nwr);
      cx<ff>* arow = rows + (size_t)q * n + (j + 1);
      for (int k = tid; k < m; k += nt) {
        const ff2 cw = pk_conj(as2(sw[k])), cv = pk_conj(as2(sv[k]));
        ff2 a = as2(arow[k]);
        a = fma(nvr_re, cw, a);
        a = fma(nvr_im, pk_i(cw), a);
        a = fma(nwr_re, cv, a);
        a = fma(nwr_im, pk_i(cv), a);
        a = ff2_settle(a);
        arow[k] = of2(a);
        if (kr == 0 && k == 0) dg[j + 1] = ffs_to_d(pk_get_re(a));
      }
    }
    {
      // v_0 = 1: x_i - v_{i+1} conj(w_0) - w_{i+1}
      const ff2 cw0 = pk_conj(as2(sw[0]));
      for (int i = tid; i < m - 1; i += nt) {
        const ff2 x = as2(sx[i]) - as2(sw[i + 1]);
        sx[i] = of2(ff2_settle(pk_fma(pk_neg(as2(sv[i + 1])), cw0, x)));
      }
    }
    __syncthreads();   // the next reflector reads all of sx
  }
}

// ---- helpers of the one-pass real tridiagonalisation and back-transformation ---------
__device__ __forceinline__ ff2 pk_shfl_idx(ff2 a, int src) {
  return {{__shfl_sync(0xffffffffu, a.hi.v, src)}, {__shfl_sync(0xffffffffu, a.lo.v, src)}};
}
// fold the per-warp partials buf[0..nw) (nw a power of two, <= 32) in one warp:
// every lane gets the sum; fixed order, the same in every CTA
__device__ __forceinline__ ff2 pk_fold_partials(const cx<ff>* buf, int nw) {
  const int lane = threadIdx.x & 31;
  ff2 t = lane < nw ? as2(buf[lane]) : pk_zero();
  for (int o = nw >> 1; o > 0; o >>= 1) t = t + pk_shfl_xor(t, o);
  return ff2_settle(pk_shfl_idx(t, 0));
}
// the warp's sums of eight rows at once: lane l ends with the sum of row (l >> 2) & 7
// (at each of the first three levels a lane keeps half of its rows and trades the
// other half with its partner, then the groups of four lanes fold)
__device__ __forceinline__ ff2 pk_warp_rows8(const ff2 (&a)[8]) {
  const int lane = threadIdx.x & 31;
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
  ff2 b[4], d[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const ff2 keep = h4 ? a[i + 4] : a[i], send = h4 ? a[i] : a[i + 4];
    b[i] = keep + pk_shfl_xor(send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const ff2 keep = h3 ? b[i + 2] : b[i], send = h3 ? b[i] : b[i + 2];
    d[i] = keep + pk_shfl_xor(send, 8);
  }
  ff2 s = (h2 ? d[1] : d[0]) + pk_shfl_xor(h2 ? d[0] : d[1], 4);
  s = s + pk_shfl_xor(s, 2);
  return s + pk_shfl_xor(s, 1);
}
// ---- the real symmetric form (k = 0 reduced problems) ------------------------------
// The reduced matrices of the k = 0 (real-in-r) Davidson are real symmetric
// (the real-output products write exact zeros).  This reduction keeps the row
// ownership, exchange vectors and single grid barrier per column of
// k_tridiag_rows_ff, with its CTA-local latency cut (phase clocks in
// k_tridiag_rows_ff over a C2 solve: 1.6 of 8.0 us per column at the grid
// barrier, 3.2 in the two passes over the rows, 1.2 in the block sums):
//  - the rank-2 update of step j - 1 on the owned rows is deferred into the pass
//    of step j that forms p = tau A v, so each element is read, updated,
//    written back and multiplied by v_j in one visit; the rows' pending pair
//    (v_{j-1}, w_{j-1}) lives beside v_j (two v buffers alternate; w overwrites
//    its predecessor once the pass is done), and row j, which no later pass
//    visits, takes its diagonal share of the pending update from its owner;
//  - one warp forms the reflector's scalars (norm, beta, tau, the scale of v),
//    the others read them from shared memory, and v is formed inside the pass;
//  - after the barrier each thread loads the published p and next-column
//    entries it needs, so w and the next column follow from one block sum;
//  - the p sums of the (at most 8) rows leave a warp in one transposing
//    butterfly (each level halves the rows a lane carries);
//  - the f32x2 lanes carry two adjacent columns instead of (re, im): a row pair
//    costs three float-float FMAs where a complex element costs six, and the
//    rows take half the shared memory.
// Rows and vectors are pair-packed by absolute index (pair P = columns 2P and
// 2P+1, as one cx<ff>: hi parts, then lo parts); vectors are zero outside their
// range (v_j and w_j below index j+1, the column below j+2), so the pass and the
// updates run over whole pairs and the lanes outside the trailing block add
// exact zeros.  The exchange vectors hold p and the next column pair-packed as
// floats.  tau leaves in the complex format (zero imaginary parts), the
// reflector rows pair-packed; heev_finish reads both with its real kernels.
// 256 threads; n <= 2 * 2 * 256.
constexpr int kTridRealThreads = 256;
constexpr int kTridRealU = 2;

// keep lane 0 and/or lane 1 of a packed pair (the other becomes +0)
__device__ __forceinline__ ff2 pk_lanes(ff2 a, bool keep0, bool keep1) {
  const unsigned long long m = (keep0 ? 0xffffffffull : 0ull) | (keep1 ? 0xffffffff00000000ull : 0ull);
  return {{a.hi.v & m}, {a.lo.v & m}};
}
__device__ __forceinline__ ff pk_lane(ff2 a, int l) { return l ? pk_get_im(a) : pk_get_re(a); }
// element i of a pair-packed vector
__device__ __forceinline__ ff pk_elem(const cx<ff>* v, int i) { return pk_lane(as2(v[i >> 1]), i & 1); }
__device__ __forceinline__ void pk_put_elem(float* base, int i, ff x) {
  base[4 * (i >> 1) + (i & 1)] = x.hi;
  base[4 * (i >> 1) + 2 + (i & 1)] = x.lo;
}

__global__ void __launch_bounds__(kTridRealThreads) k_tridiag_real_ff(z* A, int n, int lda,
                                                                    z* tau, R* e, R* dg,
                                                                    z* refl, GridBar bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int U = kTridRealU;
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int NP = (n + 1) >> 1;                     // pairs per row
  const int nrmax = (n + G - 1) / G;
  const int nr = c < n ? (n - 1 - c) / G + 1 : 0;   // rows owned: c + q G, q < nr
  cx<ff>* rows = reinterpret_cast<cx<ff>*>(smem_raw);   // nrmax x NP
  // rows + (nrmax + (j & 1)) NP: v_j; the other one v_{j-1}
  cx<ff>* sw = rows + (size_t)(nrmax + 2) * NP;   // w_{j-1} (pending), then w_j
  cx<ff>* sx = rows + (size_t)(nrmax + 3) * NP;   // column to reduce (absolute index)
  __shared__ cx<ff> rb[2][32];
  __shared__ ff scal[2];   // the scale of v (x_i -> v_i) and tau
  __shared__ cx<ff> spart[kTridRealThreads / 32][kTridRows];
  for (int q = 0; q < nr; ++q) {
    const z* src = A + (size_t)(c + q * G) * lda;
    for (int P = tid; P < NP; P += nt) {
      const ff a0 = ff(ldz(src + 2 * P).x);
      const ff a1 = 2 * P + 1 < n ? ff(ldz(src + 2 * P + 1).x) : ff(0.f, 0.f);
      rows[(size_t)q * NP + P] = of2(pk_make(a0, a1));
    }
  }
  ff2 ss = pk_zero();   // squared norm of the column below its first entry
  for (int P = tid; P < NP; P += nt) {
    const int i0 = 2 * P, i1 = 2 * P + 1;
    const ff a0 = i0 >= 1 ? ff(ldz(&A[(size_t)i0 * lda]).x) : ff(0.f, 0.f);
    const ff a1 = i1 < n ? ff(ldz(&A[(size_t)i1 * lda]).x) : ff(0.f, 0.f);
    const ff2 x = pk_make(a0, a1);
    sx[P] = of2(x);
    const ff2 xm = pk_lanes(x, i0 >= 2, i1 >= 2);
    ss = xm * xm + ss;
  }
  if (c == 0 && tid == 0) dg[0] = ldz(&A[0]).x;
  // every CTA has read A: its rows 0..3 become the exchange vectors
  if (!grid_sync_mono(bar, 1)) return;
  const ff one = ff(1.f, 0.f);
  for (int j = 0; j < n - 1; ++j) {
    const int par = j & 1;
    const bool pend = j >= 1;
    float* xpf = reinterpret_cast<float*>(A + (size_t)(2 * par) * lda);       // p, pair-packed
    float* xcf = reinterpret_cast<float*>(A + (size_t)(2 * par + 1) * lda);   // next column
    cx<ff>* sv = rows + (size_t)(nrmax + par) * NP;
    const cx<ff>* svp = rows + (size_t)(nrmax + (par ^ 1)) * NP;
    // reflector of step j from x (indices j+1 ..): one warp forms its scalars
    for (int o = 16; o > 0; o >>= 1) ss = ss + pk_shfl_xor(ss, o);
    if (lane == 0) rb[0][warp] = of2(ff2_settle(ss));
    __syncthreads();
    if (warp == 0) {
      const ff2 s2 = pk_fold_partials(rb[0], nwarp);
      if (lane == 0) {
        const ff sigma = ffs_add(pk_get_re(s2), pk_get_im(s2));
        const ff alpha = pk_elem(sx, j + 1);
        ff t, sc, beta;
        if (sigma.hi == 0.f) {   // v = e_{j+1}, tau = 0
          t = ff(0.f, 0.f);
          sc = ff(0.f, 0.f);
          beta = alpha;
        } else {
          const ff nu = ffs_sqrt(ffs_add(ffs_mul(alpha, alpha), sigma));
          beta = alpha.hi >= 0.f ? ffs_neg(nu) : nu;
          sc = ffs_div(one, ffs_sub(alpha, beta));
          t = ffs_div(ffs_sub(beta, alpha), beta);
        }
        scal[0] = sc;
        scal[1] = t;
        if (c == 0) { tau[j] = {ffs_to_d(t), R(0)}; e[j] = ffs_to_d(beta); }
      }
    } else if (pend && tid == 32 && c == j % G) {
      // row j: the diagonal share of the pending update of step j - 1 (v_j = 1 there)
      const int P = j >> 1;
      const ff2 nv = ff2_bcast(ffs_neg(pk_elem(svp, j))), nw = ff2_bcast(ffs_neg(pk_elem(sw, j)));
      ff2 a = as2(rows[(size_t)(j / G) * NP + P]);
      a = fma(nv, as2(sw[P]), a);
      a = fma(nw, as2(svp[P]), a);
      dg[j] = ffs_to_d(pk_lane(ff2_settle(a), j & 1));
    }
    __syncthreads();
    const ff2 sc = ff2_bcast(scal[0]), t2 = ff2_bcast(scal[1]);
    // v_j on the owned pairs P = tid + u nt: 0 below index j+1, 1 at j+1
    ff2 vk[U], cwk[U], cvk[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int P = tid + u * nt;
      vk[u] = cwk[u] = cvk[u] = pk_zero();
      if (P < NP) {
        const int i0 = 2 * P;
        ff2 v = pk_lanes(ff2_settle(as2(sx[P]) * sc), i0 >= j + 2, i0 + 1 >= j + 2);
        if (i0 == j + 1) v = pk_make(one, pk_get_im(v));
        if (i0 + 1 == j + 1) v = pk_make(pk_get_re(v), one);
        vk[u] = v;
        sv[P] = of2(v);
        // reflector row j pair-packed, every pair (k_wy_t_real_ff, k_backtransform_real_ff)
        if (c == 0) reinterpret_cast<cx<ff>*>(refl + (size_t)j * n)[P] = of2(v);
        if (pend) {
          cwk[u] = as2(sw[P]);
          cvk[u] = as2(svp[P]);
        }
      }
    }
    // owned rows of the trailing block (r >= j+1): the pending update of step
    // j - 1, and (A v)_r, over the pairs that hold columns j+1 ..
    const int P0 = (j + 1) >> 1;
    const int q0 = c >= j + 1 ? 0 : (j + 1 - c + G - 1) / G;
    const int nq = nr - q0;
    if (nq > 0) {
      ff2 acc[kTridRows];
#pragma unroll
      for (int q = 0; q < kTridRows; ++q) {
        acc[q] = pk_zero();
        if (q < nq) {
          const int r = c + (q0 + q) * G;
          cx<ff>* base = rows + (size_t)(q0 + q) * NP;
          ff2 nv = pk_zero(), nw = pk_zero();
          if (pend) {
            nv = ff2_bcast(ffs_neg(pk_elem(svp, r)));
            nw = ff2_bcast(ffs_neg(pk_elem(sw, r)));
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int P = tid + u * nt;
            if (P >= P0 && P < NP) {
              ff2 a = as2(base[P]);
              if (pend) {
                a = ff2_settle(fma(nw, cvk[u], fma(nv, cwk[u], a)));
                base[P] = of2(a);
              }
              acc[q] = fma(a, vk[u], acc[q]);
            }
          }
          acc[q] = ff2_settle(acc[q]);
        }
      }
      const ff2 s8 = pk_warp_rows8(acc);
      if ((lane & 3) == 0) spart[warp][lane >> 2] = of2(ff2_settle(s8));
    }
    __syncthreads();
    if (warp < nq) {
      ff2 a = lane < nwarp ? as2(spart[lane][warp]) : pk_zero();
      for (int o = nwarp >> 1; o > 0; o >>= 1) a = a + pk_shfl_xor(a, o);
      if (lane == 0) {
        const int q = q0 + warp, r = c + q * G;
        a = ff2_settle(a);
        pk_put_elem(xpf, r, ffs_mul(scal[1], ffs_add(pk_get_re(a), pk_get_im(a))));
        if (r >= j + 2) pk_put_elem(xcf, r, pk_elem(rows + (size_t)q * NP, j + 1));
      }
    }
    if (!grid_sync_mono(bar, (unsigned)j + 2)) return;
    // loads of the published vectors: p (indices j+1 ..), the column (j+2 ..), p_{j+1}
    ff2 pi[U], xi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int P = tid + u * nt, i0 = 2 * P;
      pi[u] = xi[u] = pk_zero();
      // (the padding lane of an odd n is never written: masked like the stale entries)
      if (P < NP && i0 + 1 >= j + 1) {
        pi[u] = pk_lanes(pk_load(reinterpret_cast<const z*>(xpf + 4 * P)), i0 >= j + 1, i0 + 1 < n);
        if (i0 + 1 >= j + 2)
          xi[u] = pk_lanes(pk_load(reinterpret_cast<const z*>(xcf + 4 * P)), i0 >= j + 2,
                           i0 + 1 < n);
      }
    }
    const int Pj = (j + 1) >> 1;
    const ff2 pjp = pk_load(reinterpret_cast<const z*>(xpf + 4 * Pj));
    const ff pj1 = pk_lane(pjp, (j + 1) & 1);
    ff2 sp = pk_zero();
#pragma unroll
    for (int u = 0; u < U; ++u) sp = fma(vk[u], pi[u], sp);
    for (int o = 16; o > 0; o >>= 1) sp = sp + pk_shfl_xor(sp, o);
    if (lane == 0) rb[1][warp] = of2(ff2_settle(sp));
    __syncthreads();
    // w = p - (1/2) tau (v . p) v; the next column: x_i - w_i - v_i w_{j+1}
    // (indices j+2 ..), and its squared norm below its first entry
    const ff2 vpp = pk_fold_partials(rb[1], nwarp);
    const ff vp = ffs_add(pk_get_re(vpp), pk_get_im(vpp));
    const ff2 ncoef = ff2_bcast(ffs_neg(ffs_mul(ff(0.5f, 0.f), ffs_mul(scal[1], vp))));
    const ff2 wj1 = ff2_settle(fma(ncoef, ff2_bcast(one), ff2_bcast(pj1)));
    ss = pk_zero();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int P = tid + u * nt, i0 = 2 * P;
      if (P < NP) {
        const ff2 w = ff2_settle(fma(ncoef, vk[u], pi[u]));
        sw[P] = of2(w);
        const ff2 x = pk_lanes(ff2_settle(fma(pk_neg(vk[u]), wj1, xi[u] - w)), i0 >= j + 2,
                               i0 + 1 >= j + 2);
        sx[P] = of2(x);
        const ff2 xm = pk_lanes(x, i0 >= j + 3, i0 + 1 >= j + 3);
        ss = xm * xm + ss;
      }
    }
  }
  // row n - 1: the diagonal share of the last step's update
  __syncthreads();
  if (n >= 2 && tid == 0 && c == (n - 1) % G) {
    const cx<ff>* vl = rows + (size_t)(nrmax + ((n - 2) & 1)) * NP;
    const int P = (n - 1) >> 1;
    const ff2 nv = ff2_bcast(ffs_neg(pk_elem(vl, n - 1))), nw = ff2_bcast(ffs_neg(pk_elem(sw, n - 1)));
    ff2 a = as2(rows[(size_t)((n - 1) / G) * NP + P]);
    a = fma(nv, as2(sw[P]), a);
    a = fma(nw, as2(vl[P]), a);
    dg[n - 1] = ffs_to_d(pk_lane(ff2_settle(a), (n - 1) & 1));
  }
}
#endif

// One warp per eigenvalue, two per CTA; d and e^2 staged in shared memory.
// FP64: the bracket is first narrowed in FP32 (d, e^2 rounded to float, ~60x the
// FP64 rate on GB300) to 64 float ulps of ||T||, widened by 16 ulps (the
// rounding of T and the Sturm count's backward error are a few ulps of ||T||),
// then in float-float to 2^-45 ||T|| (the counts' resolution, ~1e-14 ||T||,
// that of T itself after the float-float reduction; no FP64 rounds).
// Dynamic shared memory: n (d) + n (e^2) R, and in FP64 2 n floats + 2 n ff.
__global__ void __launch_bounds__(64) k_bisect(const R* d, const R* e, int n, int nev,
                                                R* w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sd = reinterpret_cast<R*>(smem_raw);
  R* se2 = sd + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = d[i];
    se2[i] = i < n - 1 ? e[i] * e[i] : R(0);
  }
  float* fd = reinterpret_cast<float*>(se2 + n);
  float* fe2 = fd + n;
  ff* xd = reinterpret_cast<ff*>(fe2 + n);
  ff* xe2 = xd + n;
  if constexpr (sizeof(R) == 8) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      fd[i] = (float)d[i];
      fe2[i] = i < n - 1 ? (float)(e[i] * e[i]) : 0.f;
      xd[i] = ff((double)d[i]);
      xe2[i] = i < n - 1 ? ff((double)(e[i] * e[i])) : ff(0.0);
    }
  }
  __syncthreads();
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nev) return;
  R lo = R(0), hi = R(0);
  {
    R l = 1e300, h = -1e300;
    for (int i = lane; i < n; i += 32) {
      const R r = (i > 0 ? fabs(e[i - 1]) : R(0)) + (i < n - 1 ? fabs(e[i]) : R(0));
      l = fmin(l, d[i] - r);
      h = fmax(h, d[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
      h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
    }
    lo = l;
    hi = h;
  }
  const R nrm = fmax(fabs(lo), fabs(hi));
  const R tiny = RealT<R>::tiny + RealT<R>::tiny_rel * nrm;
  lo -= RealT<R>::margin * nrm + RealT<R>::tiny;
  hi += RealT<R>::margin * nrm + RealT<R>::tiny;
  if constexpr (sizeof(R) == 8) {
    const float fe = RealT<float>::eps, fn = (float)nrm;
    float flo = __double2float_rd(lo), fhi = __double2float_ru(hi);
    multisect<float>(fd, fe2, n, k, RealT<float>::tiny + RealT<float>::tiny_rel * fn, flo, fhi,
                     0.f, 64.f * fe * fn);
    const R pad = R(16) * R(fe) * nrm + RealT<R>::tiny;
    lo = fmax(lo, R(flo) - pad);
    hi = fmin(hi, R(fhi) + pad);
    // float-float rounds down to 2^-45 ||T|| (their counts' backward error is a
    // few units of 2^-47 ||T||): the eigenvalue to ~1e-14 ||T||, the accuracy
    // that T itself carries when the FP64 path's float-float reduction formed it
    double xlo = lo, xhi = hi;
    multisect_ff(xd, xe2, n, k, (float)fmax(1e-30 * nrm, 1e-30), xlo, xhi, 0x1p-45 * nrm);
    if (lane == 0) w[k] = 0.5 * (xlo + xhi);
    return;
  }
  multisect<R>(sd, se2, n, k, tiny, lo, hi, RealT<R>::eps, R(0));
  if (lane == 0) w[k] = R(0.5) * (lo + hi);
}

// ---- tridiagonal eigenvectors: inverse iteration --------------------------------------
// splitmix64 (Steele, Lea, Flood 2014) for deterministic start vectors
__device__ __forceinline__ double start_component(unsigned long long k, unsigned long long i) {
  unsigned long long x = k * 0x9E3779B97F4A7C15ull + i * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return ((double)(x >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Inverse iterations per eigenvector.  The shift is the bisection eigenvalue
// (within a few ulps of ||T||), so each solve multiplies the wanted component
// by ~1/(eps ||T||) against 1/gap for the others: three leave ~(eps/gap_rel)^3
// of any neighbour outside the shift's cluster (clusters are orthogonalised).
// FP32 keeps a fourth (its eps is 1e9 times larger; the solves are cheap).
constexpr int kInvIters = sizeof(R) == 8 ? 3 : 4;

// One CTA per cluster of consecutive eigenvalues closer than ctol; the CTA whose
// index starts a cluster handles all of it, the others return.  Vectors are rows
// Y[k][0..n).  Shared memory: 6 arrays of n doubles (+ ints) for the factorisation.
#if !defined(QE_DENSE_FP64)   // FP64: k_inviter_ff below
__global__ void __launch_bounds__(256) k_inviter(const R* d, const R* e, int n, int nev,
                                                 const R* w, R ctol_rel, R* Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* u0 = reinterpret_cast<R*>(smem_raw);
  R* u1 = u0 + n;
  R* u2 = u1 + n;
  R* ml = u2 + n;
  R* y = ml + n;
  int* sw = reinterpret_cast<int*>(y + n);
  __shared__ R sh[33];
  const int k0 = blockIdx.x;
  if (k0 >= nev) return;
  // ||T|| bound (Gershgorin), a block-wide max: every thread a stride of rows
  R nrm = R(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    nrm = fmax(nrm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : R(0)) + (i < n - 1 ? fabs(e[i]) : R(0)));
  for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nrm;
  __syncthreads();
  nrm = R(0);
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) nrm = fmax(nrm, sh[q]);
  __syncthreads();
  const R ctol = ctol_rel * fmax(nrm, RealT<R>::tiny);
  if (k0 > 0 && w[k0] - w[k0 - 1] <= ctol) return;   // not a cluster start
  int k1 = k0 + 1;
  while (k1 < nev && w[k1] - w[k1 - 1] <= ctol) ++k1;
  const R tiny = fmax(RealT<R>::eps * nrm, RealT<R>::tiny);
  for (int k = k0; k < k1; ++k) {
    const R lam = w[k];
    // LU with partial pivoting of T - lam I (thread 0; u0 holds the reciprocal
    // pivots, so that the solves multiply)
    if (threadIdx.x == 0) {
      R c0 = d[0] - lam, c1 = n > 1 ? e[0] : R(0), c2 = R(0);
      for (int i = 0; i < n - 1; ++i) {
        R n0 = e[i], n1 = d[i + 1] - lam, n2 = (i + 2 < n) ? e[i + 1] : R(0);
        int s = 0;
        if (fabs(n0) > fabs(c0)) {
          R t;
          t = c0; c0 = n0; n0 = t;
          t = c1; c1 = n1; n1 = t;
          t = c2; c2 = n2; n2 = t;
          s = 1;
        }
        if (fabs(c0) < tiny) c0 = c0 < R(0) ? -tiny : tiny;
        const R rc = R(1) / c0;
        const R mlt = n0 * rc;
        u0[i] = rc; u1[i] = c1; u2[i] = c2; ml[i] = mlt; sw[i] = s;
        c0 = n1 - mlt * c1;
        c1 = n2 - mlt * c2;
        c2 = R(0);
      }
      if (fabs(c0) < tiny) c0 = c0 < R(0) ? -tiny : tiny;
      u0[n - 1] = R(1) / c0; u1[n - 1] = R(0); u2[n - 1] = R(0);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = start_component(k, i);
    __syncthreads();
    for (int it = 0; it < kInvIters; ++it) {
      if (threadIdx.x == 0) {
        // running entries in registers (as k_inviter_ff)
        R cur = y[0];
        for (int i = 0; i < n - 1; ++i) {
          R nxt = y[i + 1];
          if (sw[i]) { const R t = cur; cur = nxt; nxt = t; }
          y[i] = cur;
          cur = nxt - ml[i] * cur;
        }
        y[n - 1] = cur;
        R y1 = R(0), y2 = R(0);
        for (int i = n - 1; i >= 0; --i) {
          R s = y[i];
          if (i + 1 < n) s -= u1[i] * y1;
          if (i + 2 < n) s -= u2[i] * y2;
          const R yi = s * u0[i];
          y[i] = yi;
          y2 = y1;
          y1 = yi;
        }
      }
      __syncthreads();
      // scale down first (the solve grows the vector by up to 1/tiny)
      R mx = R(0);
      for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(y[i]));
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
      __syncthreads();
      if (threadIdx.x == 0) {
        R m2 = R(0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m2 = fmax(m2, sh[q]);
        sh[32] = m2 > R(0) ? m2 : R(1);
      }
      __syncthreads();
      const R inv_mx = R(1) / sh[32];
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv_mx;
      __syncthreads();
      // orthogonalise against the finished vectors of this cluster (twice)
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = k0; q < k; ++q) {
          const R* yq = Y + (size_t)q * n;
          R s = R(0);
          for (int i = threadIdx.x; i < n; i += blockDim.x) s += yq[i] * y[i];
          s = block_sum(s, sh);
          for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] -= s * yq[i];
          __syncthreads();
        }
      }
      R s = R(0);
      for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
      s = block_sum(s, sh);
      const R inv = s > R(0) ? R(1) / sqrt(s) : R(0);
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv;
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Y[(size_t)k * n + i] = y[i];
    __syncthreads();
  }
}
#endif

#if defined(QE_DENSE_FP64)
// k_inviter in float-float arithmetic (the FP64 path): the LU of T - lambda I and
// the solves are one thread's dependent chains, whose FP64 divisions and
// multiply-adds cost ~64 cycles per instruction on GB300; in float-float on the
// FP32 pipes the chain is several times shorter.  The eigenvalue shift, the
// cluster test and the output stay double; eigenvectors to ~1e-14.
__device__ __forceinline__ ff ffi_abs(ff a) { return a.hi < 0.f ? ffs_neg(a) : a; }
__device__ ff ffi_block_sum(ff v, ff* sh) {
  for (int o = 16; o > 0; o >>= 1)
    v = ffs_add(v, ff(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)));
  const int wv = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[wv] = v;
  __syncthreads();
  ff t = sh[0];
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = ffs_add(t, sh[q]);
  __syncthreads();
  return t;
}
__global__ void __launch_bounds__(256) k_inviter_ff(const R* d, const R* e, int n, int nev,
                                                    const R* w, R ctol_rel, R* Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ff* u0 = reinterpret_cast<ff*>(smem_raw);
  ff* u1 = u0 + n;
  ff* u2 = u1 + n;
  ff* ml = u2 + n;
  ff* y = ml + n;
  ff* xd = y + n;
  ff* xe = xd + n;
  int* sw = reinterpret_cast<int*>(xe + n);
  __shared__ R sh[33];
  __shared__ ff shf[33];
  const int k0 = blockIdx.x;
  if (k0 >= nev) return;
  R nrm = R(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    nrm = fmax(nrm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : R(0)) + (i < n - 1 ? fabs(e[i]) : R(0)));
  for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nrm;
  __syncthreads();
  nrm = R(0);
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) nrm = fmax(nrm, sh[q]);
  __syncthreads();
  const R ctol = ctol_rel * fmax(nrm, RealT<R>::tiny);
  if (k0 > 0 && w[k0] - w[k0 - 1] <= ctol) return;   // not a cluster start
  int k1 = k0 + 1;
  while (k1 < nev && w[k1] - w[k1 - 1] <= ctol) ++k1;
  const ff tiny((double)fmax(RealT<R>::eps * nrm, 1e-30));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xd[i] = ff((double)d[i]);
    xe[i] = i < n - 1 ? ff((double)e[i]) : ff(0.f, 0.f);
  }
  __syncthreads();
  for (int k = k0; k < k1; ++k) {
    const ff lam((double)w[k]);
    if (threadIdx.x == 0) {
      ff c0 = ffs_sub(xd[0], lam), c1 = n > 1 ? xe[0] : ff(0.f, 0.f), c2(0.f, 0.f);
      for (int i = 0; i < n - 1; ++i) {
        ff n0 = xe[i], n1 = ffs_sub(xd[i + 1], lam), n2 = (i + 2 < n) ? xe[i + 1] : ff(0.f, 0.f);
        int sp = 0;
        if (fabsf(n0.hi) > fabsf(c0.hi)) {
          ff t;
          t = c0; c0 = n0; n0 = t;
          t = c1; c1 = n1; n1 = t;
          t = c2; c2 = n2; n2 = t;
          sp = 1;
        }
        if (fabsf(c0.hi) < tiny.hi) c0 = c0.hi < 0.f ? ffs_neg(tiny) : tiny;
        const ff rc = ffs_div(ff(1.f, 0.f), c0);
        const ff mlt = ffs_mul(n0, rc);
        u0[i] = rc; u1[i] = c1; u2[i] = c2; ml[i] = mlt; sw[i] = sp;
        c0 = ffs_sub(n1, ffs_mul(mlt, c1));
        c1 = ffs_sub(n2, ffs_mul(mlt, c2));
        c2 = ff(0.f, 0.f);
      }
      if (fabsf(c0.hi) < tiny.hi) c0 = c0.hi < 0.f ? ffs_neg(tiny) : tiny;
      u0[n - 1] = ffs_div(ff(1.f, 0.f), c0); u1[n - 1] = ff(0.f, 0.f); u2[n - 1] = ff(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = ff(start_component(k, i));
    __syncthreads();
    for (int it = 0; it < kInvIters; ++it) {
      if (threadIdx.x == 0) {
        // the sweeps carry their running entries in registers: the recurrence
        // does not wait on a shared-memory store and reload per step
        ff cur = y[0];
        for (int i = 0; i < n - 1; ++i) {
          ff nxt = y[i + 1];
          if (sw[i]) { const ff t = cur; cur = nxt; nxt = t; }
          y[i] = cur;
          cur = ffs_sub(nxt, ffs_mul(ml[i], cur));
        }
        y[n - 1] = cur;
        ff y1(0.f, 0.f), y2(0.f, 0.f);   // y[i + 1], y[i + 2] of the backward sweep
        for (int i = n - 1; i >= 0; --i) {
          ff sacc = y[i];
          if (i + 1 < n) sacc = ffs_sub(sacc, ffs_mul(u1[i], y1));
          if (i + 2 < n) sacc = ffs_sub(sacc, ffs_mul(u2[i], y2));
          const ff yi = ffs_mul(sacc, u0[i]);
          y[i] = yi;
          y2 = y1;
          y1 = yi;
        }
      }
      __syncthreads();
      // scale down first (the solve grows the vector by up to 1/tiny)
      float mx = 0.f;
      for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(y[i].hi));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = ff(mx, 0.f);
      __syncthreads();
      float m2 = 0.f;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m2 = fmaxf(m2, shf[q].hi);
      __syncthreads();
      const ff inv_mx = ffs_div(ff(1.f, 0.f), ff(m2 > 0.f ? m2 : 1.f, 0.f));
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = ffs_mul(y[i], inv_mx);
      __syncthreads();
      // orthogonalise against the finished vectors of this cluster (twice)
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = k0; q < k; ++q) {
          const R* yq = Y + (size_t)q * n;
          ff sacc(0.f, 0.f);
          for (int i = threadIdx.x; i < n; i += blockDim.x) sacc = ffs_add(sacc, ffs_mul(ff((double)yq[i]), y[i]));
          const ff sdot = ffi_block_sum(sacc, shf);
          for (int i = threadIdx.x; i < n; i += blockDim.x)
            y[i] = ffs_sub(y[i], ffs_mul(sdot, ff((double)yq[i])));
          __syncthreads();
        }
      }
      ff sacc(0.f, 0.f);
      for (int i = threadIdx.x; i < n; i += blockDim.x) sacc = ffs_add(sacc, ffs_mul(y[i], y[i]));
      const ff ss = ffi_block_sum(sacc, shf);
      const ff inv = ss.hi > 0.f ? ffs_div(ff(1.f, 0.f), ffs_sqrt(ss)) : ff(0.f, 0.f);
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = ffs_mul(y[i], inv);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Y[(size_t)k * n + i] = ffs_to_d(y[i]);
    __syncthreads();
  }
}
#endif

// X[:, k] = H_0 H_1 ... H_{n-2} y_k by blocks of kWY reflectors in compact WY
// form: H_j0 ... H_j0+kWY-1 = I - V T V^+ (V = [v_j0 ...] from the rows of refl,
// v_j zero up to row j and 1 at row j+1; T upper triangular, Schreiber & Van
// Loan 1989).  k_wy_t builds every block's T, k_backtransform applies the blocks
// last to first with one block reduction per block instead of one per reflector.
constexpr int kWY = 8;

// T of block g (reflectors j0 = g kWY .. j0 + nr - 1): P = V^+ V over the
// block's rows, then T_ii = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) P(0:i, i).
// One CTA per block; T blocks of kWY x kWY complex, row-major, zero-padded.
__global__ void __launch_bounds__(256) k_wy_t(const z* __restrict__ refl, int n,
                                              const z* __restrict__ tau, z* __restrict__ T) {
  __shared__ z P[kWY][kWY];
  const int g = blockIdx.x, j0 = g * kWY, nr = min(kWY, n - 1 - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // P[a][b] = v_a^+ v_b for a < b: rows i >= j0 + b + 1 (v_b vanishes above)
  // a reflector with tau = 0 is the identity and its row of refl may be stale:
  // it contributes zero vectors (P entries 0, T row and column 0)
  for (int pq = warp; pq < kWY * kWY; pq += nw) {
    const int a = pq / kWY, bb = pq % kWY;
    if (!(a < bb && bb < nr)) continue;
    const z ta = tau[j0 + a], tb = tau[j0 + bb];
    if ((ta.x == R(0) && ta.y == R(0)) || (tb.x == R(0) && tb.y == R(0))) {
      if (lane == 0) P[a][bb] = {R(0), R(0)};
      continue;
    }
    const z* va = refl + (size_t)(j0 + a) * n;
    const z* vb = refl + (size_t)(j0 + bb) * n;
    R sr = R(0), si = R(0);
    for (int i = j0 + bb + 1 + lane; i < n; i += 32) {
      const z x = va[i], y = vb[i];
      sr = fmar(x.x, y.x, fmar(x.y, y.y, sr));
      si = fmar(x.x, y.y, fmar(-x.y, y.x, si));
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) P[a][bb] = {sr, si};
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    z t[kWY][kWY];
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) t[r][c] = {R(0), R(0)};
    for (int i = 0; i < nr; ++i) {
      const z ti = tau[j0 + i];
      for (int r = 0; r < i; ++r) {
        z acc = {R(0), R(0)};
        for (int c = r; c < i; ++c) acc = cadd(acc, cmul(t[r][c], P[c][i]));
        t[r][i] = {-(ti.x * acc.x - ti.y * acc.y), -(ti.x * acc.y + ti.y * acc.x)};
      }
      t[i][i] = ti;
    }
    z* out = T + (size_t)g * kWY * kWY;
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) out[r * kWY + c] = t[r][c];
  }
}

// One CTA per eigenvector; X [n][ldx].  Per block (last to first):
// w = V^+ x (one block reduction), u = T w, x -= V u.
__global__ void __launch_bounds__(256) k_backtransform(const z* __restrict__ refl, int n,
                                                       const z* __restrict__ T, const R* Y, z* X,
                                                       int ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* x = reinterpret_cast<z*>(smem_raw);
  __shared__ z part[8][kWY];
  __shared__ z u[kWY];
  const int k = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = {Y[(size_t)k * n + i], R(0)};
  __syncthreads();
  const int ngroups = (n - 1 + kWY - 1) / kWY;
  for (int g = ngroups - 1; g >= 0; --g) {
    const int j0 = g * kWY;
    const z* tg0 = T + (size_t)g * kWY * kWY;
    // reflectors taking part: tau = T_aa != 0 (the others are the identity, and
    // their rows of refl are not read)
    unsigned act = 0;
    const int nr = min(kWY, n - 1 - j0);
#pragma unroll
    for (int a = 0; a < kWY; ++a) {
      const z d = tg0[a * kWY + a];
      if (a < nr && (d.x != R(0) || d.y != R(0))) act |= 1u << a;
    }
    z acc[kWY];
#pragma unroll
    for (int a = 0; a < kWY; ++a) acc[a] = {R(0), R(0)};
    for (int i = j0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const z xi = x[i];
#pragma unroll
      for (int a = 0; a < kWY; ++a) {
        if (((act >> a) & 1u) && i >= j0 + a + 1) {
          const z v = refl[(size_t)(j0 + a) * n + i];
          acc[a].x = fmar(v.x, xi.x, fmar(v.y, xi.y, acc[a].x));
          acc[a].y = fmar(v.x, xi.y, fmar(-v.y, xi.x, acc[a].y));
        }
      }
    }
#pragma unroll
    for (int a = 0; a < kWY; ++a) {
      for (int o = 16; o > 0; o >>= 1) {
        acc[a].x += __shfl_xor_sync(0xffffffffu, acc[a].x, o);
        acc[a].y += __shfl_xor_sync(0xffffffffu, acc[a].y, o);
      }
      if (lane == 0) part[warp][a] = acc[a];
    }
    __syncthreads();
    if (threadIdx.x < kWY) {
      // w_c = sum over warps, then u_a = sum_{c >= a} T[a][c] w_c (c < nr)
      __shared__ z w[kWY];
      z s = {R(0), R(0)};
      for (int q = 0; q < nw; ++q) s = cadd(s, part[q][threadIdx.x]);
      w[threadIdx.x] = s;
      __syncwarp(0xffu);
      const z* tg = T + (size_t)g * kWY * kWY + threadIdx.x * kWY;
      z ua = {R(0), R(0)};
      for (int c = threadIdx.x; c < nr; ++c) ua = cadd(ua, cmul(tg[c], w[c]));
      u[threadIdx.x] = ua;
    }
    __syncthreads();
    for (int i = j0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      z xi = x[i];
#pragma unroll
      for (int a = 0; a < kWY; ++a) {
        if (((act >> a) & 1u) && i >= j0 + a + 1) xi = csub(xi, cmul(refl[(size_t)(j0 + a) * n + i], u[a]));
      }
      x[i] = xi;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)i * ldx + k] = x[i];
}

#if defined(QE_DENSE_FP64)
// k_wy_t and k_backtransform on the packed float-float reflector rows that
// k_tridiag_rows_ff leaves (the FP64 path): the dot products and the updates of
// the eigenvectors in float-float on the FP32 pipes, T and the results in double.
__device__ __forceinline__ ff2 pk_of_z(z a) { return as2(cx_from<ff>(a.x, a.y)); }

__global__ void __launch_bounds__(256) k_wy_t_ff(const z* __restrict__ refl, int n,
                                                 const z* __restrict__ tau, z* __restrict__ T) {
  __shared__ z P[kWY][kWY];
  const int g = blockIdx.x, j0 = g * kWY, nr = min(kWY, n - 1 - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const cx<ff>* rf = reinterpret_cast<const cx<ff>*>(refl);
  for (int pq = warp; pq < kWY * kWY; pq += nw) {
    const int a = pq / kWY, bb = pq % kWY;
    if (!(a < bb && bb < nr)) continue;
    const z ta = tau[j0 + a], tb = tau[j0 + bb];
    if ((ta.x == R(0) && ta.y == R(0)) || (tb.x == R(0) && tb.y == R(0))) {
      if (lane == 0) P[a][bb] = {R(0), R(0)};
      continue;
    }
    const cx<ff>* va = rf + (size_t)(j0 + a) * n;
    const cx<ff>* vb = rf + (size_t)(j0 + bb) * n;
    ff2 acc = pk_zero();
    for (int i = j0 + bb + 1 + lane; i < n; i += 32) acc = pk_fma(pk_conj(as2(va[i])), as2(vb[i]), acc);
    acc = ff2_settle(acc);
    for (int o = 16; o > 0; o >>= 1) acc = acc + pk_shfl_xor(acc, o);
    if (lane == 0) P[a][bb] = pk_to_z(ff2_settle(acc));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    z t[kWY][kWY];
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) t[r][c] = {R(0), R(0)};
    for (int i = 0; i < nr; ++i) {
      const z ti = tau[j0 + i];
      for (int r = 0; r < i; ++r) {
        z acc = {R(0), R(0)};
        for (int c = r; c < i; ++c) acc = cadd(acc, cmul(t[r][c], P[c][i]));
        t[r][i] = {-(ti.x * acc.x - ti.y * acc.y), -(ti.x * acc.y + ti.y * acc.x)};
      }
      t[i][i] = ti;
    }
    z* out = T + (size_t)g * kWY * kWY;
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) out[r * kWY + c] = t[r][c];
  }
}

__global__ void __launch_bounds__(256) k_backtransform_ff(const z* __restrict__ refl, int n,
                                                          const z* __restrict__ T, const R* Y,
                                                          z* X, int ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<ff>* x = reinterpret_cast<cx<ff>*>(smem_raw);
  __shared__ cx<ff> part[8][kWY];
  __shared__ cx<ff> u[kWY];
  __shared__ cx<ff> w[kWY];
  const cx<ff>* rf = reinterpret_cast<const cx<ff>*>(refl);
  const int k = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = cx_from<ff>(Y[(size_t)k * n + i], 0.0);
  __syncthreads();
  const int ngroups = (n - 1 + kWY - 1) / kWY;
  for (int g = ngroups - 1; g >= 0; --g) {
    const int j0 = g * kWY;
    const z* tg0 = T + (size_t)g * kWY * kWY;
    unsigned act = 0;
    const int nr = min(kWY, n - 1 - j0);
#pragma unroll
    for (int a = 0; a < kWY; ++a) {
      const z d = tg0[a * kWY + a];
      if (a < nr && (d.x != R(0) || d.y != R(0))) act |= 1u << a;
    }
    ff2 acc[kWY];
#pragma unroll
    for (int a = 0; a < kWY; ++a) acc[a] = pk_zero();
    for (int i = j0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const ff2 xi = as2(x[i]);
#pragma unroll
      for (int a = 0; a < kWY; ++a)
        if (((act >> a) & 1u) && i >= j0 + a + 1)
          acc[a] = pk_fma(pk_conj(as2(rf[(size_t)(j0 + a) * n + i])), xi, acc[a]);
    }
#pragma unroll
    for (int a = 0; a < kWY; ++a) {
      ff2 s = ff2_settle(acc[a]);
      for (int o = 16; o > 0; o >>= 1) s = s + pk_shfl_xor(s, o);
      if (lane == 0) part[warp][a] = of2(ff2_settle(s));
    }
    __syncthreads();
    if (threadIdx.x < kWY) {
      // w_c = sum over warps, then u_a = sum_{c >= a} T[a][c] w_c (c < nr)
      ff2 s = as2(part[0][threadIdx.x]);
      for (int q = 1; q < nw; ++q) s = s + as2(part[q][threadIdx.x]);
      w[threadIdx.x] = of2(ff2_settle(s));
      __syncwarp(0xffu);
      const z* tg = T + (size_t)g * kWY * kWY + threadIdx.x * kWY;
      ff2 ua = pk_zero();
      for (int c = threadIdx.x; c < nr; ++c) ua = pk_fma(pk_of_z(tg[c]), as2(w[c]), ua);
      u[threadIdx.x] = of2(ff2_settle(ua));
    }
    __syncthreads();
    for (int i = j0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      ff2 xi = as2(x[i]);
#pragma unroll
      for (int a = 0; a < kWY; ++a)
        if (((act >> a) & 1u) && i >= j0 + a + 1)
          xi = pk_fma(pk_neg(as2(rf[(size_t)(j0 + a) * n + i])), as2(u[a]), xi);
      x[i] = of2(ff2_settle(xi));
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)i * ldx + k] = pk_to_z(as2(x[i]));
}

// ---- the back-transformation of the real symmetric form ----------------------------
// k_tridiag_real_ff leaves reflector row j pair-packed (pair P = entries 2P and
// 2P+1, zero below j+1, every pair of the row written); these are k_wy_t_ff and
// k_backtransform_ff on real pairs: each f32x2 lane pair carries two entries of
// a real vector, the dot products of a group leave the warp in the transposing
// butterfly, and T (real) is kept in the complex format with zero imaginary parts.
// n <= 2 * 2 * 256.
__device__ __forceinline__ const cx<ff>* refl_pairs(const z* refl, int n, int j) {
  return reinterpret_cast<const cx<ff>*>(refl + (size_t)j * n);
}

__global__ void __launch_bounds__(256) k_wy_t_real_ff(const z* __restrict__ refl, int n,
                                                      const z* __restrict__ tau, z* __restrict__ T) {
  __shared__ z P[kWY][kWY];
  const int g = blockIdx.x, j0 = g * kWY, nr = min(kWY, n - 1 - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int NP = (n + 1) >> 1;
  for (int pq = warp; pq < kWY * kWY; pq += nw) {
    const int a = pq / kWY, bb = pq % kWY;
    if (!(a < bb && bb < nr)) continue;
    const z ta = tau[j0 + a], tb = tau[j0 + bb];
    if (ta.x == R(0) || tb.x == R(0)) {
      if (lane == 0) P[a][bb] = {R(0), R(0)};
      continue;
    }
    const cx<ff>* va = refl_pairs(refl, n, j0 + a);
    const cx<ff>* vb = refl_pairs(refl, n, j0 + bb);
    ff2 acc = pk_zero();
    for (int p = ((j0 + bb + 1) >> 1) + lane; p < NP; p += 32) acc = fma(as2(va[p]), as2(vb[p]), acc);
    acc = ff2_settle(acc);
    for (int o = 16; o > 0; o >>= 1) acc = acc + pk_shfl_xor(acc, o);
    if (lane == 0) P[a][bb] = {ffs_to_d(ffs_add(pk_get_re(acc), pk_get_im(acc))), R(0)};
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    z t[kWY][kWY];
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) t[r][c] = {R(0), R(0)};
    for (int i = 0; i < nr; ++i) {
      const z ti = tau[j0 + i];
      for (int r = 0; r < i; ++r) {
        z acc = {R(0), R(0)};
        for (int c = r; c < i; ++c) acc = cadd(acc, cmul(t[r][c], P[c][i]));
        t[r][i] = {-(ti.x * acc.x - ti.y * acc.y), -(ti.x * acc.y + ti.y * acc.x)};
      }
      t[i][i] = ti;
    }
    z* out = T + (size_t)g * kWY * kWY;
    for (int r = 0; r < kWY; ++r)
      for (int c = 0; c < kWY; ++c) out[r * kWY + c] = t[r][c];
  }
}

__global__ void __launch_bounds__(256) k_backtransform_real_ff(const z* __restrict__ refl, int n,
                                                               const z* __restrict__ T,
                                                               const R* Y, z* X, int ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int U = 2;
  cx<ff>* x = reinterpret_cast<cx<ff>*>(smem_raw);   // pair-packed eigenvector
  __shared__ cx<ff> part[8][kWY];
  __shared__ ff wv[kWY], uv[kWY];
  const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int NP = (n + 1) >> 1;
  for (int p = tid; p < NP; p += nt) {
    const ff a0 = ff(Y[(size_t)k * n + 2 * p]);
    const ff a1 = 2 * p + 1 < n ? ff(Y[(size_t)k * n + 2 * p + 1]) : ff(0.f, 0.f);
    x[p] = of2(pk_make(a0, a1));
  }
  __syncthreads();
  const int ngroups = (n - 1 + kWY - 1) / kWY;
  for (int g = ngroups - 1; g >= 0; --g) {
    const int j0 = g * kWY, p0 = (j0 + 1) >> 1;
    const int nr = min(kWY, n - 1 - j0);
    const z* tg0 = T + (size_t)g * kWY * kWY;
    unsigned act = 0;
#pragma unroll
    for (int a = 0; a < kWY; ++a)
      if (a < nr && tg0[a * kWY + a].x != R(0)) act |= 1u << a;
    // w_a = v_a . x over the pairs from p0 (v_a is zero below its own start)
    ff2 acc[kWY];
#pragma unroll
    for (int a = 0; a < kWY; ++a) acc[a] = pk_zero();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + tid + u * nt;
      if (p < NP) {
        const ff2 xp = as2(x[p]);
#pragma unroll
        for (int a = 0; a < kWY; ++a)
          if ((act >> a) & 1u) acc[a] = fma(as2(refl_pairs(refl, n, j0 + a)[p]), xp, acc[a]);
      }
    }
#pragma unroll
    for (int a = 0; a < kWY; ++a) acc[a] = ff2_settle(acc[a]);
    const ff2 s8 = pk_warp_rows8(acc);
    if ((lane & 3) == 0) part[warp][lane >> 2] = of2(ff2_settle(s8));
    __syncthreads();
    if (warp == 0) {
      if (lane < kWY) {
        ff2 s = as2(part[0][lane]);
        for (int q = 1; q < nw; ++q) s = s + as2(part[q][lane]);
        s = ff2_settle(s);
        wv[lane] = ffs_add(pk_get_re(s), pk_get_im(s));
      }
      __syncwarp();
      if (lane < kWY) {
        // u_a = sum_{c >= a} T[a][c] w_c (c < nr)
        const z* tg = tg0 + lane * kWY;
        ff ua = ff(0.f, 0.f);
        for (int c = lane; c < nr; ++c) ua = ffs_add(ua, ffs_mul(ff(tg[c].x), wv[c]));
        uv[lane] = ua;
      }
    }
    __syncthreads();
    // x -= sum_a v_a u_a
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + tid + u * nt;
      if (p < NP) {
        ff2 xp = as2(x[p]);
#pragma unroll
        for (int a = 0; a < kWY; ++a)
          if ((act >> a) & 1u)
            xp = fma(pk_neg(as2(refl_pairs(refl, n, j0 + a)[p])), ff2_bcast(uv[a]), xp);
        x[p] = of2(ff2_settle(xp));
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) X[(size_t)i * ldx + k] = {ffs_to_d(pk_elem(x, i)), R(0)};
}
#endif

// Eigenvalues and eigenvectors of the tridiagonal T (wk.d, wk.e) and the
// back-transformation through the reflectors (wk.tau, wk.refl) into X.
static int heev_finish(int n, int nev, R* w, z* X, int ldx, DenseWorkT<R>& wk, cudaStream_t st,
                       Prof* pf, bool ff_refl = false, bool real_refl = false) {
  int rc = QE_OK;
  {
    ProfScope ps(pf, "heev_bisect", st);
    // two warps per block: the Sturm counts are FP64-bound, so spread them over the SMs
    const size_t bsm_b = (size_t)n * (2 * sizeof(R) + (sizeof(R) == 8 ? 2 * sizeof(float) + 2 * sizeof(ff) : 0));
    set_max_dynamic_smem(k_bisect);
    k_bisect<<<(nev * 32 + 63) / 64, 64, bsm_b, st>>>(wk.d, wk.e, n, nev, w);
  }
  rc = check_launch("k_bisect");
  if (rc) return rc;
  // same (largest) cap for every caller: the attribute is shared process-wide
  set_max_dynamic_smem(k_backtransform);
  // eigenvalues within 1e-10 of each other (relative to the spread of T) share a cluster
#if defined(QE_DENSE_FP64)
  {
    const size_t ism = (size_t)n * (7 * sizeof(ff) + sizeof(int));
    set_max_dynamic_smem(k_inviter_ff);
    ProfScope ps(pf, "heev_inviter", st);
    k_inviter_ff<<<nev, 256, ism, st>>>(wk.d, wk.e, n, nev, w, wk.ctol_rel, wk.y);
  }
#else
  {
    const size_t ism = (size_t)n * (5 * sizeof(R) + sizeof(int));
    set_max_dynamic_smem(k_inviter);
    ProfScope ps(pf, "heev_inviter", st);
    k_inviter<<<nev, 256, ism, st>>>(wk.d, wk.e, n, nev, w, wk.ctol_rel, wk.y);
  }
#endif
  rc = check_launch("k_inviter");
  if (rc) return rc;
  const size_t bsm = (size_t)n * sizeof(z);
  {
    ProfScope ps(pf, "heev_backtransform", st);
#if defined(QE_DENSE_FP64)
    if (real_refl) {
      set_max_dynamic_smem(k_backtransform_real_ff);
      if (n > 1) k_wy_t_real_ff<<<(n - 1 + kWY - 1) / kWY, 256, 0, st>>>(wk.refl, n, wk.tau, wk.wyt);
      k_backtransform_real_ff<<<nev, 256, ((n + 1) / 2) * sizeof(cx<ff>), st>>>(wk.refl, n, wk.wyt,
                                                                              wk.y, X, ldx);
    } else if (ff_refl) {
      set_max_dynamic_smem(k_backtransform_ff);
      if (n > 1) k_wy_t_ff<<<(n - 1 + kWY - 1) / kWY, 256, 0, st>>>(wk.refl, n, wk.tau, wk.wyt);
      k_backtransform_ff<<<nev, 256, bsm, st>>>(wk.refl, n, wk.wyt, wk.y, X, ldx);
    } else
#endif
    {
      if (n > 1) k_wy_t<<<(n - 1 + kWY - 1) / kWY, 256, 0, st>>>(wk.refl, n, wk.tau, wk.wyt);
      k_backtransform<<<nev, 256, bsm, st>>>(wk.refl, n, wk.wyt, wk.y, X, ldx);
    }
  }
  return check_launch("k_backtransform");
}

// Grid of k_tridiag_rows for an n x n matrix (0: use k_tridiag_coop): one CTA per
// SM (at most n), provided every CTA's rows and vectors fit in shared memory.
// The FP64 instantiation runs the float-float kernel (k_tridiag_rows_ff, the same
// layout and launch shape).
#if defined(QE_DENSE_FP64)
#define QE_TRIDIAG_ROWS k_tridiag_rows_ff
#else
#define QE_TRIDIAG_ROWS k_tridiag_rows
#endif
static int tridiag_rows_grid(int n, size_t* smem) {
  if (n < 16) return 0;
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)QE_TRIDIAG_ROWS) != cudaSuccess) return 0;
  // At least 4 rows per CTA: a grid barrier costs less with fewer arrivals, and
  // reductions of solves that run side by side (lockstep batches, serving)
  // overlap on the SMs.  C3 batched FP64 Davidson 2.03 -> 1.85 s with the
  // one-by-one solves within 2 % and C2 unchanged (one row per CTA before;
  // 8 rows: batched 1.83 s, one-by-one 5 % slower).
  const int g = std::min(nsm, (n + 3) / 4);
  const int nrmax = (n + g - 1) / g;
  if (nrmax > kTridRows) return 0;
  const size_t sm = (size_t)(nrmax + 3) * n * sizeof(z);
  if (sm + fa.sharedSizeBytes > (size_t)optin) return 0;
  set_max_dynamic_smem(QE_TRIDIAG_ROWS);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, QE_TRIDIAG_ROWS, 256, sm) != cudaSuccess ||
      occ < 1)
    return 0;
  *smem = sm;
  return g;
}

#if defined(QE_DENSE_FP64)
// Grid of k_tridiag_real_ff (0: it does not fit): the CTA count of
// k_tridiag_rows_ff, with (ceil(n / G) + 4) ceil(n / 2) pairs of shared memory.
static int tridiag_real_grid(int n, size_t* smem) {
  if (n < 16 || n > 2 * kTridRealU * kTridRealThreads) return 0;
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)k_tridiag_real_ff) != cudaSuccess) return 0;
  const int g = std::min(nsm, (n + 3) / 4);
  const int nrmax = (n + g - 1) / g;
  if (nrmax > kTridRows) return 0;
  const size_t sm = (size_t)(nrmax + 4) * ((n + 1) / 2) * sizeof(cx<ff>);
  if (sm + fa.sharedSizeBytes > (size_t)optin) return 0;
  set_max_dynamic_smem(k_tridiag_real_ff);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tridiag_real_ff, kTridRealThreads,
                                                    sm) != cudaSuccess ||
      occ < 1)
    return 0;
  *smem = sm;
  return g;
}

#endif

int heev_lowest(z* A, int n, int lda, int nev, R* w, z* X, int ldx, DenseWorkT<R>& wk,
                cudaStream_t st, Prof* pf, bool real_sym) {
  (void)real_sym;   // the FP32 instantiation reduces every matrix in complex form
  if (n <= 0 || nev <= 0) return QE_OK;
  if (nev > n || n > kMaxDense) {
    set_error("heev_lowest: n = %d, nev = %d (max n %d)", n, nev, kMaxDense);
    return QE_EINVAL;
  }
  if (cudaMemsetAsync(wk.bar.count, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
    set_error("heev_lowest: memset failed");
    return QE_ECUDA;
  }
  GridBar bar = wk.bar;
  size_t rsm = 0;
#if defined(QE_DENSE_FP64)
  if (real_sym) {
    const int gr = tridiag_real_grid(n, &rsm);
    if (gr > 0) {
      void* args[] = {&A, &n, &lda, &wk.tau, &wk.e, &wk.d, &wk.refl, &bar};
      {
        ProfScope ps(pf, "heev_tridiag", st);
        int rc0 = launch_coop((const void*)k_tridiag_real_ff, gr, args, st, "k_tridiag_real_ff",
                              rsm, kTridRealThreads);
        if (rc0) return rc0;
      }
      return heev_finish(n, nev, w, X, ldx, wk, st, pf, true, true);   // real pair-packed reflectors
    }
  }
#endif
  const int g = tridiag_rows_grid(n, &rsm);
  if (g > 0) {
    void* args[] = {&A, &n, &lda, &wk.tau, &wk.e, &wk.d, &wk.refl, &bar};
    ProfScope ps(pf, "heev_tridiag", st);
    int rc0 = launch_coop((const void*)QE_TRIDIAG_ROWS, g, args, st, "k_tridiag_rows", rsm);
    if (rc0) return rc0;
  } else {
    void* args[] = {&A, &n, &lda, &wk.tau, &wk.e, &wk.p, &wk.d, &wk.vbuf, &wk.refl, &bar};
    const size_t tsm = 2 * (size_t)n * sizeof(z);
    set_max_dynamic_smem(k_tridiag_coop);
    // all SMs once the trailing block is large: the FP64 work is spread
    const int blocks = coop_blocks((const void*)k_tridiag_coop, (size_t)n * n * 4, tsm);
    ProfScope ps(pf, "heev_tridiag", st);
    int rc0 = launch_coop((const void*)k_tridiag_coop, blocks, args, st, "k_tridiag_coop", tsm);
    if (rc0) return rc0;
  }
#if defined(QE_DENSE_FP64)
  return heev_finish(n, nev, w, X, ldx, wk, st, pf, g > 0);   // rows kernel: packed reflectors
#else
  return heev_finish(n, nev, w, X, ldx, wk, st, pf);
#endif
}

// ---- small generalised problems in one CTA ---------------------------------------------
// For n <= kSmallDense the whole reduction runs in one CTA on a shared-memory
// copy of the matrix: the multi-CTA kernels above spend ~15 us per column on
// L2 round trips and barriers even with one CTA, while one SM's FP64 rate
// (1/152 of the GPU) is still enough for n^3 work at this size.
//   S = L L^+ (L -> Lg, lower, upper zeroed; status = 1 + column on a
//   non-positive pivot), A = L^-1 H L^-+, A = Q T Q^+ (T -> d, e; Q as
//   reflectors -> tau, refl rows, as k_tridiag_coop).
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

#if !defined(QE_DENSE_FP64)   // FP64: k_rr_small_ff below
__global__ void __launch_bounds__(512) k_rr_small(const z* __restrict__ H, const z* __restrict__ S,
                                                  int ld, int n, z* Lg, R* dgl, R* egl,
                                                  z* taug, z* refl, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* A = reinterpret_cast<z*>(smem_raw);          // n x n: H, then the reduced matrix
  z* L = A + (size_t)n * n;                        // n x n: S, then its Cholesky factor
  z* sv = L + (size_t)n * n;                       // n
  z* sw = sv + n;                                  // n
  R* piv = reinterpret_cast<R*>(sw + n); // n
  __shared__ R sred[4];
  __shared__ R s_inv;
  __shared__ int s_fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  if (tid == 0) s_fail = 0;
  // 1. Cholesky of S in place (right-looking, lower triangle)
  for (int t = tid; t < n * n; t += nt) {
    L[t] = S[(size_t)(t / n) * ld + t % n];
    A[t] = H[(size_t)(t / n) * ld + t % n];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const R dj = L[(size_t)j * n + j].x;
    if (!(dj > R(0))) {
      if (tid == 0) { s_fail = 1; *status = 1 + j; }
      break;
    }
    // one thread divides (an FP64 division is ~10 dependent FP64 instructions,
    // each a whole warp-instruction slot of the narrow FP64 pipe)
    if (tid == 0) { piv[j] = sqrt(dj); s_inv = R(1) / dj; }
    __syncthreads();
    const R inv = s_inv;
    const int m = n - j - 1;
    for (int t = tid; t < m * m; t += nt) {
      const int r = j + 1 + t / m, c = j + 1 + t % m;
      if (c > r) continue;
      const z arj = L[(size_t)r * n + j], acj = L[(size_t)c * n + j];
      z& a = L[(size_t)r * n + c];
      a = {a.x - (arj.x * acj.x + arj.y * acj.y) * inv, a.y - (arj.y * acj.x - arj.x * acj.y) * inv};
    }
    __syncthreads();
  }
  __syncthreads();
  if (s_fail) {
    for (int i = tid; i < n; i += nt) { dgl[i] = R(0); egl[i] = R(0); taug[i] = {R(0), R(0)}; }
    return;
  }
  // reciprocal pivots, one division per thread
  R* rpiv = reinterpret_cast<R*>(sw);
  for (int i = tid; i < n; i += nt) rpiv[i] = R(1) / piv[i];
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t % n;
    const z a = L[t];
    const z l = c > r ? z{R(0), R(0)} : (c == r ? z{piv[c], R(0)} : z{a.x * rpiv[c], a.y * rpiv[c]});
    L[t] = l;
    Lg[t] = l;
  }
  __syncthreads();
  // 2. A = L^-1 H L^-+: two forward substitutions (rows in order, columns in
  // parallel: for n <= 32 the lanes of one warp, whose FP64 instructions cost
  // the same for 1 or 32 active lanes); reciprocal pivots instead of a division
  // per row in every thread
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n; ++i) {
      const z* li = L + (size_t)i * n;
      const R inv = rpiv[i];
      for (int c = tid; c < n; c += nt) {
        z acc = A[(size_t)i * n + c];
        for (int k = 0; k < i; ++k) {
          const z l = li[k], x = A[(size_t)k * n + c];
          acc.x = fmar(-l.x, x.x, fmar(l.y, x.y, acc.x));
          acc.y = fmar(-l.x, x.y, fmar(-l.y, x.x, acc.y));
        }
        A[(size_t)i * n + c] = {acc.x * inv, acc.y * inv};
      }
      __syncthreads();
    }
    if (pass == 0) {
      // A <- A^+ (then the second substitution gives L^-1 (L^-1 H)^+ = L^-1 H L^-+)
      for (int t = tid; t < n * n; t += nt) {
        const int r = t / n, c = t % n;
        if (c < r) continue;
        const z a = A[t], b = A[(size_t)c * n + r];
        A[t] = {b.x, -b.y};
        A[(size_t)c * n + r] = {a.x, -a.y};
      }
      __syncthreads();
    }
  }
  // Hermitian part
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t % n;
    if (c < r) continue;
    const z a = A[t], b = A[(size_t)c * n + r];
    const z h = {R(0.5) * (a.x + b.x), R(0.5) * (a.y - b.y)};
    A[t] = h;
    A[(size_t)c * n + r] = {h.x, -h.y};
  }
  __syncthreads();
  // 3. Householder tridiagonalisation in place
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;
    // reflector of column j (warp 0)
    if (warp == 0) {
      const z alpha = A[(size_t)(j + 1) * n + j];
      R sg = R(0);
      for (int i = 1 + lane; i < m; i += 32) {
        const z x = A[(size_t)(j + 1 + i) * n + j];
        sg += x.x * x.x + x.y * x.y;
      }
      sg = warp_sum(sg);
      if (sg == R(0) && alpha.y == R(0)) {
        if (lane == 0) { taug[j] = {R(0), R(0)}; egl[j] = alpha.x; sred[0] = R(0); sred[1] = R(0); }
      } else {
        const R nu = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + sg);
        const R beta = alpha.x >= R(0) ? -nu : nu;
        const z am = {alpha.x - beta, alpha.y};
        const R rden = R(1) / (am.x * am.x + am.y * am.y), rbeta = R(1) / beta;
        const z sc = {am.x * rden, -am.y * rden};
        z* rrow = refl + (size_t)j * n + (j + 1);
        for (int i = 1 + lane; i < m; i += 32) {
          z* x = &A[(size_t)(j + 1 + i) * n + j];
          const z v = cmul(*x, sc);
          *x = v;
          sv[i] = v;
          rrow[i] = v;
        }
        if (lane == 0) {
          const z t = {(beta - alpha.x) * rbeta, -alpha.y * rbeta};
          taug[j] = t;
          egl[j] = beta;
          A[(size_t)(j + 1) * n + j] = {beta, R(0)};
          sv[0] = {R(1), R(0)};
          rrow[0] = {R(1), R(0)};
          sred[0] = t.x;
          sred[1] = t.y;
        }
      }
    }
    __syncthreads();
    const z t = {sred[0], sred[1]};
    if (t.x == R(0) && t.y == R(0)) {   // uniform: every thread read the same
      __syncthreads();                // before warp 0 writes the next reflector's tau
      continue;
    }
    // p = tau A_trail v (one warp per row)
    for (int r = warp; r < m; r += nwarps) {
      const z* row = A + (size_t)(j + 1 + r) * n + (j + 1);
      R ax = R(0), ay = R(0);
      for (int c = lane; c < m; c += 32) {
        const z a = row[c], v = sv[c];
        ax += a.x * v.x - a.y * v.y;
        ay += a.x * v.y + a.y * v.x;
      }
      ax = warp_sum(ax);
      ay = warp_sum(ay);
      if (lane == 0) sw[r] = cmul(t, z{ax, ay});
    }
    __syncthreads();
    // w = p - (1/2) conj(tau) (v^+ p) v
    if (warp == 0) {
      R sr = R(0), si = R(0);
      for (int i = lane; i < m; i += 32) {
        const z v = sv[i], pr = sw[i];
        sr += v.x * pr.x + v.y * pr.y;
        si += v.x * pr.y - v.y * pr.x;
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      if (lane == 0) { sred[2] = R(0.5) * (t.x * sr + t.y * si); sred[3] = R(0.5) * (t.x * si - t.y * sr); }
    }
    __syncthreads();
    const z coef = {sred[2], sred[3]};
    for (int i = tid; i < m; i += nt) sw[i] = csub(sw[i], cmul(coef, sv[i]));
    __syncthreads();
    // A_trail -= v w^+ + w v^+
    for (int q = tid; q < m * m; q += nt) {
      const int r = q / m, c = q % m;
      const z dlt = cadd(cmul(sv[r], zconj(sw[c])), cmul(sw[r], zconj(sv[c])));
      z& a = A[(size_t)(j + 1 + r) * n + (j + 1 + c)];
      a = csub(a, dlt);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) dgl[i] = A[(size_t)i * n + i].x;
}
#endif

#if defined(QE_DENSE_FP64)
// k_rr_small in float-float arithmetic (the FP64 path): the same steps, order
// and layout on packed float-float complex values, whose dependent chains
// (the substitutions, the reductions, the pivots' square roots and divisions)
// are far shorter on the FP32 pipes than on GB300's FP64 pipe.  Lg, d, e and tau
// leave in double, the reflector rows packed float-float (k_backtransform_ff).
__device__ __forceinline__ ff2 pk_warp_sum(ff2 a) {
  for (int o = 16; o > 0; o >>= 1) a = a + pk_shfl_xor(a, o);
  return ff2_settle(a);
}
__global__ void __launch_bounds__(512) k_rr_small_ff(const z* __restrict__ H,
                                                     const z* __restrict__ S, int ld, int n,
                                                     z* Lg, R* dgl, R* egl, z* taug, z* refl,
                                                     int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<ff>* A = reinterpret_cast<cx<ff>*>(smem_raw);   // n x n: H, then the reduced matrix
  cx<ff>* L = A + (size_t)n * n;                     // n x n: S, then its Cholesky factor
  cx<ff>* sv = L + (size_t)n * n;                    // n
  cx<ff>* sw = sv + n;                               // n
  ff* piv = reinterpret_cast<ff*>(sw + n);           // n
  ff* rpiv = piv + n;                                // n
  __shared__ cx<ff> sred[2];                          // tau, coefficient of w
  __shared__ ff s_inv;
  __shared__ int s_fail;
  cx<ff>* rf = reinterpret_cast<cx<ff>*>(refl);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  if (tid == 0) s_fail = 0;
  // 1. Cholesky of S in place (right-looking, lower triangle)
  for (int t = tid; t < n * n; t += nt) {
    const z sv0 = S[(size_t)(t / n) * ld + t % n], hv0 = H[(size_t)(t / n) * ld + t % n];
    L[t] = cx_from<ff>(sv0.x, sv0.y);
    A[t] = cx_from<ff>(hv0.x, hv0.y);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const ff dj = pk_get_re(as2(L[(size_t)j * n + j]));
    if (!(dj.hi > 0.f)) {
      if (tid == 0) { s_fail = 1; *status = 1 + j; }
      break;
    }
    if (tid == 0) { piv[j] = ffs_sqrt(dj); s_inv = ffs_div(ff(1.f, 0.f), dj); }
    __syncthreads();
    const ff2 inv = ff2_bcast(s_inv);
    const int m = n - j - 1;
    for (int t = tid; t < m * m; t += nt) {
      const int r = j + 1 + t / m, c = j + 1 + t % m;
      if (c > r) continue;
      const ff2 p = pk_mul(as2(L[(size_t)r * n + j]), pk_conj(as2(L[(size_t)c * n + j])));
      cx<ff>& a = L[(size_t)r * n + c];
      a = of2(ff2_settle(as2(a) - p * inv));
    }
    __syncthreads();
  }
  __syncthreads();
  if (s_fail) {
    for (int i = tid; i < n; i += nt) { dgl[i] = R(0); egl[i] = R(0); taug[i] = {R(0), R(0)}; }
    return;
  }
  for (int i = tid; i < n; i += nt) rpiv[i] = ffs_div(ff(1.f, 0.f), piv[i]);
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t % n;
    ff2 l;
    if (c > r) l = pk_zero();
    else if (c == r) l = pk_make(piv[c], ff(0.f, 0.f));
    else l = ff2_settle(as2(L[t]) * ff2_bcast(rpiv[c]));
    L[t] = of2(l);
    Lg[t] = pk_to_z(l);
  }
  __syncthreads();
  // 2. A = L^-1 H L^-+: two forward substitutions, columns in parallel
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n; ++i) {
      const cx<ff>* li = L + (size_t)i * n;
      const ff2 inv = ff2_bcast(rpiv[i]);
      for (int c = tid; c < n; c += nt) {
        ff2 acc = as2(A[(size_t)i * n + c]);
        for (int k = 0; k < i; ++k) acc = pk_fma(pk_neg(as2(li[k])), as2(A[(size_t)k * n + c]), acc);
        A[(size_t)i * n + c] = of2(ff2_settle(ff2_settle(acc) * inv));
      }
      __syncthreads();
    }
    if (pass == 0) {
      for (int t = tid; t < n * n; t += nt) {
        const int r = t / n, c = t % n;
        if (c < r) continue;
        const ff2 a = as2(A[t]), b = as2(A[(size_t)c * n + r]);
        A[t] = of2(pk_conj(b));
        A[(size_t)c * n + r] = of2(pk_conj(a));
      }
      __syncthreads();
    }
  }
  // Hermitian part
  {
    const ff2 half = {f2_of(0.5f, 0.5f), f2_of(0.5f, 0.5f)};
    for (int t = tid; t < n * n; t += nt) {
      const int r = t / n, c = t % n;
      if (c < r) continue;
      const ff2 hs = as2(A[t]) + pk_conj(as2(A[(size_t)c * n + r]));
      const ff2 h = ff2_settle({mul2(hs.hi, half.hi), mul2(hs.lo, half.lo)});
      A[t] = of2(h);
      A[(size_t)c * n + r] = of2(pk_conj(h));
    }
  }
  __syncthreads();
  // 3. Householder tridiagonalisation in place
  const ff2 one = {f2_of(1.f, 0.f), f2_of(0.f, 0.f)};
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;
    if (warp == 0) {
      const ff2 alpha = as2(A[(size_t)(j + 1) * n + j]);
      ff2 ss = pk_zero();
      for (int i = 1 + lane; i < m; i += 32) {
        const ff2 x = as2(A[(size_t)(j + 1 + i) * n + j]);
        ss = x * x + ss;
      }
      ss = pk_warp_sum(ff2_settle(ss));
      const ff sg = ffs_add(pk_get_re(ss), pk_get_im(ss));
      const ff ar = pk_get_re(alpha), ai = pk_get_im(alpha);
      if (sg.hi == 0.f && ai.hi == 0.f) {
        if (lane == 0) { taug[j] = {R(0), R(0)}; egl[j] = ffs_to_d(ar); sred[0] = of2(pk_zero()); }
      } else {
        const ff nu = ffs_sqrt(ffs_add(ffs_add(ffs_mul(ar, ar), ffs_mul(ai, ai)), sg));
        const ff beta = ar.hi >= 0.f ? ffs_neg(nu) : nu;
        const ff amr = ffs_sub(ar, beta);
        const ff rden = ffs_div(ff(1.f, 0.f), ffs_add(ffs_mul(amr, amr), ffs_mul(ai, ai)));
        const ff rbeta = ffs_div(ff(1.f, 0.f), beta);
        const ff2 sc = pk_make(ffs_mul(amr, rden), ffs_neg(ffs_mul(ai, rden)));
        cx<ff>* rrow = rf + (size_t)j * n + (j + 1);
        for (int i = 1 + lane; i < m; i += 32) {
          cx<ff>* x = &A[(size_t)(j + 1 + i) * n + j];
          const cx<ff> v = of2(ff2_settle(pk_mul(as2(*x), sc)));
          *x = v;
          sv[i] = v;
          rrow[i] = v;
        }
        if (lane == 0) {
          const ff2 t = pk_make(ffs_mul(ffs_sub(beta, ar), rbeta), ffs_neg(ffs_mul(ai, rbeta)));
          taug[j] = pk_to_z(t);
          egl[j] = ffs_to_d(beta);
          A[(size_t)(j + 1) * n + j] = of2(pk_make(beta, ff(0.f, 0.f)));
          sv[0] = of2(one);
          rrow[0] = of2(one);
          sred[0] = of2(t);
        }
      }
    }
    __syncthreads();
    const ff2 t = as2(sred[0]);
    {
      float th, tih, tl, til;
      f2_split(t.hi, th, tih);
      f2_split(t.lo, tl, til);
      if (th == 0.f && tih == 0.f && tl == 0.f && til == 0.f) {   // uniform
        __syncthreads();
        continue;
      }
    }
    // p = tau A_trail v (one warp per row)
    for (int r = warp; r < m; r += nwarps) {
      const cx<ff>* row = A + (size_t)(j + 1 + r) * n + (j + 1);
      ff2 acc = pk_zero();
      for (int c = lane; c < m; c += 32) acc = pk_fma(as2(row[c]), as2(sv[c]), acc);
      acc = pk_warp_sum(ff2_settle(acc));
      if (lane == 0) sw[r] = of2(ff2_settle(pk_mul(t, acc)));
    }
    __syncthreads();
    // w = p - (1/2) conj(tau) (v^+ p) v
    if (warp == 0) {
      ff2 acc = pk_zero();
      for (int i = lane; i < m; i += 32) acc = pk_fma(pk_conj(as2(sv[i])), as2(sw[i]), acc);
      acc = pk_warp_sum(ff2_settle(acc));
      if (lane == 0) {
        const ff2 cf = ff2_settle(pk_mul(pk_conj(t), acc));
        const ff2 half = {f2_of(0.5f, 0.5f), f2_of(0.5f, 0.5f)};
        sred[1] = of2(ff2{mul2(cf.hi, half.hi), mul2(cf.lo, half.lo)});
      }
    }
    __syncthreads();
    const ff2 ncoef = pk_neg(as2(sred[1]));
    for (int i = tid; i < m; i += nt) sw[i] = of2(ff2_settle(pk_fma(ncoef, as2(sv[i]), as2(sw[i]))));
    __syncthreads();
    // A_trail -= v w^+ + w v^+
    for (int q = tid; q < m * m; q += nt) {
      const int r = q / m, c = q % m;
      cx<ff>& a = A[(size_t)(j + 1 + r) * n + (j + 1 + c)];
      ff2 x = pk_fma(pk_neg(as2(sv[r])), pk_conj(as2(sw[c])), as2(a));
      x = pk_fma(pk_neg(as2(sw[r])), pk_conj(as2(sv[c])), x);
      a = of2(ff2_settle(x));
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) dgl[i] = ffs_to_d(pk_get_re(as2(A[(size_t)i * n + i])));
}
#endif

int rr_small_fits(int n) { return n > 0 && n <= kSmallDense; }

int rr_small(const z* H, const z* S, int ld, int n, int nev, z* L, R* w, z* X, int ldx,
             DenseWorkT<R>& wk, cudaStream_t st, Prof* pf) {
  if (!rr_small_fits(n) || nev <= 0 || nev > n) {
    set_error("rr_small: n = %d, nev = %d", n, nev);
    return QE_EINVAL;
  }
#if defined(QE_DENSE_FP64)
  const size_t smem = 2 * (size_t)n * n * sizeof(z) + 2 * (size_t)n * sizeof(z) + 2 * (size_t)n * sizeof(ff);
  set_max_dynamic_smem(k_rr_small_ff);
  {
    ProfScope ps(pf, "rr_small", st);
    k_rr_small_ff<<<1, 512, smem, st>>>(H, S, ld, n, L, wk.d, wk.e, wk.tau, wk.refl, wk.status);
  }
  const int rc = check_launch("k_rr_small");
  if (rc) return rc;
  return heev_finish(n, nev, w, X, ldx, wk, st, pf, true);
#else
  const size_t smem = 2 * (size_t)n * n * sizeof(z) + 2 * (size_t)n * sizeof(z) + (size_t)n * sizeof(R);
  set_max_dynamic_smem(k_rr_small);
  {
    ProfScope ps(pf, "rr_small", st);
    k_rr_small<<<1, 512, smem, st>>>(H, S, ld, n, L, wk.d, wk.e, wk.tau, wk.refl, wk.status);
  }
  const int rc = check_launch("k_rr_small");
  if (rc) return rc;
  return heev_finish(n, nev, w, X, ldx, wk, st, pf);
#endif
}


}  // namespace QE_DENSE_NS
