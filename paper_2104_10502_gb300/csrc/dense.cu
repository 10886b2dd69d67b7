// FP64 complex dense linear algebra of the Rayleigh-Ritz step and of the
// Cholesky orthonormalisation (Sec. 3.2.1 of the paper: LAXlib, parallel dense
// linear algebra and diagonalisation; Sec. 3.3: generalized eigenproblems).
//
// Matrices are row-major complex (interleaved doubles), A[i][j] at i*lda + j.
//   cholesky      right-looking, one launch per column, optional dropping of
//                 columns whose remaining pivot is below a threshold (this is
//                 Gram-Schmidt with dropping, expressed on the Gram matrix);
//   trsm_lower    L X = B, column-parallel forward substitution;
//   trsm_upper_h  L^+ X = B, column-parallel back substitution;
//   heev_lowest   lowest eigenpairs of a Hermitian matrix: Householder
//                 tridiagonalisation (real off-diagonal), Sturm bisection,
//                 inverse iteration with re-orthogonalisation inside clusters
//                 of (nearly) equal eigenvalues, back-transformation.
// Every kernel is a plain data-parallel launch; there is no inter-CTA waiting.
#include <algorithm>
#include <cmath>

#include "dense.h"
#include "plan.h"
#include "fft_device.cuh"

namespace qe {

using z = cx<double>;

static int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

__device__ __forceinline__ z zconj(z a) { return {a.x, -a.y}; }
__device__ __forceinline__ double zabs2(z a) { return a.x * a.x + a.y * a.y; }

// Block-wide sum (blockDim.x a multiple of 32, <= 1024).  Every thread gets the result.
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
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
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ double ldd(const double* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Every wait
// is bounded (2 s); on time-out the error word is set, every later barrier
// returns false at once and the kernel leaves.
__device__ bool grid_sync(const GridBar& b) {
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)b.err == 0) {
    const unsigned int g = *(volatile unsigned int*)b.gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(b.count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      const unsigned long long t0 = gtime_ns();
      while (*(volatile unsigned int*)b.gen == g) {
        if (*(volatile int*)b.err) break;
        if (gtime_ns() - t0 > 2000000000ull) { atomicExch(b.err, 1); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)b.err == 0;
}

// Cholesky of the lower triangle, all columns in one launch (one barrier per column).
__global__ void __launch_bounds__(256) k_chol_coop(z* A, int n, int lda, double drop2, int allow_drop,
                                                   double* piv, int* status, GridBar bar) {
  const size_t nthr = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = 0; j < n; ++j) {
    const double d = ldz(&A[(size_t)j * lda + j]).x;
    const bool keep = allow_drop ? (d > drop2) : (d > 0.0);
    if (gtid == 0) {
      piv[j] = keep ? sqrt(d) : 0.0;
      if (!keep && !allow_drop) *status = 1 + j;
    }
    if (keep) {
      const double inv = 1.0 / d;
      const int m = n - j - 1;
      const size_t total = (size_t)m * m;
      for (size_t t = gtid; t < total; t += nthr) {
        const int r = j + 1 + (int)(t / m), c = j + 1 + (int)(t % m);
        if (c > r) continue;
        const z arj = ldz(&A[(size_t)r * lda + j]), acj = ldz(&A[(size_t)c * lda + j]);
        z& a = A[(size_t)r * lda + c];
        const z av = ldz(&a);
        a = {av.x - (arj.x * acj.x + arj.y * acj.y) * inv, av.y - (arj.y * acj.x - arj.x * acj.y) * inv};
      }
    }
    if (!grid_sync(bar)) return;
  }
  const size_t total = (size_t)n * n;
  for (size_t t = gtid; t < total; t += nthr) {
    const int i = (int)(t / n), j = (int)(t % n);
    z& a = A[(size_t)i * lda + j];
    const double pj = ldd(&piv[j]);
    if (j > i || pj == 0.0) { a = {0.0, 0.0}; continue; }
    if (i == j) { a = {pj, 0.0}; continue; }
    const z av = ldz(&a);
    a = {av.x / pj, av.y / pj};
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
                       size_t smem = 0) {
  cudaError_t e = cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(256), args, smem, st);
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

int cholesky(z* A, int n, int lda, double drop2, bool allow_drop, double* piv, int* status,
             GridBar bar, cudaStream_t st) {
  if (n <= 0) return QE_OK;
  if (cudaMemsetAsync(bar.count, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
    set_error("cholesky: memset failed");
    return QE_ECUDA;
  }
  int allow = allow_drop ? 1 : 0;
  void* args[] = {&A, &n, &lda, &drop2, &allow, &piv, &status, &bar};
  const int blocks = coop_blocks((const void*)k_chol_coop, (size_t)n * n / 2);
  return launch_coop((const void*)k_chol_coop, blocks, args, st, "k_chol_coop");
}

// ---- triangular solves ---------------------------------------------------------
constexpr int TCOLS = 4;

// L X = B, L lower with real positive diagonal; B [n][ldb], columns c0.. of this CTA.
__global__ void __launch_bounds__(256) k_trsm_lower(const z* L, int n, int ldl, z* B, int ldb,
                                                    int ncols) {
  const int c0 = blockIdx.x * TCOLS;
  const int nc = min(TCOLS, ncols - c0);
  for (int i = 0; i < n; ++i) {
    if (threadIdx.x < nc) {
      const double inv = 1.0 / L[(size_t)i * ldl + i].x;
      z& b = B[(size_t)i * ldb + c0 + threadIdx.x];
      b = {b.x * inv, b.y * inv};
    }
    __syncthreads();
    const int rows = n - i - 1;
    for (int t = threadIdx.x; t < rows * nc; t += blockDim.x) {
      const int r = i + 1 + t / nc, c = c0 + t % nc;
      const z l = L[(size_t)r * ldl + i], x = B[(size_t)i * ldb + c];
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
      const double inv = 1.0 / L[(size_t)i * ldl + i].x;
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

int trsm_lower(const z* L, int n, int ldl, z* B, int ldb, int ncols, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return QE_OK;
  k_trsm_lower<<<(ncols + TCOLS - 1) / TCOLS, 256, 0, st>>>(L, n, ldl, B, ldb, ncols);
  return check_launch("k_trsm_lower");
}

int trsm_upper_h(const z* L, int n, int ldl, z* B, int ldb, int ncols, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return QE_OK;
  k_trsm_upper_h<<<(ncols + TCOLS - 1) / TCOLS, 256, 0, st>>>(L, n, ldl, B, ldb, ncols);
  return check_launch("k_trsm_upper_h");
}

// ---- element-wise helpers ------------------------------------------------------
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
    const z m = {0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
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
__device__ void house_step(z* A, int n, int lda, int j, z* tau, double* e, z* vbuf, z* refl,
                           double* sh) {
  const int m = n - j - 1;
  const z alpha = ldz(&A[(size_t)(j + 1) * lda + j]);
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) s += zabs2(ldz(&A[(size_t)(j + 1 + i) * lda + j]));
  const double sigma = block_sum(s, sh);
  if (sigma == 0.0 && alpha.y == 0.0) {
    if (threadIdx.x == 0) { tau[j] = {0.0, 0.0}; e[j] = alpha.x; }
    return;
  }
  const double nu = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + sigma);
  const double beta = alpha.x >= 0.0 ? -nu : nu;
  const z am = {alpha.x - beta, alpha.y};
  const double den = am.x * am.x + am.y * am.y;
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
    A[(size_t)(j + 1) * lda + j] = {beta, 0.0};
    vbuf[0] = {1.0, 0.0};
    rrow[0] = {1.0, 0.0};
  }
}

// Householder tridiagonalisation, all steps in one launch, two barriers per
// step: (matvec p = tau A v) | (rank-2 update A -= v w^+ + w v^+, and, in CTA 0,
// the update of the next column followed by the next reflector).  The
// reflector is also kept contiguous in vbuf; every CTA stages v and w of the
// step in shared memory, so the two phases stream only the trailing block of A.
// Dynamic shared memory: 2 n complex.
__global__ void __launch_bounds__(256) k_tridiag_coop(z* A, int n, int lda, z* tau, double* e, z* p,
                                                      double* dg, z* vbuf, z* refl, GridBar bar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* sv = reinterpret_cast<z*>(smem_raw);
  z* sw = sv + n;
  __shared__ double sh[33];
  const size_t nthr = (size_t)gridDim.x * blockDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nwarp = (int)(nthr >> 5), gwarp = (int)(gtid >> 5), lane = threadIdx.x & 31;
  if (n >= 2 && blockIdx.x == 0) house_step(A, n, lda, 0, tau, e, vbuf, refl, sh);
  if (!grid_sync(bar)) return;
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;
    const z t = ldz(&tau[j]);
    const bool active = t.x != 0.0 || t.y != 0.0;
    if (active) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = ldz(&vbuf[i]);
      __syncthreads();
      // p = tau A v over the trailing block (one warp per row)
      for (int w = gwarp; w < m; w += nwarp) {
        const z* row = A + (size_t)(j + 1 + w) * lda + (j + 1);
        z acc = {0.0, 0.0};
        for (int c = lane; c < m; c += 32) acc = cadd(acc, cmul(ldz(row + c), sv[c]));
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
      double sr = 0.0, si = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const z v = sv[i], pr = ldz(&p[j + 1 + i]);
        sw[i] = pr;
        sr += v.x * pr.x + v.y * pr.y;
        si += v.x * pr.y - v.y * pr.x;
      }
      const double vpr = block_sum(sr, sh);
      const double vpi = block_sum(si, sh);
      const z coef = {0.5 * (t.x * vpr + t.y * vpi), 0.5 * (t.x * vpi - t.y * vpr)};
      for (int i = threadIdx.x; i < m; i += blockDim.x) sw[i] = csub(sw[i], cmul(coef, sv[i]));
      __syncthreads();
      // all columns but the first of the trailing block (CTA 0 owns that one)
      if (m > 1) {
        const size_t total = (size_t)m * (m - 1);
        for (size_t q = gtid; q < total; q += nthr) {
          const int r = (int)(q / (m - 1)), c = 1 + (int)(q % (m - 1));
          const z dlt = cadd(cmul(sv[r], zconj(sw[c])), cmul(sw[r], zconj(sv[c])));
          z* a = &A[(size_t)(j + 1 + r) * lda + (j + 1 + c)];
          *a = csub(ldz(a), dlt);
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

// ---- tridiagonal eigenvalues: Sturm bisection, one thread per eigenvalue --------
__device__ int sturm_count(const double* d, const double* e, int n, double x, double tiny) {
  int cnt = 0;
  double q = d[0] - x;
  if (q == 0.0) q = -tiny;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// One warp per eigenvalue: multisection.  Each round the 32 lanes evaluate the
// Sturm count at 32 interior points of the current bracket and the bracket
// shrinks to the sub-interval holding the (k+1)-th eigenvalue (a factor 33 per
// round instead of 2 for bisection).
__global__ void __launch_bounds__(64) k_bisect(const double* d, const double* e, int n, int nev,
                                                double* w) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nev) return;
  double lo = 0.0, hi = 0.0;
  {
    double l = 1e300, h = -1e300;
    for (int i = lane; i < n; i += 32) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
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
  const double nrm = fmax(fabs(lo), fabs(hi));
  const double tiny = 1e-300 + 1e-30 * nrm;
  lo -= 1e-14 * nrm + 1e-300;
  hi += 1e-14 * nrm + 1e-300;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi))) break;
    const double step = (hi - lo) / 33.0;
    const double x = lo + step * (lane + 1);
    const int c = (x > lo && x < hi) ? sturm_count(d, e, n, x, tiny) : (x <= lo ? 0 : n);
    // lanes whose point has more than k eigenvalues below it bound from above
    const unsigned above = __ballot_sync(0xffffffffu, c > k);
    const int first = above ? __ffs(above) - 1 : 32;    // first lane with count > k
    const double nlo = first == 0 ? lo : lo + step * first;
    const double nhi = first == 32 ? hi : lo + step * (first + 1);
    if (!(nhi < hi || nlo > lo)) break;                 // no progress at this resolution
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[k] = 0.5 * (lo + hi);
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

// One CTA per cluster of consecutive eigenvalues closer than ctol; the CTA whose
// index starts a cluster handles all of it, the others return.  Vectors are rows
// Y[k][0..n).  Shared memory: 6 arrays of n doubles (+ ints) for the factorisation.
__global__ void __launch_bounds__(256) k_inviter(const double* d, const double* e, int n, int nev,
                                                 const double* w, double ctol_rel, double* Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* u0 = reinterpret_cast<double*>(smem_raw);
  double* u1 = u0 + n;
  double* u2 = u1 + n;
  double* ml = u2 + n;
  double* y = ml + n;
  int* sw = reinterpret_cast<int*>(y + n);
  __shared__ double sh[33];
  const int k0 = blockIdx.x;
  if (k0 >= nev) return;
  double nrm = 0.0;
  for (int i = 0; i < n; ++i)
    nrm = fmax(nrm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0));
  const double ctol = ctol_rel * fmax(nrm, 1e-300);
  if (k0 > 0 && w[k0] - w[k0 - 1] <= ctol) return;   // not a cluster start
  int k1 = k0 + 1;
  while (k1 < nev && w[k1] - w[k1 - 1] <= ctol) ++k1;
  const double tiny = fmax(2.2e-16 * nrm, 1e-300);
  for (int k = k0; k < k1; ++k) {
    const double lam = w[k];
    // LU with partial pivoting of T - lam I (thread 0)
    if (threadIdx.x == 0) {
      double c0 = d[0] - lam, c1 = n > 1 ? e[0] : 0.0, c2 = 0.0;
      for (int i = 0; i < n - 1; ++i) {
        double n0 = e[i], n1 = d[i + 1] - lam, n2 = (i + 2 < n) ? e[i + 1] : 0.0;
        int s = 0;
        if (fabs(n0) > fabs(c0)) {
          double t;
          t = c0; c0 = n0; n0 = t;
          t = c1; c1 = n1; n1 = t;
          t = c2; c2 = n2; n2 = t;
          s = 1;
        }
        if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
        const double mlt = n0 / c0;
        u0[i] = c0; u1[i] = c1; u2[i] = c2; ml[i] = mlt; sw[i] = s;
        c0 = n1 - mlt * c1;
        c1 = n2 - mlt * c2;
        c2 = 0.0;
      }
      if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
      u0[n - 1] = c0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = start_component(k, i);
    __syncthreads();
    for (int it = 0; it < 4; ++it) {
      if (threadIdx.x == 0) {
        for (int i = 0; i < n - 1; ++i) {
          if (sw[i]) { const double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
          y[i + 1] -= ml[i] * y[i];
        }
        for (int i = n - 1; i >= 0; --i) {
          double s = y[i];
          if (i + 1 < n) s -= u1[i] * y[i + 1];
          if (i + 2 < n) s -= u2[i] * y[i + 2];
          y[i] = s / u0[i];
        }
      }
      __syncthreads();
      // scale down first (the solve grows the vector by up to 1/tiny)
      double mx = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(y[i]));
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
      __syncthreads();
      if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m2 = fmax(m2, sh[q]);
        sh[32] = m2 > 0.0 ? m2 : 1.0;
      }
      __syncthreads();
      const double inv_mx = 1.0 / sh[32];
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv_mx;
      __syncthreads();
      // orthogonalise against the finished vectors of this cluster (twice)
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = k0; q < k; ++q) {
          const double* yq = Y + (size_t)q * n;
          double s = 0.0;
          for (int i = threadIdx.x; i < n; i += blockDim.x) s += yq[i] * y[i];
          s = block_sum(s, sh);
          for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] -= s * yq[i];
          __syncthreads();
        }
      }
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
      s = block_sum(s, sh);
      const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv;
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Y[(size_t)k * n + i] = y[i];
    __syncthreads();
  }
}

// X[:, k] = H_0 H_1 ... H_{n-2} y_k, one CTA per eigenvector; X [n][ldx].  The
// reflectors are read from their rows in refl (contiguous, coalesced).
__global__ void __launch_bounds__(256) k_backtransform(const z* __restrict__ refl, int n,
                                                       const z* tau, const double* Y, z* X, int ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z* x = reinterpret_cast<z*>(smem_raw);
  __shared__ double sh[33];
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = {Y[(size_t)k * n + i], 0.0};
  __syncthreads();
  for (int j = n - 2; j >= 0; --j) {
    const z t = tau[j];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const z* v = refl + (size_t)j * n;
    double sr = 0.0, si = 0.0;
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) {
      const z vr = v[r], xr = x[r];
      sr += vr.x * xr.x + vr.y * xr.y;
      si += vr.x * xr.y - vr.y * xr.x;
    }
    const double a = block_sum(sr, sh);
    const double b = block_sum(si, sh);
    const z f = cmul(t, z{a, b});     // tau (v^+ x)
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) x[r] = csub(x[r], cmul(f, v[r]));
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)i * ldx + k] = x[i];
}

int heev_lowest(z* A, int n, int lda, int nev, double* w, z* X, int ldx, DenseWork& wk,
                cudaStream_t st, Prof* pf) {
  if (n <= 0 || nev <= 0) return QE_OK;
  if (nev > n || n > kMaxDense) {
    set_error("heev_lowest: n = %d, nev = %d (max n %d)", n, nev, kMaxDense);
    return QE_EINVAL;
  }
  if (cudaMemsetAsync(wk.bar.count, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
    set_error("heev_lowest: memset failed");
    return QE_ECUDA;
  }
  {
    GridBar bar = wk.bar;
    void* args[] = {&A, &n, &lda, &wk.tau, &wk.e, &wk.p, &wk.d, &wk.vbuf, &wk.refl, &bar};
    const size_t tsm = 2 * (size_t)n * sizeof(z);
    set_max_dynamic_smem(k_tridiag_coop);
    // all SMs once the trailing block is large: the FP64 work is spread
    const int blocks = coop_blocks((const void*)k_tridiag_coop, (size_t)n * n * 4, tsm);
    ProfScope ps(pf, "heev_tridiag", st);
    int rc0 = launch_coop((const void*)k_tridiag_coop, blocks, args, st, "k_tridiag_coop", tsm);
    if (rc0) return rc0;
  }
  int rc = QE_OK;
  {
    ProfScope ps(pf, "heev_bisect", st);
    // two warps per block: the Sturm counts are FP64-bound, so spread them over the SMs
    k_bisect<<<(nev * 32 + 63) / 64, 64, 0, st>>>(wk.d, wk.e, n, nev, w);
  }
  rc = check_launch("k_bisect");
  if (rc) return rc;
  const size_t ism = (size_t)n * (5 * sizeof(double) + sizeof(int));
  // same (largest) cap for every caller: the attribute is shared process-wide
  set_max_dynamic_smem(k_inviter);
  set_max_dynamic_smem(k_backtransform);
  // eigenvalues within 1e-10 of each other (relative to the spread of T) share a cluster
  {
    ProfScope ps(pf, "heev_inviter", st);
    k_inviter<<<nev, 256, ism, st>>>(wk.d, wk.e, n, nev, w, wk.ctol_rel, wk.y);
  }
  rc = check_launch("k_inviter");
  if (rc) return rc;
  const size_t bsm = (size_t)n * sizeof(z);
  {
    ProfScope ps(pf, "heev_backtransform", st);
    k_backtransform<<<nev, 256, bsm, st>>>(wk.refl, n, wk.tau, wk.y, X, ldx);
  }
  return check_launch("k_backtransform");
}

}  // namespace qe
