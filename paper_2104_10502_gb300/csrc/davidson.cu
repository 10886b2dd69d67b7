// Block Davidson on the device (Sec. 3.3 of the paper: iterative solution of
// the Kohn-Sham Hamiltonian with the Davidson method; Sec. 3.2.1: KS_Solvers,
// which call the Hamiltonian builder as an external routine, and LAXlib's dense
// generalized eigensolver).
//
// The host drives the iteration; every step runs in device kernels:
//   H products            hpsi_core (FFT local + kinetic, projector GEMMs)
//   reduced matrices      gemm_inner, updated column block by column block
//   Rayleigh-Ritz (FP64)  Cholesky of S_r, L^-1 H_r L^-+, tridiagonal eigensolver,
//                         back substitution (dense.cu)
//   Ritz vectors          gemm_outer (Psi = V X, H Psi = (HV) X)
//   residuals (FP64)      k_resid: r_n = H psi_n - e_n psi_n and ||r_n||
//   corrections           k_precond: r_n / sqrt((h_G - e_n)^2 + pmin^2), normalised
//   orthonormalisation    two passes of projection against V, each followed by
//                         a Cholesky orthonormalisation of the block that drops
//                         corrections left without a new direction
// Per iteration the host reads nb eigenvalues, nb residual norms, the Cholesky
// status word and the kept-correction flags (a few KB).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <string>
#include <thread>

#include "ctx.h"
#include "dense.h"
#include "dvtask.h"
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

#define DV_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define DV_CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error("%s: %s", #x, cudaGetErrorString(e_)); return QE_ECUDA; } } while (0)

__device__ double dv_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// r_b = hpsi_b - e_b psi_b ; rn[b] = ||r_b||_2 (FP64, fixed reduction order)
__global__ void __launch_bounds__(256) k_resid(const z* psi, const z* hpsi, const double* e, int npw,
                                               z* r, double* rn) {
  __shared__ double sh[33];
  const int b = blockIdx.x;
  const double eb = e[b];
  const z* p = psi + (size_t)b * npw;
  const z* hp = hpsi + (size_t)b * npw;
  z* rr = r + (size_t)b * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const z a = hp[g], c = p[g];
    const z v = {a.x - eb * c.x, a.y - eb * c.y};
    rr[g] = v;
    s += v.x * v.x + v.y * v.y;
  }
  s = dv_block_sum(s, sh);
  if (threadIdx.x == 0) rn[b] = sqrt(s);
}

// d_j = r_{idx[j]} / sqrt((h_G - e)^2 + pmin^2), normalised to unit norm
__global__ void __launch_bounds__(256) k_precond(const z* r, const int* idx, const double* e,
                                                 const double* hd, int npw, double pmin2, z* d) {
  __shared__ double sh[33];
  const int j = blockIdx.x;
  const int b = idx[j];
  const double eb = e[b];
  const z* rr = r + (size_t)b * npw;
  z* dd = d + (size_t)j * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double x = hd[g] - eb;
    const double inv = rsqrt(x * x + pmin2);
    const z v = {rr[g].x * inv, rr[g].y * inv};
    dd[g] = v;
    s += v.x * v.x + v.y * v.y;
  }
  s = dv_block_sum(s, sh);
  const double sc = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    dd[g].x *= sc;
    dd[g].y *= sc;
  }
}

// h_G = |k+G|^2 + vmean + sum_i D_ii |B_i(G)|^2
__global__ void k_hdiag(const double* kin, const double* vmean, const z* beta, const double* D,
                        int np, int npw, double* hd) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw) return;
  double h = kin[g] + *vmean;
  for (int i = 0; i < np; ++i) {
    const double dii = D[(size_t)i * np + i];
    if (dii != 0.0) {
      const z b = beta[(size_t)i * npw + g];
      h += dii * (b.x * b.x + b.y * b.y);
    }
  }
  hd[g] = h;
}

__global__ void __launch_bounds__(1024) k_mean(const double* v, size_t n, double* out) {
  __shared__ double sh[33];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = dv_block_sum(s, sh);
  if (threadIdx.x == 0) *out = s / (double)n;
}

// H[n0 + j][i] = conj(H[i][n0 + j]) for i < n0 <= n0 + j < n1
__global__ void k_mirror(z* H, int ld, int n0, int n1) {
  const int m = n1 - n0;
  const size_t total = (size_t)m * n0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = n0 + (int)(t / n0), i = (int)(t % n0);
    const z a = H[(size_t)i * ld + j];
    H[(size_t)j * ld + i] = {a.x, -a.y};
  }
}

// dst[a][b] = src[keep[a]][keep[b]]
__global__ void k_gather_sub(const z* src, int lds, const int* keep, int nk, z* dst, int ldd) {
  const size_t total = (size_t)nk * nk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / nk), b = (int)(t % nk);
    dst[(size_t)a * ldd + b] = src[(size_t)keep[a] * lds + keep[b]];
  }
}

// identity nk x nk (ld ldd)
__global__ void k_identity(z* dst, int nk, int ldd) {
  const size_t total = (size_t)nk * nk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / nk), b = (int)(t % nk);
    dst[(size_t)a * ldd + b] = {a == b ? 1.0 : 0.0, 0.0};
  }
}

// full[keep[a]][c] = M[a][c]; full is [nrow][nk], zeroed beforehand
__global__ void k_place_rows(const z* M, int ldm, const int* keep, int nk, z* full) {
  const size_t total = (size_t)nk * nk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / nk), c = (int)(t % nk);
    full[(size_t)keep[a] * nk + c] = M[(size_t)a * ldm + c];
  }
}

static int grid_for(size_t total) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 152 * 8));
}

// ---- k = 0: bands real in r ---------------------------------------------------
// Row r of X becomes the larger of its two real-in-r parts,
//   A = (X + conj X(-G)) / 2   and   B = (X - conj X(-G)) / 2i   (X = A + i B),
// so that no start vector can vanish.  One CTA per row; every mirror pair
// (g, -g) is read and written by one thread.
__global__ void __launch_bounds__(256) k_gamma_start(z* X, int npw, const int* __restrict__ mg) {
  __shared__ double sh[33];
  z* x = X + (size_t)blockIdx.x * npw;
  double na = 0.0, nbv = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const z a = x[g], b = x[mg[g]];
    const double ax = 0.5 * (a.x + b.x), ay = 0.5 * (a.y - b.y);   // A_g
    const double bx = 0.5 * (a.y + b.y), by = 0.5 * (b.x - a.x);   // B_g
    na += ax * ax + ay * ay;
    nbv += bx * bx + by * by;
  }
  na = dv_block_sum(na, sh);
  nbv = dv_block_sum(nbv, sh);
  const bool use_a = na >= nbv;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const int m = mg[g];
    if (m < g) continue;
    const z a = x[g], b = x[m];
    z c = use_a ? z{0.5 * (a.x + b.x), 0.5 * (a.y - b.y)} : z{0.5 * (a.y + b.y), 0.5 * (b.x - a.x)};
    if (m == g) c.y = 0.0;
    x[g] = c;
    x[m] = {c.x, -c.y};
  }
}

// X <- (X + conj X(-G)) / 2 for rows [0, rows): the real-in-r part.
__global__ void k_gamma_sym(z* X, int rows, int npw, const int* __restrict__ mg) {
  const size_t total = (size_t)rows * npw;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / npw), g = (int)(t % npw);
    const int m = mg[g];
    if (m < g) continue;
    z* x = X + (size_t)r * npw;
    const z a = x[g], b = x[m];
    z c = {0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
    if (m == g) c.y = 0.0;
    x[g] = c;
    x[m] = {c.x, -c.y};
  }
}

// Largest |beta_i(-G) - conj beta_i(G)| and largest |beta_i(G)|, as the bit
// patterns of non-negative doubles (ordered like the values) in out[0], out[1].
__global__ void k_beta_mirror(const z* __restrict__ beta, int np, int npw, const int* __restrict__ mg,
                              unsigned long long* out) {
  double dmax = 0.0, bmax = 0.0;
  const size_t total = (size_t)np * npw;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / npw;
    const int g = (int)(t % npw);
    const z a = beta[t], b = beta[i * npw + mg[g]];
    dmax = fmax(dmax, fmax(fabs(b.x - a.x), fabs(b.y + a.y)));
    bmax = fmax(bmax, fmax(fabs(a.x), fabs(a.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(bmax));
  }
}

struct DvState {
  int npw = 0, nb = 0, max_dim = 0, np = 0;
  z *V = nullptr, *HV = nullptr, *Psi = nullptr, *HPsi = nullptr, *R = nullptr, *D = nullptr,
    *D2 = nullptr;
  z *Hr = nullptr, *Sr = nullptr, *Lw = nullptr, *Zw = nullptr, *Aw = nullptr, *X = nullptr,
    *C = nullptr, *G = nullptr, *Mf = nullptr, *Mk = nullptr, *Lk = nullptr;
  double *e = nullptr, *rn = nullptr, *hd = nullptr, *vmean = nullptr;
  int* idx = nullptr;
  DenseWork dw;
  void* part = nullptr;
  size_t part_bytes = 0;
  // FP64 subspace products on the tensor cores: operand slices + partials
  void* oz = nullptr;
  size_t oz_bytes = 0;
  // the row slices of V[0:vrows), kept across products (oz_cache_rows): the
  // basis only grows by appended rows between the points that rewrite it
  // (restart, collapse, refinement), which set vrows = 0
  void* vcache = nullptr;
  int vrows = 0;
  // the mixed path's subspace products on the tensor cores (TF32 x3)
  void* tc = nullptr;
  size_t tc_bytes = 0;
  // k = 0 with real projectors: every basis vector real in r (psi(-G) =
  // conj psi(G), mg the sphere index of -G); two bands share each FFT and the
  // reduced matrices are real
  bool gamma = false;
  const int* mg = nullptr;
};

// Scratch of the mixed path's tensor-core subspace products (largest inner and
// outer product of a solve).
static size_t dv_tc_bytes(size_t npw, size_t nb, size_t md, bool fp64) {
  if (fp64) return 0;
  return std::max(tc_inner_bytes((int)md, (int)nb, (int)npw), tc_outer_bytes((int)npw, (int)nb, (int)md)) +
         256;
}

// Products below ~4 M complex multiply-adds stay on the SIMT kernels (the
// tensor-core path's packing launches cost more there).
static bool tc_worth(long long M, long long N, long long K) { return M > 0 && N > 0 && M * N * K >= (1ll << 22); }

// Scratch of the FP64 tensor-core subspace products: the largest inner product
// (basis x new block over the plane waves) and outer product (rotation of the
// basis) of a solve.
// The mixed path needs it for its final FP64 Rayleigh-Ritz and FP64 iterations.
static size_t dv_oz_bytes(size_t npw, size_t nb, size_t md, bool fp64) {
  (void)fp64;   // the mixed path may end with FP64 iterations over the whole basis
  if (!fp64_gemm_on_tensor_cores()) return 0;
  const size_t n = md;
  return std::max(oz_inner_scratch((int)n, (int)nb, (int)npw),
                  oz_outer_scratch((int)npw, (int)nb, (int)n)) + 256;
}

// The kept row slices of the basis, where its inner products run on the tensor
// cores.
static size_t dv_vcache_bytes(size_t npw, size_t nb, size_t md) {
  if (!fp64_gemm_on_tensor_cores() || !oz_worth((long long)md, (long long)nb, (long long)npw)) return 0;
  return oz_cache_bytes((int)md, (int)npw) + 256;
}

static size_t dv_bytes(size_t npw, size_t nb, size_t md) {
  const size_t zb = sizeof(z);
  const size_t big = (2 * md + 5 * nb) * npw * zb;
  const size_t smallz = (6 * md * md + 2 * md * nb + 4 * nb * nb) * zb;
  const size_t dbl = (2 * nb + npw + 1 + 3 * md + nb * md) * sizeof(double);
  const size_t dwz = (3 * md + 8 * md + 64) * zb;   // tau, p, vbuf; compact-WY T blocks
  const size_t ints = (nb + 16) * sizeof(int);
  return big + smallz + dbl + dwz + ints + 48 * 256;
}

static size_t dv_red_bytes(size_t md) {
  const size_t tiles = (size_t)((md + 31) / 32) * ((md + 31) / 32);
  return (2 * 152 * 4 + tiles + 1) * 32 * 32 * sizeof(z);
}

// Upper bound of the device memory one qe_davidson call holds (FP64 path; the
// mixed path needs less): Davidson state, H|psi> workspaces, operator copies of
// host inputs and the plan.
size_t davidson_footprint(int npw, int nb, int max_dim, int nproj, const int grid[3], int nst) {
  const size_t md = std::max(max_dim, 2 * nb);
  const size_t ngrid = (size_t)grid[0] * grid[1] * grid[2];
  const size_t per_band = (size_t)grid[2] * nst * sizeof(z);
  const size_t nbc = std::max<size_t>(1, std::min<size_t>(nb, ((size_t)64 << 20) / std::max<size_t>(per_band, 1)));
  size_t b = dv_bytes(npw, nb, md) + dv_red_bytes(md) + dv_oz_bytes(npw, nb, md, true) +
             dv_vcache_bytes(npw, nb, md);
  b += ngrid * sizeof(double) * 2;                                  // V copy + permuted V
  b += nbc * per_band;                                              // stick buffer
  b += gemm_inner_scratch(nproj, nb, npw, sizeof(double));          // split-K partials
  if (nproj > 0 && fp64_gemm_on_tensor_cores())                     // beta slices + work
    b += nonlocal_oz_bytes(nproj, nb, npw) + nonlocal_oz_beta_bytes(nproj, npw);
  b += 2 * (size_t)nproj * nb * sizeof(z);                          // projections
  b += (size_t)nproj * npw * sizeof(z) + (size_t)nproj * nproj * sizeof(double);   // beta, D
  b += (size_t)npw * 24 + 16 * (size_t)npw + 64 * (size_t)(grid[0] + grid[1] + grid[2]);   // plan
  return b + ((size_t)1 << 20);
}

static int dv_alloc(DevBuf& basis, DevBuf& red, DvState& S, bool fp64) {
  const size_t npw = S.npw, nb = S.nb, md = S.max_dim;
  const size_t zb = sizeof(z);
  // big: V, HV [md][npw]; Psi, HPsi, R, D, D2 [nb][npw]
  const size_t big = (2 * md + 5 * nb) * npw * zb;
  // small complex: Hr, Sr, Lw, Zw, Aw, reflectors [md][md]; X [md][nb]; C [md][nb]; G, Mf, Mk, Lk [nb][nb]
  const size_t smallz = (6 * md * md + 2 * md * nb + 4 * nb * nb) * zb;
  // doubles: e, rn [nb]; hd [npw]; vmean; dense work: d, e, piv [md], y [nb][md]
  const size_t dbl = (2 * nb + npw + 1 + 3 * md + nb * md) * sizeof(double);
  // dense work complex: tau, p, vbuf [md]
  const size_t dwz = (3 * md + 8 * md + 64) * zb;   // tau, p, vbuf; compact-WY T blocks
  const size_t ints = (nb + 16) * sizeof(int);
  const size_t total = big + smallz + dbl + dwz + ints + 48 * 256;   // + alignment of 31 pieces
  if (total != dv_bytes(npw, nb, md)) {
    set_error("davidson: workspace size mismatch");
    return QE_EINVAL;
  }
  DV_TRY(basis.ensure(total));
  char* p = (char*)basis.p;
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  S.V = (z*)take(md * npw * zb);
  S.HV = (z*)take(md * npw * zb);
  S.Psi = (z*)take(nb * npw * zb);
  S.HPsi = (z*)take(nb * npw * zb);
  S.R = (z*)take(nb * npw * zb);
  S.D = (z*)take(nb * npw * zb);
  S.D2 = (z*)take(nb * npw * zb);
  S.Hr = (z*)take(md * md * zb);
  S.Sr = (z*)take(md * md * zb);
  S.Lw = (z*)take(md * md * zb);
  S.Zw = (z*)take(md * md * zb);
  S.Aw = (z*)take(md * md * zb);
  S.X = (z*)take(md * nb * zb);
  S.C = (z*)take(md * nb * zb);
  S.G = (z*)take(nb * nb * zb);
  S.Mf = (z*)take(nb * nb * zb);
  S.Mk = (z*)take(nb * nb * zb);
  S.Lk = (z*)take(nb * nb * zb);
  S.e = (double*)take(nb * sizeof(double));
  S.rn = (double*)take(nb * sizeof(double));
  S.hd = (double*)take(npw * sizeof(double));
  S.vmean = (double*)take(sizeof(double));
  S.dw.d = (double*)take(md * sizeof(double));
  S.dw.e = (double*)take(md * sizeof(double));
  S.dw.piv = (double*)take(md * sizeof(double));
  S.dw.y = (double*)take(nb * md * sizeof(double));
  S.dw.tau = (z*)take(md * zb);
  S.dw.p = (z*)take(md * zb);
  S.dw.vbuf = (z*)take(md * zb);
  S.dw.wyt = (z*)take((8 * md + 64) * zb);
  S.dw.refl = (z*)take(md * md * zb);
  S.idx = (int*)take(nb * sizeof(int));
  S.dw.status = (int*)take(16 * sizeof(int));
  S.dw.bar.count = reinterpret_cast<unsigned int*>(S.dw.status + 4);
  S.dw.bar.gen = S.dw.bar.count + 1;
  S.dw.bar.err = S.dw.status + 8;
  if ((size_t)(p - (char*)basis.p) > basis.bytes) {
    set_error("davidson: workspace layout overflow");
    return QE_EINVAL;
  }
  // split-K partials: at most (splits for ~4 CTAs/SM + tiles) 32x32 tiles of FP64 complex
  const size_t sb = dv_red_bytes(md);
  const size_t ob = dv_oz_bytes(npw, nb, md, fp64);
  const size_t tb = dv_tc_bytes(npw, nb, md, fp64);
  const size_t vb = dv_vcache_bytes(npw, nb, md);
  DV_TRY(red.ensure(sb + ob + tb + vb));
  S.part = red.p;
  S.part_bytes = sb;
  S.oz = ob ? static_cast<char*>(red.p) + sb : nullptr;
  S.oz_bytes = ob;
  S.tc = tb ? static_cast<char*>(red.p) + sb + ob : nullptr;
  S.tc_bytes = tb;
  S.vcache = vb ? static_cast<char*>(red.p) + sb + ob + tb : nullptr;
  S.vrows = 0;
  return QE_OK;
}

// The status word of the tensor-core products of a solve (a bounded wait that
// ran out); read with the other status words at every convergence test.
static int* dv_tc_status(const DvState& S) { return S.dw.status + 12; }

// C = A^+ B over the plane waves; real for vectors real in r (k = 0 mode), so
// that the combinations built from C keep them real in r exactly (the SIMT
// path drops Im C in its split reduction, the tensor-core paths compute only
// Re C).
template <typename T>
static int gram(DvState& S, const z* A, int m, const z* B, int n, z* C, int ldc,
                cudaStream_t st, Prof* pf) {
  if (sizeof(T) == sizeof(double) && A == S.V && S.vcache && S.oz && oz_worth(m, n, S.npw) &&
      oz_inner_cached_scratch(m, n, S.npw) <= S.oz_bytes) {
    // the basis: slice only the rows added since the last product with it
    if (S.vrows < m) {
      DV_TRY(oz_cache_rows((const double*)S.V, S.npw, S.vrows, m, S.npw, S.max_dim, S.vcache, st, pf));
      S.vrows = m;
    }
    return oz_inner_cached(S.vcache, S.max_dim, m, (const double*)B, S.npw, n, S.npw, (double*)C, ldc,
                           S.oz, S.oz_bytes, dv_tc_status(S), st, pf, S.gamma);
  }
  if (sizeof(T) == sizeof(float) && S.tc && tc_worth(m, n, S.npw))
    return tc_inner((const double*)A, (const double*)B, m, n, S.npw, (double*)C, ldc, S.tc,
                    S.tc_bytes, dv_tc_status(S), st, pf, S.gamma);
  if (sizeof(T) == sizeof(double) && S.oz && oz_worth(m, n, S.npw))
    return oz_inner((const double*)A, S.npw, (const double*)B, S.npw, m, n, S.npw, (double*)C, ldc,
                    S.oz, S.oz_bytes, dv_tc_status(S), st, pf, S.gamma);
  return gemm_inner<T>((const double*)A, S.npw, (const double*)B, S.npw, m, n, S.npw, (double*)C,
                       ldc, S.part, S.part_bytes, st, pf, S.gamma);
}

// C[n][m] (+)= (-) sum_k A[k][m] B[k][n]: rotations and projections out of the basis
template <typename T>
static int outer_any(const DvState& S, const z* A, int lda, const z* B, int ldb, int M, int N,
                     int K, z* C, int ldc, int alpha_neg, int beta, cudaStream_t st, Prof* pf) {
  if (sizeof(T) == sizeof(float) && S.tc && tc_worth(M, N, K) && lda == M && ldb == N) {
    // k = 0 mode: the right-hand matrices (Ritz vectors, Gram blocks) are real
    if (S.gamma && tc_outer_real_bytes(M, N, K) <= S.tc_bytes)
      return tc_outer_real((const double*)A, (const double*)B, M, N, K, (double*)C, ldc, alpha_neg,
                           beta, S.tc, S.tc_bytes, dv_tc_status(S), st, pf);
    return tc_outer((const double*)A, (const double*)B, M, N, K, (double*)C, ldc, alpha_neg, beta,
                    S.tc, S.tc_bytes, dv_tc_status(S), st, pf);
  }
  if (sizeof(T) == sizeof(double) && S.oz && oz_worth(M, N, K)) {
    // k = 0 mode: the right-hand matrices (Ritz vectors, Gram blocks) are real
    if (S.gamma && oz_outer_real_scratch(M, N, K) <= S.oz_bytes)
      return oz_outer_real((const double*)A, lda, (const double*)B, ldb, M, N, K, (double*)C, ldc,
                           alpha_neg, beta, S.oz, S.oz_bytes, dv_tc_status(S), st, pf);
    return oz_outer((const double*)A, lda, (const double*)B, ldb, M, N, K, (double*)C, ldc,
                    alpha_neg, beta, S.oz, S.oz_bytes, dv_tc_status(S), st, pf);
  }
  return gemm_outer_ab<T>((const double*)A, lda, (const double*)B, ldb, M, N, K, (double*)C, ldc,
                          alpha_neg, beta, st, pf);
}

// outer_any; in the k = 0 mode the rows produced (plane-wave vectors) are made
// real in r again: the combinations are real, but the SIMT kernels' three-
// multiplication complex product does not round conjugate pairs alike.
template <typename T>
static int outer(const DvState& S, const z* A, int lda, const z* B, int ldb, int M, int N, int K,
                 z* C, int ldc, int alpha_neg, int beta, cudaStream_t st, Prof* pf) {
  DV_TRY(outer_any<T>(S, A, lda, B, ldb, M, N, K, C, ldc, alpha_neg, beta, st, pf));
  if (!S.gamma || N <= 0 || M != S.npw || ldc != S.npw) return QE_OK;
  k_gamma_sym<<<grid_for((size_t)N * M), 256, 0, st>>>(C, N, M, S.mg);
  return check_launch("k_gamma_sym");
}

// Reduced matrices: columns [n0, n1) for rows [0, n1), then the mirrored rows.
// The overlap S_r only when the Rayleigh-Ritz that follows is a generalised one.
template <typename T>
static int update_reduced(DvState& S, int n0, int n1, bool with_s, cudaStream_t st, Prof* pf) {
  const int md = S.max_dim;
  DV_TRY(gram<T>(S, S.V, n1, S.HV + (size_t)n0 * S.npw, n1 - n0, S.Hr + n0, md, st, pf));
  if (with_s) DV_TRY(gram<T>(S, S.V, n1, S.V + (size_t)n0 * S.npw, n1 - n0, S.Sr + n0, md, st, pf));
  if (n0 > 0) {
    const size_t t = (size_t)(n1 - n0) * n0;
    k_mirror<<<grid_for(t), 256, 0, st>>>(S.Hr, md, n0, n1);
    if (with_s) k_mirror<<<grid_for(t), 256, 0, st>>>(S.Sr, md, n0, n1);
  }
  return check_launch("k_mirror");
}

// ---- Rayleigh-Ritz by Loewdin orthonormalisation ---------------------------------
// After the first iteration the basis is orthonormal up to the previous
// reduced problem's rounding: S_r = I + E with E tiny, and
//   M = S_r^(-1/2) = I - E/2 + 3/8 E^2 + O(E^3)
// makes A = M H_r M the standard problem whose eigenvectors Y give X = M Y
// (X^+ S_r X = I to O(E^3)).  Four n x n (x nb) matrix products on the tensor
// cores replace the Cholesky factorisation and the three triangular solves,
// which take one grid-wide step per column.
__global__ void k_lowdin_e(const z* __restrict__ Sr, int ld, int n, z* __restrict__ E) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    z v = Sr[(size_t)i * ld + j];
    if (i == j) v.x -= 1.0;
    E[t] = v;
  }
}

// M = I - E/2 + 3/8 conj(F), F = conj(E E) (the inner product of E with itself)
__global__ void k_lowdin_m(const z* __restrict__ E, const z* __restrict__ F, int n, z* __restrict__ M) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const z e = E[t], f = F[t];
    z m = {-0.5 * e.x + 0.375 * f.x, -0.5 * e.y - 0.375 * f.y};
    if (i == j) m.x += 1.0;
    M[t] = m;
  }
}

__global__ void k_compact(const z* __restrict__ src, int lds, int n, z* __restrict__ dst) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = src[(t / n) * lds + t % n];
}

__global__ void k_conj(const z* __restrict__ src, z* __restrict__ dst, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x) {
    const z v = src[t];
    dst[t] = {v.x, -v.y};
  }
}

// C[m][n] = sum_k conj(A[m][k]) B[n][k] for compact operands (rows of length K),
// on the tensor cores when the product is large enough and the scratch holds it.
template <typename T>
static int dense_inner(const DvState& S, const z* A, int M, const z* B, int N, int K, z* C, int ldc,
                       cudaStream_t st, Prof* pf) {
  if (sizeof(T) == sizeof(float) && S.tc && tc_worth(M, N, K) && tc_inner_bytes(M, N, K) <= S.tc_bytes)
    return tc_inner((const double*)A, (const double*)B, M, N, K, (double*)C, ldc, S.tc, S.tc_bytes,
                    dv_tc_status(S), st, pf, S.gamma);
  if (sizeof(T) == sizeof(double) && S.oz && oz_worth(M, N, K) && oz_inner_scratch(M, N, K) <= S.oz_bytes)
    return oz_inner((const double*)A, K, (const double*)B, K, M, N, K, (double*)C, ldc, S.oz,
                    S.oz_bytes, dv_tc_status(S), st, pf);
  return gemm_inner<T>((const double*)A, K, (const double*)B, K, M, N, K, (double*)C, ldc, S.part,
                       S.part_bytes, st, pf);
}

template <typename T>
static int rayleigh_ritz_lowdin(DvState& S, int n, cudaStream_t st, Prof* pf) {
  const int md = S.max_dim, nb = S.nb;
  const size_t nn = (size_t)n * n;
  ProfScope ps(pf, "rr_lowdin", st);
  k_lowdin_e<<<grid_for(nn), 256, 0, st>>>(S.Sr, md, n, S.Lw);                     // E
  DV_TRY(check_launch("k_lowdin_e"));
  DV_TRY(dense_inner<T>(S, S.Lw, n, S.Lw, n, n, S.Zw, n, st, pf));                 // conj(E E)
  k_lowdin_m<<<grid_for(nn), 256, 0, st>>>(S.Lw, S.Zw, n, S.Aw);                    // M
  k_compact<<<grid_for(nn), 256, 0, st>>>(S.Hr, md, n, S.Lw);                       // H
  DV_TRY(check_launch("k_lowdin_m"));
  DV_TRY(dense_inner<T>(S, S.Aw, n, S.Lw, n, n, S.Zw, n, st, pf));                 // conj(M H)
  k_conj<<<grid_for(nn), 256, 0, st>>>(S.Zw, S.Zw, nn);                             // M H
  DV_TRY(dense_inner<T>(S, S.Zw, n, S.Aw, n, n, S.Lw, n, st, pf));                 // conj(M H M)
  k_conj<<<grid_for(nn), 256, 0, st>>>(S.Lw, S.Lw, nn);
  DV_TRY(check_launch("k_conj"));
  DV_TRY(hermitize(S.Lw, n, n, st));
  pf->launches += 4;
  return QE_OK;
}

// X = M Y for the Loewdin Rayleigh-Ritz: Y [n][nb] in S.X, M in S.Aw.
template <typename T>
static int lowdin_back(DvState& S, int n, cudaStream_t st, Prof* pf) {
  const int nb = S.nb;
  k_conj<<<grid_for((size_t)n * n), 256, 0, st>>>(S.Aw, S.Zw, (size_t)n * n);        // conj(M)
  DV_TRY(check_launch("k_conj"));
  DV_TRY(transpose(S.X, nb, S.C, n, n, nb, st));                                    // Y^T
  return dense_inner<T>(S, S.Zw, n, S.C, nb, n, S.X, nb, st, pf);                  // M Y
}

// FP64 <-> FP32 copies of the reduced problem for the mixed path.
__global__ void k_z_to_c(const z* __restrict__ src, int lds, cx<float>* __restrict__ dst, int ldd,
                         int rows, int cols) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    const z v = src[(size_t)r * lds + c];
    dst[(size_t)r * ldd + c] = {(float)v.x, (float)v.y};
  }
}

__global__ void k_c_to_z(const cx<float>* __restrict__ src, int lds, z* __restrict__ dst, int ldd,
                         int rows, int cols, const float* __restrict__ ws, double* __restrict__ wd,
                         int nw) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    const cx<float> v = src[(size_t)r * lds + c];
    dst[(size_t)r * ldd + c] = {(double)v.x, (double)v.y};
    if (t < (size_t)nw) wd[t] = (double)ws[t];
  }
}

// Rayleigh-Ritz of the mixed path's iterations in FP32: its reduced matrices
// come from FP32 products (~1e-6 relative), so solving them in FP64 buys no
// accuracy, and GB300 runs FP32 ~60x faster.  The final FP64 Rayleigh-Ritz of
// the converged Ritz vectors (refine) restores FP64 eigenpairs.  The FP32
// matrices live in the FP64 work buffers (half their size).
static int rayleigh_ritz_f32(DvState& S, int n, cudaStream_t st, Prof* pf) {
  using zf = cx<float>;
  const int md = S.max_dim, nb = S.nb;
  zf* H32 = reinterpret_cast<zf*>(S.Zw);
  zf* L32 = reinterpret_cast<zf*>(S.Lw);
  zf* A32 = reinterpret_cast<zf*>(S.Aw);
  zf* X32 = reinterpret_cast<zf*>(S.C);
  float* e32 = reinterpret_cast<float*>(S.rn);
  DenseWorkT<float> w;
  w.tau = reinterpret_cast<zf*>(S.dw.tau);
  w.p = reinterpret_cast<zf*>(S.dw.p);
  w.vbuf = reinterpret_cast<zf*>(S.dw.vbuf);
  w.wyt = reinterpret_cast<zf*>(S.dw.wyt);
  w.refl = reinterpret_cast<zf*>(S.dw.refl);
  w.d = reinterpret_cast<float*>(S.dw.d);
  w.e = reinterpret_cast<float*>(S.dw.e);
  w.y = reinterpret_cast<float*>(S.dw.y);
  w.piv = reinterpret_cast<float*>(S.dw.piv);
  w.status = S.dw.status;
  w.bar = S.dw.bar;
  k_z_to_c<<<grid_for((size_t)n * n), 256, 0, st>>>(S.Hr, md, H32, n, n, n);
  k_z_to_c<<<grid_for((size_t)n * n), 256, 0, st>>>(S.Sr, md, L32, n, n, n);
  DV_TRY(check_launch("k_z_to_c"));
  if (f32::rr_small_fits(n)) {
    DV_TRY(f32::rr_small(H32, L32, n, n, nb, L32, e32, X32, nb, w, st, pf));
  } else {
    {
      ProfScope ps(pf, "rr_cholesky", st);
      DV_TRY(f32::cholesky(L32, n, n, 0.f, false, w.piv, w.status, w.bar, st, S.gamma));
    }
    {
      ProfScope ps(pf, "rr_reduce", st);
      DV_TRY(f32::transpose(L32, n, w.refl, n, n, n, st));
      DV_TRY(f32::trsm_lower_t(w.refl, n, n, H32, n, n, st));
      DV_TRY(f32::conj_transpose(H32, n, A32, n, n, n, st));
      DV_TRY(f32::trsm_lower_t(w.refl, n, n, A32, n, n, st));
      DV_TRY(f32::hermitize(A32, n, n, st));
      pf->launches += 4;
    }
    DV_TRY(f32::heev_lowest(A32, n, n, nb, e32, X32, nb, w, st, pf));
  }
  {
    ProfScope ps(pf, "rr_backsub", st);
    DV_TRY(f32::trsm_upper_h(L32, n, n, X32, nb, nb, st, S.gamma));
  }
  k_c_to_z<<<grid_for((size_t)n * nb), 256, 0, st>>>(X32, nb, S.X, nb, n, nb, e32, S.e, nb);
  return check_launch("k_c_to_z");
}

// Lowest nb eigenpairs of the Hermitian n x n matrix in S.Lw (compact; destroyed)
// into S.e, S.X (ld nb), in FP32 or FP64.
static int rr_standard_eig(DvState& S, int n, bool fp32, cudaStream_t st, Prof* pf) {
  const int nb = S.nb;
  if (!fp32) return heev_lowest(S.Lw, n, n, nb, S.e, S.X, nb, S.dw, st, pf, S.gamma);
  using zf = cx<float>;
  zf* A32 = reinterpret_cast<zf*>(S.Zw);
  zf* X32 = reinterpret_cast<zf*>(S.C);
  float* e32 = reinterpret_cast<float*>(S.rn);
  DenseWorkT<float> w;
  w.tau = reinterpret_cast<zf*>(S.dw.tau);
  w.p = reinterpret_cast<zf*>(S.dw.p);
  w.vbuf = reinterpret_cast<zf*>(S.dw.vbuf);
  w.wyt = reinterpret_cast<zf*>(S.dw.wyt);
  w.refl = reinterpret_cast<zf*>(S.dw.refl);
  w.d = reinterpret_cast<float*>(S.dw.d);
  w.e = reinterpret_cast<float*>(S.dw.e);
  w.y = reinterpret_cast<float*>(S.dw.y);
  w.piv = reinterpret_cast<float*>(S.dw.piv);
  w.status = S.dw.status;
  w.bar = S.dw.bar;
  k_z_to_c<<<grid_for((size_t)n * n), 256, 0, st>>>(S.Lw, n, A32, n, n, n);
  DV_TRY(check_launch("k_z_to_c"));
  DV_TRY(f32::heev_lowest(A32, n, n, nb, e32, X32, nb, w, st, pf));
  k_c_to_z<<<grid_for((size_t)n * nb), 256, 0, st>>>(X32, nb, S.X, nb, n, nb, e32, S.e, nb);
  return check_launch("k_c_to_z");
}

// Rayleigh-Ritz on span(V[0:n]): eigenvalues e[0:nb], X [n][nb] (ld nb).
// Generalised (S_r = L L^+ by Cholesky, then the standard problem of
// L^-1 H_r L^-+) in every iteration: the basis is orthonormal only up to the
// eigenvector accuracy of the previous reduced problem (inverse iteration
// re-orthogonalises only within clusters of eigenvalues closer than 1e-10 of
// the spread), and a standard Rayleigh-Ritz that assumed S_r = I stalled the
// C0 iteration.  `generalised = false` (S_r = I) is kept for callers that know
// their basis is orthonormal.
static int rayleigh_ritz(DvState& S, int n, bool generalised, cudaStream_t st, Prof* pf) {
  const int md = S.max_dim, nb = S.nb;
  const size_t zb = sizeof(z);
  if (!generalised) {
    DV_CU(cudaMemcpy2DAsync(S.Aw, n * zb, S.Hr, md * zb, n * zb, n, cudaMemcpyDeviceToDevice, st));
    DV_TRY(hermitize(S.Aw, n, n, st));
    return heev_lowest(S.Aw, n, n, nb, S.e, S.X, nb, S.dw, st, pf, S.gamma);
  }
  if (rr_small_fits(n)) {
    // one CTA in shared memory: Cholesky, reduction, tridiagonalisation
    DV_TRY(rr_small(S.Hr, S.Sr, md, n, nb, S.Lw, S.e, S.X, nb, S.dw, st, pf));
    ProfScope ps(pf, "rr_backsub", st);
    return trsm_upper_h(S.Lw, n, n, S.X, nb, nb, st, S.gamma);   // X = L^-+ Y
  }
  DV_CU(cudaMemcpy2DAsync(S.Lw, n * zb, S.Sr, md * zb, n * zb, n, cudaMemcpyDeviceToDevice, st));
  DV_CU(cudaMemcpy2DAsync(S.Zw, n * zb, S.Hr, md * zb, n * zb, n, cudaMemcpyDeviceToDevice, st));
  {
    ProfScope ps(pf, "rr_cholesky", st);
    DV_TRY(cholesky(S.Lw, n, n, 0.0, false, S.dw.piv, S.dw.status, S.dw.bar, st, S.gamma));
  }
  {
    // L^T in the reflector buffer (free until the eigensolver) for coalesced solves
    ProfScope ps(pf, "rr_reduce", st);
    DV_TRY(transpose(S.Lw, n, S.dw.refl, n, n, n, st));
    DV_TRY(trsm_lower_t(S.dw.refl, n, n, S.Zw, n, n, st));        // Z = L^-1 H
    DV_TRY(conj_transpose(S.Zw, n, S.Aw, n, n, n, st));           // Z^+ = H L^-+
    DV_TRY(trsm_lower_t(S.dw.refl, n, n, S.Aw, n, n, st));        // A = L^-1 H L^-+
    DV_TRY(hermitize(S.Aw, n, n, st));
    pf->launches += 4;
  }
  DV_TRY(heev_lowest(S.Aw, n, n, nb, S.e, S.X, nb, S.dw, st, pf, S.gamma));
  {
    ProfScope ps(pf, "rr_backsub", st);
    DV_TRY(trsm_upper_h(S.Lw, n, n, S.X, nb, nb, st, S.gamma));   // X = L^-+ Y
  }
  return QE_OK;
}

// Orthonormalise the nd rows of `in` against V[0:n] and among themselves; the
// kept vectors are written to `out` (rows).  Returns the number kept in *nk.
template <typename T>
static int orthonormalise(DvState& S, int n, z* in, int nd, z* out, int* nk_out, double drop,
                          cudaStream_t st, Prof* pf) {
  const int npw = S.npw;
  z* cur = in;
  int ncur = nd;
  for (int pass = 0; pass < 2 && ncur > 0; ++pass) {
    // cur -= V (V^+ cur)
    DV_TRY(gram<T>(S, S.V, n, cur, ncur, S.C, ncur, st, pf));
    DV_TRY(outer<T>(S, S.V, npw, S.C, ncur, npw, ncur, n, cur, npw, 1, 1, st, pf));
    // Cholesky of the block's Gram matrix with dropping
    DV_TRY(gram<T>(S, cur, ncur, cur, ncur, S.G, ncur, st, pf));
    DV_TRY(hermitize(S.G, ncur, ncur, st));
    DV_CU(cudaMemsetAsync(S.dw.status, 0, sizeof(int), st));
    DV_TRY(cholesky(S.G, ncur, ncur, drop * drop, true, S.dw.piv, S.dw.status, S.dw.bar, st,
                    S.gamma));
    std::vector<double> piv(ncur);
    DV_CU(cudaMemcpyAsync(piv.data(), S.dw.piv, ncur * sizeof(double), cudaMemcpyDeviceToHost, st));
    DV_CU(cudaStreamSynchronize(st));
    std::vector<int> keep;
    double pmin_kept = 1.0;
    for (int j = 0; j < ncur; ++j)
      if (piv[j] > 0.0) { keep.push_back(j); pmin_kept = std::min(pmin_kept, piv[j]); }
    const int nk = (int)keep.size();
    if (nk == 0) { *nk_out = 0; return QE_OK; }
    // "twice is enough": a second pass is needed only when this one removed most
    // of some vector (its remaining norm fell below 1/2 of the unit input)
    const bool last = pass == 1 || pmin_kept > 0.5;
    DV_CU(cudaMemcpyAsync(S.idx, keep.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st));
    // Mk = Lk^-+ with Lk the kept sub-factor; Mf = rows of Mk at the kept positions
    k_gather_sub<<<grid_for((size_t)nk * nk), 256, 0, st>>>(S.G, ncur, S.idx, nk, S.Lk, nk);
    k_identity<<<grid_for((size_t)nk * nk), 256, 0, st>>>(S.Mk, nk, nk);
    DV_TRY(check_launch("orthonormalise"));
    DV_TRY(trsm_upper_h(S.Lk, nk, nk, S.Mk, nk, nk, st, S.gamma));
    DV_CU(cudaMemsetAsync(S.Mf, 0, (size_t)ncur * nk * sizeof(z), st));
    k_place_rows<<<grid_for((size_t)nk * nk), 256, 0, st>>>(S.Mk, nk, S.idx, nk, S.Mf);
    DV_TRY(check_launch("k_place_rows"));
    z* dst = last ? out : S.D2;
    DV_TRY(outer<T>(S, cur, npw, S.Mf, nk, npw, nk, ncur, dst, npw, 0, 0, st, pf));
    cur = dst;
    ncur = nk;
    *nk_out = nk;
    if (last) break;
  }
  return QE_OK;
}

// Mixed-precision defect correction: one FP64 H|psi> of the Ritz vectors and a
// FP64 Rayleigh-Ritz on their span.  The FP32 accumulation of the reduced
// matrices over ~1e4-1e5 plane waves leaves ~1e-5 relative noise in H_r; this
// last step brings the eigenvalue error down to O(residual^2 / gap) and reports
// FP64 residual norms of the returned vectors.
// Split in two around the H product so that a batch can apply it to all its
// solves at once: refine_pre copies the Ritz vectors into V[0:nb], the caller
// applies FP64 H to them into HV[0:nb], refine_post does the Rayleigh-Ritz.
static int refine_pre(DvState& S, cudaStream_t st) {
  DV_CU(cudaMemcpyAsync(S.V, S.Psi, (size_t)S.nb * S.npw * sizeof(z), cudaMemcpyDeviceToDevice, st));
  S.vrows = 0;   // V rewritten: its kept slices are stale
  return QE_OK;
}

static int refine_post(DvState& S, cudaStream_t st, Prof* pf) {
  const int npw = S.npw, nb = S.nb;
  DV_TRY(update_reduced<double>(S, 0, nb, true, st, pf));
  DV_CU(cudaMemsetAsync(S.dw.status, 0, sizeof(int), st));
  DV_TRY(rayleigh_ritz(S, nb, true, st, pf));
  DV_TRY(outer<double>(S, S.V, npw, S.X, nb, npw, nb, nb, S.Psi, npw, 0, 0, st, pf));
  DV_TRY(outer<double>(S, S.HV, npw, S.X, nb, npw, nb, nb, S.HPsi, npw, 0, 0, st, pf));
  k_resid<<<nb, 256, 0, st>>>(S.Psi, S.HPsi, S.e, npw, S.R, S.rn);
  return check_launch("k_resid");
}

// One Davidson solve as a state machine, so that a batch can advance many
// solves in lockstep and apply H to all their new vectors in one batched call:
//   begin -> [H on V[0:nb]] -> after_first_h -> { step -> [H on the new rows] -> after_h }*
struct DvSolve {
  const DevPlan* P = nullptr;
  OpView op;
  int precision = QE_FP64;
  double tol = 0.0;
  int max_iter = 0;
  DvState S;
  int n = 0, it = 0, nk = 0;
  bool first = true, done = false, conv = false;
  std::vector<double> e, rn;
  // pending H product: rows [h_row, h_row + h_rows) of V into the same rows of HV
  int h_row = 0, h_rows = 0;
  // largest residual norm of the last convergence test; the Rayleigh-Ritz of
  // the last iteration ran in FP32
  double rmax = HUGE_VAL;
  bool rr32 = false;
  // mixed path: best largest residual so far and iterations without a 20 % gain
  double best_rmax = HUGE_VAL;
  int stall = 0;
  // mixed path: solve the reduced eigenproblems of its iterations in FP32
  // (QE_RR_FP32) instead of FP64
  bool mixed_rr32 = false;
};

// The FP64 path solves small reduced problems (n <= 64, the single-CTA path) in
// FP32 while every residual is above max(1e-3 Ry, 1000 tol): the eigenvectors
// then only steer the next corrections, and FP32 is ~60x faster on GB300.
// Convergence is accepted only after an FP64 Rayleigh-Ritz.  (On C2, n up to
// 1024, FP32 Ritz vectors doubled the iteration count, 19 -> 38.)
// The mixed path keeps its Rayleigh-Ritz (Cholesky of S_r, the reduced
// eigenproblem) in FP64 by default, on reduced matrices from its TF32x3
// products; with QE_RR_FP32 it solves them in FP32 like the small FP64 ones.
static bool rr_in_fp32(const DvSolve& v) {
  if (v.precision != QE_FP64) return v.mixed_rr32;
  return v.n <= kSmallDense && v.rmax > std::max(1e-3, 1e3 * v.tol);
}

static int dv_begin(DvSolve& v, cudaStream_t st) {
  DvState& S = v.S;
  const DevPlan& P = *v.P;
  const int npw = S.npw, nb = S.nb;
  const size_t ngrid = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  k_mean<<<1, 1024, 0, st>>>(v.op.vloc, ngrid, S.vmean);
  k_hdiag<<<(npw + 255) / 256, 256, 0, st>>>(P.kin, S.vmean, (const z*)v.op.beta, v.op.dmat,
                                              v.op.nproj, npw, S.hd);
  DV_TRY(check_launch("k_hdiag"));
  DV_CU(cudaMemsetAsync(S.dw.status, 0, 16 * sizeof(int), st));
  if (S.gamma) {
    k_gamma_start<<<nb, 256, 0, st>>>(S.V, npw, S.mg);
    S.vrows = 0;   // V rewritten: its kept slices are stale
    DV_TRY(check_launch("k_gamma_start"));
  }
  v.e.assign(nb, 0.0);
  v.rn.assign(nb, 0.0);
  v.n = nb;
  v.h_row = 0;
  v.h_rows = nb;
  return QE_OK;
}

template <typename T>
static int dv_after_first_h(DvSolve& v, cudaStream_t st, Prof* pf) {
  v.h_rows = 0;
  return update_reduced<T>(v.S, 0, v.n, true, st, pf);
}

// Rayleigh-Ritz and residuals, launched without waiting (a batch queues every
// solve's before the first wait) ...
template <typename T>
static int dv_step_launch(DvSolve& v, cudaStream_t st, Prof* pf) {
  DvState& S = v.S;
  const int npw = S.npw, nb = S.nb;
  const size_t zb = sizeof(z);
  DV_CU(cudaMemsetAsync(S.dw.status, 0, sizeof(int), st));   // keeps the barrier error word
  v.rr32 = rr_in_fp32(v);
  if (!v.first && v.n > kSmallDense) {
    // nearly orthonormal basis: Loewdin form on the tensor cores
    DV_TRY(rayleigh_ritz_lowdin<T>(S, v.n, st, pf));
    DV_TRY(rr_standard_eig(S, v.n, v.rr32, st, pf));
    DV_TRY(lowdin_back<T>(S, v.n, st, pf));
  } else if (v.rr32) {
    DV_TRY(rayleigh_ritz_f32(S, v.n, st, pf));
  } else {
    DV_TRY(rayleigh_ritz(S, v.n, true, st, pf));
  }
  DV_TRY(outer<T>(S, S.V, npw, S.X, nb, npw, nb, v.n, S.Psi, npw, 0, 0, st, pf));
  DV_TRY(outer<T>(S, S.HV, npw, S.X, nb, npw, nb, v.n, S.HPsi, npw, 0, 0, st, pf));
  if (v.first) {
    // the Ritz vectors of the start block become the (orthonormal) basis
    DV_CU(cudaMemcpyAsync(S.V, S.Psi, (size_t)nb * npw * zb, cudaMemcpyDeviceToDevice, st));
    S.vrows = 0;   // V rewritten: its kept slices are stale
    DV_CU(cudaMemcpyAsync(S.HV, S.HPsi, (size_t)nb * npw * zb, cudaMemcpyDeviceToDevice, st));
    v.n = nb;
    DV_TRY(update_reduced<T>(S, 0, v.n, true, st, pf));
    v.first = false;
  }
  k_resid<<<nb, 256, 0, st>>>(S.Psi, S.HPsi, S.e, npw, S.R, S.rn);
  return check_launch("k_resid");
}

// ... then the convergence test on the host; either done, or the corrections
// are appended to V and their H product is left pending.
template <typename T>
static int dv_step_finish(qe_ctx* ctx, DvSolve& v, cudaStream_t st, Prof* pf) {
  DvState& S = v.S;
  const int npw = S.npw, nb = S.nb, md = S.max_dim;
  const size_t zb = sizeof(z);
  const double pmin = 0.1;
  const double drop = 1e-6;
  int status[16];
  DV_CU(cudaMemcpyAsync(v.e.data(), S.e, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaMemcpyAsync(v.rn.data(), S.rn, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaMemcpyAsync(status, S.dw.status, sizeof(status), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaStreamSynchronize(st));
  DV_TRY(tc_check(ctx, st));
  if (status[8] != 0) {
    set_error("davidson: a grid barrier of the dense eigensolver timed out");
    return QE_ETIMEOUT;
  }
  if (status[12] != 0) {
    set_error("davidson: a tensor-core product wait timed out (code %d)", status[12]);
    return QE_ETIMEOUT;
  }
  if (status[0] != 0) {
    set_error("davidson: reduced overlap matrix not positive definite (column %d)", status[0] - 1);
    return QE_ENOCONV;
  }
  std::vector<int> unc;
  double rmax = 0.0;
  // the mixed iteration stops at 1e-4 at the finest (its FP32 rounding floor on
  // C2 is ~3e-5); dv_fp64_phase then meets the caller's tolerance
  const double tol = v.precision != QE_FP64 ? std::max(v.tol, 1e-4) : v.tol;
  for (int b = 0; b < nb; ++b) {
    if (!(v.rn[b] <= tol)) unc.push_back(b);
    rmax = std::max(rmax, std::isfinite(v.rn[b]) ? v.rn[b] : HUGE_VAL);
  }
  v.rmax = rmax;
  if (!unc.empty() && v.precision != QE_FP64) {
    // an FP32 iteration that stalls above 1e-4 (five iterations without a 20 %
    // gain) hands over to the FP64 refinement and iterations (dv_fp64_phase)
    if (rmax < 0.8 * v.best_rmax) {
      v.best_rmax = rmax;
      v.stall = 0;
    } else if (++v.stall >= 5 && rmax < 1e-3) {
      v.done = true;
      return QE_OK;
    }
  }
  if (unc.empty() && v.precision == QE_FP64 && v.rr32) {
    // converged on an FP32 Rayleigh-Ritz: redo it in FP64 before accepting
    v.rmax = 0.0;
    v.h_rows = 0;
    return QE_OK;
  }
  if (unc.empty()) { v.conv = true; v.done = true; return QE_OK; }
  if (v.it >= v.max_iter) { v.done = true; return QE_OK; }
  ++v.it;
  const int nu = (int)unc.size();
  DV_CU(cudaMemcpyAsync(S.idx, unc.data(), nu * sizeof(int), cudaMemcpyHostToDevice, st));
  k_precond<<<nu, 256, 0, st>>>(S.R, S.idx, S.e, S.hd, npw, pmin * pmin, S.D);
  DV_TRY(check_launch("k_precond"));
  if (S.gamma) {
    k_gamma_sym<<<grid_for((size_t)nu * npw), 256, 0, st>>>(S.D, nu, npw, S.mg);
    DV_TRY(check_launch("k_gamma_sym"));
  }
  if (v.n + nu > md) {
    DV_CU(cudaMemcpyAsync(S.V, S.Psi, (size_t)nb * npw * zb, cudaMemcpyDeviceToDevice, st));
    S.vrows = 0;   // V rewritten: its kept slices are stale
    DV_CU(cudaMemcpyAsync(S.HV, S.HPsi, (size_t)nb * npw * zb, cudaMemcpyDeviceToDevice, st));
    v.n = nb;
    DV_TRY(update_reduced<T>(S, 0, v.n, true, st, pf));
  }
  int nk = 0;
  DV_TRY(orthonormalise<T>(S, v.n, S.D, nu, S.V + (size_t)v.n * npw, &nk, drop, st, pf));
  if (nk == 0) { v.done = true; return QE_OK; }
  v.nk = nk;
  v.h_row = v.n;
  v.h_rows = nk;
  return QE_OK;
}

template <typename T>
static int dv_after_h(DvSolve& v, cudaStream_t st, Prof* pf) {
  DV_TRY(update_reduced<T>(v.S, v.n, v.n + v.nk, true, st, pf));
  v.n += v.nk;
  v.h_rows = 0;
  return QE_OK;
}

static int dv_apply_h(qe_ctx* ctx, DvSolve& v, cudaStream_t st) {
  const size_t off = (size_t)v.h_row * v.S.npw;
  return hpsi_core(ctx, *v.P, v.op, v.precision, (const double*)(v.S.V + off),
                   (double*)(v.S.HV + off), v.h_rows, st, v.S.gamma);
}

template <typename T>
static int dv_loop(qe_ctx* ctx, DvSolve& v, cudaStream_t st) {
  Prof* pf = &ctx->prof;
  while (true) {
    DV_TRY(dv_step_launch<T>(v, st, pf));
    DV_TRY(dv_step_finish<T>(ctx, v, st, pf));
    if (v.done) break;
    if (v.h_rows == 0) continue;   // Rayleigh-Ritz redone in FP64, no new vectors
    DV_TRY(dv_apply_h(ctx, v, st));
    DV_TRY(dv_after_h<T>(v, st, pf));
  }
  return QE_OK;
}

// End of the mixed path, after the FP64 Rayleigh-Ritz of its Ritz vectors
// (refine_pre/post): accept them if every FP64 residual is within tol, else go
// on as an FP64 Davidson from them (they are an orthonormal basis to FP64
// rounding) until tol or max_iter.  The mixed path thus meets the same
// residual criterion as the FP64 one, with most iterations in FP32.
// First half: the decision and the FP64 basis; *more = true when FP64
// iterations follow (dv_loop<double>, or a lockstep driver's rounds).
static int dv_fp64_begin(qe_ctx* ctx, DvSolve& v, cudaStream_t st, bool* more) {
  DvState& S = v.S;
  const int nb = S.nb, npw = S.npw;
  *more = false;
  DV_CU(cudaMemcpyAsync(v.rn.data(), S.rn, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaStreamSynchronize(st));
  double rmax = 0.0;
  bool all = true;
  for (int b = 0; b < nb; ++b) {
    if (!(v.rn[b] <= v.tol)) all = false;
    rmax = std::max(rmax, std::isfinite(v.rn[b]) ? v.rn[b] : HUGE_VAL);
  }
  v.conv = all;
  if (all || v.it >= v.max_iter) return QE_OK;
  const size_t bytes = (size_t)nb * npw * sizeof(z);
  DV_CU(cudaMemcpyAsync(S.V, S.Psi, bytes, cudaMemcpyDeviceToDevice, st));
  S.vrows = 0;   // V rewritten: its kept slices are stale
  DV_CU(cudaMemcpyAsync(S.HV, S.HPsi, bytes, cudaMemcpyDeviceToDevice, st));
  v.n = nb;
  DV_TRY(update_reduced<double>(S, 0, nb, true, st, &ctx->prof));
  v.precision = QE_FP64;
  v.first = false;
  v.done = false;
  v.conv = false;
  v.rmax = rmax;
  v.h_rows = 0;
  *more = true;
  return QE_OK;
}

static int dv_fp64_phase(qe_ctx* ctx, DvSolve& v, cudaStream_t st) {
  bool more = false;
  DV_TRY(dv_fp64_begin(ctx, v, st, &more));
  return more ? dv_loop<double>(ctx, v, st) : QE_OK;
}

template <typename T>
static int davidson_run(qe_ctx* ctx, DvSolve& v, cudaStream_t st) {
  Prof* pf = &ctx->prof;
  DV_TRY(dv_begin(v, st));
  DV_TRY(dv_apply_h(ctx, v, st));
  DV_TRY(dv_after_first_h<T>(v, st, pf));
  DV_TRY(dv_loop<T>(ctx, v, st));
  if (v.precision != QE_FP64) {
    DV_TRY(refine_pre(v.S, st));
    DV_TRY(hpsi_core(ctx, *v.P, v.op, QE_FP64, (const double*)v.S.V, (double*)v.S.HV, v.S.nb, st,
                     v.S.gamma));
    DV_TRY(refine_post(v.S, st, pf));
    DV_TRY(dv_fp64_phase(ctx, v, st));
  }
  return QE_OK;
}

// Lockstep over a batch of solves: each H product of an iteration, for every
// solve still running, goes through one batched H|psi> (batch.cu).
template <typename T>
static int davidson_batch_run(qe_ctx* ctx, std::vector<DvSolve>& vs,
                              const std::vector<qe_problem>& probs, cudaStream_t st,
                              std::vector<int>& rcs) {
  Prof* pf = &ctx->prof;
  const int np = (int)vs.size();
  auto apply_pending = [&](int precision) -> int {
    std::vector<qe_problem> pr;
    std::vector<const double*> in;
    std::vector<double*> out;
    std::vector<char> pair;
    for (int p = 0; p < np; ++p) {
      DvSolve& v = vs[p];
      if (rcs[p] != QE_OK || v.h_rows == 0) continue;
      qe_problem q = probs[p];
      q.nbnd = v.h_rows;
      pr.push_back(q);
      const size_t off = (size_t)v.h_row * v.S.npw;
      in.push_back((const double*)(v.S.V + off));
      out.push_back((double*)(v.S.HV + off));
      pair.push_back(v.S.gamma ? 1 : 0);
    }
    if (pr.empty()) return QE_OK;
    return hpsi_batch_core(ctx, (int)pr.size(), pr.data(), precision, in.data(), out.data(), st,
                           pair.data());
  };
  for (int p = 0; p < np; ++p) rcs[p] = dv_begin(vs[p], st);
  DV_TRY(apply_pending(vs[0].precision));
  for (int p = 0; p < np; ++p)
    if (rcs[p] == QE_OK) rcs[p] = dv_after_first_h<T>(vs[p], st, pf);
  while (true) {
    bool any = false;
    for (int p = 0; p < np; ++p)
      if (rcs[p] == QE_OK && !vs[p].done) rcs[p] = dv_step_launch<T>(vs[p], st, pf);
    for (int p = 0; p < np; ++p) {
      DvSolve& v = vs[p];
      if (rcs[p] != QE_OK || v.done) continue;
      rcs[p] = dv_step_finish<T>(ctx, v, st, pf);
      if (rcs[p] == QE_OK && !v.done) any = true;
    }
    if (!any) break;
    DV_TRY(apply_pending(vs[0].precision));
    for (int p = 0; p < np; ++p) {
      DvSolve& v = vs[p];
      if (rcs[p] == QE_OK && !v.done && v.h_rows > 0) rcs[p] = dv_after_h<T>(v, st, pf);
    }
  }
  if (vs[0].precision != QE_FP64) {
    for (int p = 0; p < np; ++p) {
      DvSolve& v = vs[p];
      v.h_rows = 0;
      if (rcs[p] != QE_OK) continue;
      rcs[p] = refine_pre(v.S, st);
      v.h_row = 0;
      v.h_rows = v.S.nb;
    }
    DV_TRY(apply_pending(QE_FP64));
    for (int p = 0; p < np; ++p)
      if (rcs[p] == QE_OK) rcs[p] = refine_post(vs[p].S, st, pf);
    for (int p = 0; p < np; ++p)
      if (rcs[p] == QE_OK) rcs[p] = dv_fp64_phase(ctx, vs[p], st);
  }
  return QE_OK;
}

// Default basis size.  Four nbnd for small blocks; with two (Quantum ESPRESSO's
// default workspace) the iteration stalls on the SMALL cell (7 bands, band 7
// close to band 8) and the FP64 C2 solve needs 48 instead of 19 iterations.
// From 64 bands on, where the reduced eigenproblem's cost dominates an
// iteration, 3.5 nbnd: on C2 (256 bands) the same 19 FP64 / 16 mixed
// iterations as with 4 nbnd, 1.44 s against 1.48 s FP64 and 0.26 s against
// 0.31 s mixed (3 nbnd: 28 FP64 iterations).  Callers can pass max_dim.
int default_max_dim(int nb) { return nb < 64 ? 4 * nb : (7 * nb + 1) / 2; }

}  // namespace qe

using namespace qe;

namespace {

// Whether a k = 0 solve keeps its bands real in r (QE_GAMMA / QE_NO_GAMMA
// decide when given).  By default on grids of at least 48^3 points: C2 (96^3)
// at the matched tolerance takes 12 iterations either way, FP64 0.31 -> 0.23 s
// and mixed 0.21 -> 0.17 s (FFTs halved, real products and real reduced
// problems); on smaller grids the FFTs are a small share and the mode's extra
// launches cost as much as it saves (C0, 32^3: 17 -> 18 ms).  A mixed solve
// with FP32 reduced problems (QE_RR_FP32) keeps complex bands unless asked:
// with real bands its FP32 phase needed 23 instead of 16 iterations on C2 (a
// complex basis spans the real and imaginary parts of its vectors, twice the
// real dimension).
static bool gamma_mode(int precision, int flags, const int grid[3]) {
  if (flags & QE_NO_GAMMA) return false;
  if (flags & QE_GAMMA) return true;
  if (precision == QE_MIXED && (flags & QE_RR_FP32)) return false;
  return (long long)grid[0] * grid[1] * grid[2] >= 48ll * 48 * 48;
}

// Checks of one problem's arguments, its plan and operator, and the layout of
// its Davidson workspace in `basis` / `red`.
int dv_setup(qe_ctx* ctx, const qe_problem* prob, int precision, double tol, int max_iter,
             int max_dim, DevBuf& basis, DevBuf& red, DvSolve& v, cudaStream_t st, const char* who,
             bool allow_gamma) {
  DV_TRY(check_problem(prob, who));
  const int nb = prob->nbnd;
  DevPlan* P = nullptr;
  DV_TRY(get_plan(ctx, prob->lat, prob->k, prob->ecutwfc, prob->grid, &P));
  const int npw = P->h.npw;
  if (nb > npw) { set_error("%s: %d bands > %d plane waves", who, nb, npw); return QE_EINVAL; }
  int md = max_dim > 0 ? max_dim : default_max_dim(nb);
  if (md < 2 * nb) { set_error("%s: max_dim %d < 2 nbnd", who, md); return QE_EINVAL; }
  md = std::min(md, std::max(2 * nb, npw));
  if (md > kMaxDense) { set_error("%s: max_dim %d above %d", who, md, kMaxDense); return QE_EINVAL; }
  v.P = P;
  DV_TRY(resolve_operator(ctx, prob, *P, v.op, st));
  v.precision = precision;
  v.tol = tol;
  v.max_iter = max_iter;
  DvState& S = v.S;
  S.npw = npw;
  S.nb = nb;
  S.max_dim = md;
  S.np = prob->nproj;
  DV_TRY(dv_alloc(basis, red, S, precision == QE_FP64));
  if (ctx->test_wait_ns) {
    S.dw.bar.wait_ns = ctx->test_wait_ns;
    S.dw.bar.stall = 1;
  }
  S.gamma = false;
  S.mg = nullptr;
  if (allow_gamma && P->h.gamma && P->mg) {
    // real-in-r mode needs real projectors: B_i(-G) = conj B_i(G)
    bool real_beta = true;
    if (v.op.nproj > 0) {
      unsigned long long* w = reinterpret_cast<unsigned long long*>(S.dw.y);
      DV_CU(cudaMemsetAsync(w, 0, 2 * sizeof(unsigned long long), st));
      k_beta_mirror<<<grid_for((size_t)v.op.nproj * npw), 256, 0, st>>>(
          (const z*)v.op.beta, v.op.nproj, npw, P->mg, w);
      DV_TRY(check_launch("k_beta_mirror"));
      unsigned long long hw[2];
      DV_CU(cudaMemcpyAsync(hw, w, sizeof(hw), cudaMemcpyDeviceToHost, st));
      DV_CU(cudaStreamSynchronize(st));
      double dmax, bmax;
      std::memcpy(&dmax, &hw[0], sizeof(double));
      std::memcpy(&bmax, &hw[1], sizeof(double));
      real_beta = dmax <= 1e-12 * bmax;
    }
    S.gamma = real_beta;
    S.mg = real_beta ? P->mg : nullptr;
  }
  return QE_OK;
}

// Final status of a solve: barrier and overlap checks of the last Rayleigh-Ritz.
int dv_final_status(DvSolve& v, cudaStream_t st, const char* who) {
  int fin[16];
  DV_CU(cudaMemcpyAsync(fin, v.S.dw.status, sizeof(fin), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaStreamSynchronize(st));
  if (fin[8] != 0) { set_error("%s: a grid barrier of the dense eigensolver timed out", who); return QE_ETIMEOUT; }
  if (fin[12] != 0) { set_error("%s: a tensor-core product wait timed out", who); return QE_ETIMEOUT; }
  if (fin[0] != 0) { set_error("%s: final overlap matrix not positive definite", who); return QE_ENOCONV; }
  return QE_OK;
}

// ---- band-by-band conjugate gradient ------------------------------------------------
// Sec. 3.3 names the conjugate-gradient method beside Davidson.  Each band
// minimises the Rayleigh quotient in the complement of the bands below it, along
// preconditioned Polak-Ribiere directions, with an exact line minimisation on
// the unit sphere (Teter, Payne and Allan 1989); a sweep over the bands ends with
// a Rayleigh-Ritz rotation of the block.  The vector operations of one band run
// in single-CTA kernels (one fixed-order reduction each); the projections on the
// lower bands and H are the library's products.

// e = Re<p|hp>; g = hp - e p; ||g||; z = g / sqrt((h_G - e)^2 + pmin^2)
__global__ void __launch_bounds__(1024) k_cg_grad(const z* __restrict__ p, const z* __restrict__ hp,
                                                  const double* __restrict__ hd, int npw, double pmin2,
                                                  z* __restrict__ g, z* __restrict__ zz, double* sc) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) s += p[i].x * hp[i].x + p[i].y * hp[i].y;
  const double e = dv_block_sum(s, sh);
  double gg = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    const z a = hp[i], b = p[i];
    const z v = {a.x - e * b.x, a.y - e * b.y};
    g[i] = v;
    gg += v.x * v.x + v.y * v.y;
    const double x = hd[i] - e;
    const double inv = rsqrt(x * x + pmin2);
    zz[i] = {v.x * inv, v.y * inv};
  }
  gg = dv_block_sum(gg, sh);
  if (threadIdx.x == 0) { sc[0] = e; sc[1] = sqrt(gg); }
}

// d = z (first) or z + max(0, Re<z, g - g_prev> / gz_prev) d_prev; sc[3] = Re<z, g>
__global__ void __launch_bounds__(1024) k_cg_dir(const z* __restrict__ zz, const z* __restrict__ g,
                                                 const z* __restrict__ gp, const z* __restrict__ dp,
                                                 z* __restrict__ d, int npw, int first, double* sc) {
  __shared__ double sh[33];
  double num = 0.0, gz = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    const z a = zz[i], b = g[i];
    gz += a.x * b.x + a.y * b.y;
    if (!first) {
      const z c = gp[i];
      num += a.x * (b.x - c.x) + a.y * (b.y - c.y);
    }
  }
  gz = dv_block_sum(gz, sh);
  num = dv_block_sum(num, sh);
  const double beta = first ? 0.0 : fmax(0.0, num / sc[2]);
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    const z a = zz[i];
    if (first) d[i] = a;
    else d[i] = {a.x + beta * dp[i].x, a.y + beta * dp[i].y};
  }
  if (threadIdx.x == 0) sc[3] = gz;
}

// dn = d / ||d||
__global__ void __launch_bounds__(1024) k_cg_unit(const z* __restrict__ d, z* __restrict__ dn, int npw) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) s += d[i].x * d[i].x + d[i].y * d[i].y;
  s = dv_block_sum(s, sh);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) dn[i] = {d[i].x * inv, d[i].y * inv};
}

// exact line minimum on p(t) = cos t p + sin t dn: b = Re<p|H dn>, c = <dn|H dn>,
// t = atan2(-2b, c - e) / 2; p, hp move there; gz_prev <- gz
__global__ void __launch_bounds__(1024) k_cg_step(z* __restrict__ p, z* __restrict__ hp,
                                                  const z* __restrict__ dn, const z* __restrict__ hdn,
                                                  int npw, double* sc) {
  __shared__ double sh[33];
  double b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    const z h = hdn[i];
    b += p[i].x * h.x + p[i].y * h.y;
    c += dn[i].x * h.x + dn[i].y * h.y;
  }
  b = dv_block_sum(b, sh);
  c = dv_block_sum(c, sh);
  const double t = 0.5 * atan2(-2.0 * b, c - sc[0]);
  double sn, cs;
  sincos(t, &sn, &cs);
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    const z a = p[i], u = dn[i], ha = hp[i], hu = hdn[i];
    p[i] = {cs * a.x + sn * u.x, cs * a.y + sn * u.y};
    hp[i] = {cs * ha.x + sn * hu.x, cs * ha.y + sn * hu.y};
  }
  __syncthreads();
  if (threadIdx.x == 0) sc[2] = sc[3];
}

// p, hp <- p / ||p||, hp / ||p||
__global__ void __launch_bounds__(1024) k_cg_renorm(z* __restrict__ p, z* __restrict__ hp, int npw) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < npw; i += blockDim.x) s += p[i].x * p[i].x + p[i].y * p[i].y;
  s = dv_block_sum(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int i = threadIdx.x; i < npw; i += blockDim.x) {
    p[i] = {p[i].x * inv, p[i].y * inv};
    hp[i] = {hp[i].x * inv, hp[i].y * inv};
  }
}

// x -= A^T (A^+ x) over the rows [0, m) of A (projection on orthonormal rows);
// with hx, also hx -= HA^T (A^+ x) (the same combination of the H products).
template <typename T>
static int cg_project(const DvState& S, const z* A, const z* HA, int m, z* x, z* hx,
                      cudaStream_t st, Prof* pf) {
  if (m <= 0) return QE_OK;
  const int npw = S.npw;
  DV_TRY(gemm_inner<T>((const double*)A, npw, (const double*)x, npw, m, 1, npw, (double*)S.G, 1,
                       S.part, S.part_bytes, st, pf));
  if (hx)
    DV_TRY(gemm_outer_ab<T>((const double*)HA, npw, (const double*)S.G, 1, npw, 1, m, (double*)hx,
                            npw, 1, 1, st, pf));
  return gemm_outer_ab<T>((const double*)A, npw, (const double*)S.G, 1, npw, 1, m, (double*)x, npw,
                          1, 1, st, pf);
}

struct CgRun {
  int iters = 0, sweeps = 0;
  bool conv = false;
};

// Rayleigh-Ritz of span(Psi) (FP64 reduced problem, products in T), the
// rotated bands and their residual norms; returns the largest residual norm.
template <typename T>
static int cg_rotate(qe_ctx* ctx, DvSolve& v, cudaStream_t st, double* rmax) {
  DvState& S = v.S;
  Prof* pf = &ctx->prof;
  const int nb = S.nb, npw = S.npw;
  const size_t bytes = (size_t)nb * npw * sizeof(z);
  DV_CU(cudaMemcpyAsync(S.V, S.Psi, bytes, cudaMemcpyDeviceToDevice, st));
  S.vrows = 0;   // V rewritten: its kept slices are stale
  DV_CU(cudaMemcpyAsync(S.HV, S.HPsi, bytes, cudaMemcpyDeviceToDevice, st));
  DV_TRY(update_reduced<T>(S, 0, nb, true, st, pf));
  DV_CU(cudaMemsetAsync(S.dw.status, 0, sizeof(int), st));
  DV_TRY(rayleigh_ritz(S, nb, true, st, pf));
  DV_TRY(outer<T>(S, S.V, npw, S.X, nb, npw, nb, nb, S.Psi, npw, 0, 0, st, pf));
  DV_TRY(outer<T>(S, S.HV, npw, S.X, nb, npw, nb, nb, S.HPsi, npw, 0, 0, st, pf));
  k_resid<<<nb, 256, 0, st>>>(S.Psi, S.HPsi, S.e, npw, S.R, S.rn);
  DV_TRY(check_launch("k_resid"));
  DV_CU(cudaMemcpyAsync(v.rn.data(), S.rn, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  DV_CU(cudaStreamSynchronize(st));
  DV_TRY(tc_check(ctx, st));
  double r = 0.0;
  for (int b = 0; b < nb; ++b) r = std::max(r, std::isfinite(v.rn[b]) ? v.rn[b] : HUGE_VAL);
  *rmax = r;
  return QE_OK;
}

// One sweep: every band in turn, at most max_iter CG iterations each.
template <typename T>
static int cg_sweep(qe_ctx* ctx, DvSolve& v, int precision, double tol, int max_iter, CgRun& run,
                    cudaStream_t st) {
  DvState& S = v.S;
  Prof* pf = &ctx->prof;
  const int nb = S.nb, npw = S.npw;
  const double pmin2 = 0.1 * 0.1;
  // scratch rows past the bands: V[nb..nb+3], HV[nb..nb+3] (max_dim >= nb + 4)
  z* g = S.V + (size_t)nb * npw;
  z* gp = g + npw;
  z* zz = gp + npw;
  z* zp = zz + npw;
  z* d = S.HV + (size_t)(nb + 2) * npw;
  z* dp = d + npw;
  z* dn = S.HV + (size_t)nb * npw;
  z* hdn = dn + npw;
  double* sc = reinterpret_cast<double*>(S.C);
  for (int n = 0; n < nb; ++n) {
    z* p = S.Psi + (size_t)n * npw;
    z* hp = S.HPsi + (size_t)n * npw;
    if (n > 0) {
      DV_TRY(cg_project<T>(S, S.Psi, S.HPsi, n, p, hp, st, pf));
      k_cg_renorm<<<1, 1024, 0, st>>>(p, hp, npw);
      DV_TRY(check_launch("k_cg_renorm"));
    }
    for (int it = 0; it < max_iter; ++it) {
      k_cg_grad<<<1, 1024, 0, st>>>(p, hp, S.hd, npw, pmin2, g, zz, sc);
      DV_TRY(check_launch("k_cg_grad"));
      double gn = 0.0;
      DV_CU(cudaMemcpyAsync(&gn, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      DV_CU(cudaStreamSynchronize(st));
      if (!(gn > tol)) break;
      DV_TRY(cg_project<T>(S, S.Psi, nullptr, n + 1, zz, nullptr, st, pf));
      k_cg_dir<<<1, 1024, 0, st>>>(zz, g, gp, dp, d, npw, it == 0 ? 1 : 0, sc);
      DV_TRY(check_launch("k_cg_dir"));
      DV_TRY(cg_project<T>(S, S.Psi, nullptr, n + 1, d, nullptr, st, pf));
      k_cg_unit<<<1, 1024, 0, st>>>(d, dn, npw);
      DV_TRY(check_launch("k_cg_unit"));
      DV_TRY(hpsi_core(ctx, *v.P, v.op, precision, (const double*)dn, (double*)hdn, 1, st));
      k_cg_step<<<1, 1024, 0, st>>>(p, hp, dn, hdn, npw, sc);
      DV_TRY(check_launch("k_cg_step"));
      std::swap(g, gp);
      std::swap(zz, zp);
      std::swap(d, dp);
      ++run.iters;
    }
  }
  ++run.sweeps;
  return QE_OK;
}

// The whole solve: start block rotated, sweeps until every residual <= tol.
// The mixed path sweeps with FP32 products and H while its residuals are above
// max(tol, 1e-4) (the FP32 rounding floor), then recomputes H Psi in FP64 and
// goes on in FP64.
static int cg_run(qe_ctx* ctx, DvSolve& v, double tol, int max_iter, int max_sweeps, CgRun& run,
                  cudaStream_t st) {
  DvState& S = v.S;
  const int nb = S.nb, npw = S.npw;
  const size_t bytes = (size_t)nb * npw * sizeof(z);
  DV_TRY(dv_begin(v, st));
  int prec = v.precision;
  DV_TRY(hpsi_core(ctx, *v.P, v.op, prec, (const double*)S.V, (double*)S.HV, nb, st));
  DV_CU(cudaMemcpyAsync(S.Psi, S.V, bytes, cudaMemcpyDeviceToDevice, st));
  DV_CU(cudaMemcpyAsync(S.HPsi, S.HV, bytes, cudaMemcpyDeviceToDevice, st));
  double rmax = HUGE_VAL;
  DV_TRY(prec == QE_FP64 ? cg_rotate<double>(ctx, v, st, &rmax) : cg_rotate<float>(ctx, v, st, &rmax));
  while (true) {
    if (prec != QE_FP64 && (rmax <= std::max(tol, 1e-4) || run.sweeps >= max_sweeps)) {
      prec = QE_FP64;
      DV_TRY(hpsi_core(ctx, *v.P, v.op, prec, (const double*)S.Psi, (double*)S.HPsi, nb, st));
      DV_TRY(cg_rotate<double>(ctx, v, st, &rmax));
    }
    if (rmax <= tol || run.sweeps >= max_sweeps) break;
    DV_TRY(prec == QE_FP64 ? cg_sweep<double>(ctx, v, prec, tol, max_iter, run, st)
                           : cg_sweep<float>(ctx, v, prec, std::max(tol, 1e-4), max_iter, run, st));
    DV_TRY(prec == QE_FP64 ? cg_rotate<double>(ctx, v, st, &rmax) : cg_rotate<float>(ctx, v, st, &rmax));
  }
  run.conv = prec == QE_FP64 && rmax <= tol;
  (void)npw;
  return QE_OK;
}

}  // namespace

// ---- lockstep rounds of independent solves (serving) --------------------------------
namespace qe {

enum { DV_FIRST_H = 0, DV_STEP = 1, DV_H = 2, DV_REFINE_H = 3, DV_DONE = 4 };

struct DvTask {
  cudaStream_t cur = nullptr;   // stream of the task's buffers (the driver's)
  DevBuf basis, red, opbuf;     // Davidson workspace; device copies of V, beta, D
  qe_problem prob{};            // device pointers into opbuf
  DvSolve v;
  int phase = DV_FIRST_H;
  int h_prec = QE_FP64;         // arithmetic of the pending H product
  int rc = QE_OK;
  std::string err;              // message of the error that ended it
  DvTask() {
    basis.sp = &cur;
    red.sp = &cur;
    opbuf.sp = &cur;
  }
};

int dv_task_create(qe_ctx* ctx, const qe_problem* prob, int precision, double tol, int max_iter,
                   int max_dim, const double* psi0, void* stream, DvTask** out) {
  *out = nullptr;
  DV_TRY(check_problem(prob, "dv_task"));
  if (!psi0) { set_error("dv_task: null start bands"); return QE_EINVAL; }
  const bool dev_in = prob->mem == QE_DEVICE;
  const int flags = precision & (QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  precision &= ~(QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  cudaStream_t st = (cudaStream_t)stream;
  DevPlan* P = nullptr;
  DV_TRY(get_plan(ctx, prob->lat, prob->k, prob->ecutwfc, prob->grid, &P));
  auto t = std::make_unique<DvTask>();
  t->cur = st;
  t->prob = *prob;
  if (!dev_in) {
    // host operator: device copies owned by the task
    const size_t ngrid = (size_t)P->grid[0] * P->grid[1] * P->grid[2];
    const size_t nbeta = (size_t)prob->nproj * P->h.npw * 2, nd = (size_t)prob->nproj * prob->nproj;
    const size_t ov = (ngrid * sizeof(double) + 255) & ~(size_t)255;
    const size_t ob = (nbeta * sizeof(double) + 255) & ~(size_t)255;
    DV_TRY(t->opbuf.ensure(ov + ob + nd * sizeof(double) + 256));
    char* base = static_cast<char*>(t->opbuf.p);
    DV_CU(cudaMemcpyAsync(base, prob->vloc_r, ngrid * sizeof(double), cudaMemcpyHostToDevice, st));
    if (prob->nproj > 0) {
      DV_CU(cudaMemcpyAsync(base + ov, prob->beta, nbeta * sizeof(double), cudaMemcpyHostToDevice, st));
      DV_CU(cudaMemcpyAsync(base + ov + ob, prob->dmat, nd * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    t->prob.vloc_r = reinterpret_cast<const double*>(base);
    t->prob.beta = prob->nproj > 0 ? reinterpret_cast<const double*>(base + ov) : nullptr;
    t->prob.dmat = prob->nproj > 0 ? reinterpret_cast<const double*>(base + ov + ob) : nullptr;
    t->prob.mem = QE_DEVICE;
  }
  DV_TRY(dv_setup(ctx, &t->prob, precision, tol, max_iter, max_dim, t->basis, t->red, t->v, st,
                  "dv_task", gamma_mode(precision, flags, prob->grid)));
  t->v.mixed_rr32 = (flags & QE_RR_FP32) != 0;
  DvState& S = t->v.S;
  DV_CU(cudaMemcpyAsync(S.V, psi0, (size_t)S.nb * S.npw * sizeof(z),
                        dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  S.vrows = 0;
  DV_TRY(dv_begin(t->v, st));
  t->phase = DV_FIRST_H;
  t->h_prec = precision;
  *out = t.release();
  return QE_OK;
}

bool dv_task_done(const DvTask* t) { return t->phase == DV_DONE || t->rc != QE_OK; }

// After the FP64 Rayleigh-Ritz that ends the mixed path's FP32 phase.
static int dv_task_after_refine(qe_ctx* ctx, DvTask& t, cudaStream_t st) {
  bool more = false;
  DV_TRY(dv_fp64_begin(ctx, t.v, st, &more));
  t.phase = more ? DV_STEP : DV_DONE;
  return QE_OK;
}

int dv_round(qe_ctx* ctx, DvTask* const* tasks, int n, void* stream, void* const* side, int nside,
             void* const* events) {
  cudaStream_t st = (cudaStream_t)stream;
  Prof* pf = &ctx->prof;
  auto live = [&](const DvTask* t) { return t->rc == QE_OK && t->phase != DV_DONE; };
  // task i runs its own work on side stream i % nside (the same stream in every
  // round, so a task's work stays in order)
  const int ns = std::max(1, nside);
  auto sst = [&](int i) { return nside > 0 ? (cudaStream_t)side[i % ns] : st; };
  // 1. the pending H products, one batched call per arithmetic on `stream`
  std::vector<int> after;   // tasks whose H product ran in this round
  for (int prec : {QE_FP64, QE_MIXED}) {
    std::vector<int> ts;
    std::vector<qe_problem> pr;
    std::vector<const double*> in;
    std::vector<double*> outp;
    std::vector<char> pair;
    for (int i = 0; i < n; ++i) {
      DvTask* t = tasks[i];
      const bool wants = t->phase == DV_FIRST_H || t->phase == DV_H || t->phase == DV_REFINE_H;
      if (!live(t) || !wants || t->h_prec != prec || t->v.h_rows <= 0) continue;
      qe_problem q = t->prob;
      q.nbnd = t->v.h_rows;
      const size_t off = (size_t)t->v.h_row * t->v.S.npw;
      ts.push_back(i);
      pr.push_back(q);
      in.push_back(reinterpret_cast<const double*>(t->v.S.V + off));
      outp.push_back(reinterpret_cast<double*>(t->v.S.HV + off));
      pair.push_back(t->v.S.gamma ? 1 : 0);
    }
    if (pr.empty()) continue;
    const int rc = hpsi_batch_core(ctx, (int)pr.size(), pr.data(), prec, in.data(), outp.data(), st,
                                   pair.data());
    if (rc) {
      for (int i : ts) tasks[i]->rc = rc;
      continue;
    }
    after.insert(after.end(), ts.begin(), ts.end());
  }
  // fork: every side stream follows the H products
  bool forked = false;
  auto fork = [&]() -> int {
    if (forked || nside <= 0) return QE_OK;
    forked = true;
    DV_CU(cudaEventRecord((cudaEvent_t)events[0], st));
    for (int k = 0; k < ns; ++k) DV_CU(cudaStreamWaitEvent((cudaStream_t)side[k], (cudaEvent_t)events[0], 0));
    return QE_OK;
  };
  // 2. what follows each H product (the new reduced-matrix blocks), each task
  //    on its side stream
  if (!after.empty()) DV_TRY(fork());
  for (int i : after) {
    DvTask* t = tasks[i];
    DvSolve& v = t->v;
    const bool f64 = v.precision == QE_FP64;
    const cudaStream_t s = sst(i);
    if (t->phase == DV_FIRST_H) {
      t->rc = f64 ? dv_after_first_h<double>(v, s, pf) : dv_after_first_h<float>(v, s, pf);
      t->phase = DV_STEP;
    } else if (t->phase == DV_H) {
      t->rc = f64 ? dv_after_h<double>(v, s, pf) : dv_after_h<float>(v, s, pf);
      t->phase = DV_STEP;
    } else {
      v.h_rows = 0;
      t->rc = refine_post(v.S, s, pf);
      if (t->rc == QE_OK) t->rc = dv_task_after_refine(ctx, *t, s);
    }
  }
  // 3. one Rayleigh-Ritz step of every task at that stage: all launched, then
  //    the convergence tests in turn (each waits for its own stream only)
  std::vector<int> step;
  for (int i = 0; i < n; ++i)
    if (live(tasks[i]) && tasks[i]->phase == DV_STEP) step.push_back(i);
  if (!step.empty()) DV_TRY(fork());
  for (int i : step) {
    DvTask* t = tasks[i];
    t->rc = t->v.precision == QE_FP64 ? dv_step_launch<double>(t->v, sst(i), pf)
                                      : dv_step_launch<float>(t->v, sst(i), pf);
  }
  // The convergence test and the orthonormalisation of the corrections wait on
  // the host for their task's stream (residual norms, dropped columns): one
  // host thread per side stream takes that stream's tasks in order, so that
  // one task's waits do not hold back the launches of the others.
  auto finish = [&](int i) {
    DvTask* t = tasks[i];
    if (t->rc != QE_OK) return;
    DvSolve& v = t->v;
    t->rc = v.precision == QE_FP64 ? dv_step_finish<double>(ctx, v, sst(i), pf)
                                   : dv_step_finish<float>(ctx, v, sst(i), pf);
    if (t->rc != QE_OK) { t->err = qe_last_error(); return; }
    if (v.done) {
      if (v.precision != QE_FP64) {
        // the FP32 phase ended: FP64 H of the Ritz vectors, FP64 Rayleigh-Ritz
        t->rc = refine_pre(v.S, sst(i));
        if (t->rc != QE_OK) t->err = qe_last_error();
        v.h_row = 0;
        v.h_rows = v.S.nb;
        t->h_prec = QE_FP64;
        t->phase = DV_REFINE_H;
      } else {
        t->phase = DV_DONE;
      }
    } else if (v.h_rows > 0) {
      t->h_prec = v.precision;
      t->phase = DV_H;
    }
  };
  const int nworkers = std::min(ns, (int)step.size());
  if (nside > 1 && nworkers > 1) {
    std::vector<std::thread> workers;
    workers.reserve(nworkers);
    for (int k = 0; k < nworkers; ++k)
      workers.emplace_back([&, k]() {
        cudaSetDevice(ctx->device);
        for (int i : step)
          if (i % ns == k) finish(i);
      });
    for (auto& w : workers) w.join();
  } else {
    for (int i : step) finish(i);
  }
  for (int i : step)
    if (tasks[i]->rc != QE_OK && !tasks[i]->err.empty()) set_error("%s", tasks[i]->err.c_str());
  if (forked) {
    // join: the next round's H products follow every task's work
    for (int k = 0; k < ns; ++k) {
      DV_CU(cudaEventRecord((cudaEvent_t)events[1 + k], (cudaStream_t)side[k]));
      DV_CU(cudaStreamWaitEvent(st, (cudaEvent_t)events[1 + k], 0));
    }
  }
  return QE_OK;
}

int dv_task_result(qe_ctx* ctx, DvTask* t, double* psi, double* evals, double* resid, int* iters,
                   bool device_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  DvSolve& v = t->v;
  DvState& S = v.S;
  const cudaMemcpyKind kind = device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (iters) *iters = v.it;
  if (t->rc != QE_OK && t->rc != QE_ENOCONV) {
    if (!t->err.empty()) set_error("%s", t->err.c_str());
    return t->rc;
  }
  if (psi) DV_CU(cudaMemcpyAsync(psi, S.Psi, (size_t)S.nb * S.npw * sizeof(z), kind, st));
  if (evals) DV_CU(cudaMemcpyAsync(evals, S.e, S.nb * sizeof(double), kind, st));
  if (resid) DV_CU(cudaMemcpyAsync(resid, S.rn, S.nb * sizeof(double), kind, st));
  DV_TRY(dv_final_status(v, st, "davidson"));
  if (t->rc == QE_ENOCONV) return QE_ENOCONV;
  if (!v.conv) {
    set_error("davidson: not converged after %d iterations", v.it);
    return QE_ENOCONV;
  }
  return QE_OK;
}

void dv_task_destroy(DvTask* t, void* stream) {
  if (!t) return;
  t->cur = (cudaStream_t)stream;
  t->basis.release();
  t->red.release();
  t->opbuf.release();
  delete t;
}

}  // namespace qe

extern "C" int qe_davidson(qe_ctx* ctx, const qe_problem* prob, int precision, double tol,
                           int max_iter, int max_dim, double* psi_inout, double* evals,
                           double* resid, int* iters, void* stream) {
  clear_error();
  if (!ctx) { set_error("qe_davidson: null context"); return QE_EINVAL; }
  DV_TRY(check_problem(prob, "qe_davidson"));
  const int flags = precision & (QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  precision &= ~(QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_davidson: bad precision"); return QE_EINVAL; }
  if (!(tol > 0.0) || max_iter < 0) { set_error("qe_davidson: tol must be > 0, max_iter >= 0"); return QE_EINVAL; }
  const bool allow_gamma = gamma_mode(precision, flags, prob->grid);
  const int nb = prob->nbnd;
  if (iters) *iters = 0;
  if (nb == 0) return QE_OK;
  if (!psi_inout || !evals) { set_error("qe_davidson: null psi/evals"); return QE_EINVAL; }
  DV_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DV_TRY(ctx_begin(ctx, st));
  DvSolve v;
  DV_TRY(dv_setup(ctx, prob, precision, tol, max_iter, max_dim, ctx->dv_basis, ctx->dv_red, v, st,
                  "qe_davidson", allow_gamma));
  v.mixed_rr32 = (flags & QE_RR_FP32) != 0;
  DvState& S = v.S;
  const size_t bytes = (size_t)nb * S.npw * sizeof(z);
  const cudaMemcpyKind in_kind = prob->mem == QE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind out_kind = prob->mem == QE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  DV_CU(cudaMemcpyAsync(S.V, psi_inout, bytes, in_kind, st));
  S.vrows = 0;   // V rewritten: its kept slices are stale
  int rc = precision == QE_FP64 ? davidson_run<double>(ctx, v, st) : davidson_run<float>(ctx, v, st);
  if (iters) *iters = v.it;
  if (rc && rc != QE_ENOCONV) return rc;
  DV_CU(cudaMemcpyAsync(psi_inout, S.Psi, bytes, out_kind, st));
  DV_CU(cudaMemcpyAsync(evals, S.e, nb * sizeof(double), out_kind, st));
  if (resid) DV_CU(cudaMemcpyAsync(resid, S.rn, nb * sizeof(double), out_kind, st));
  DV_TRY(dv_final_status(v, st, "qe_davidson"));
  DV_TRY(tc_check(ctx, st));
  if (rc == QE_ENOCONV) return rc;
  if (!v.conv) {
    set_error("qe_davidson: not converged after %d iterations", v.it);
    return QE_ENOCONV;
  }
  return QE_OK;
}

extern "C" int qe_davidson_batch(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                                 double tol, int max_iter, int max_dim, double* const* psi_inout,
                                 double* const* evals, double* const* resid, int* iters,
                                 int* status, void* stream) {
  clear_error();
  if (!ctx) { set_error("qe_davidson_batch: null context"); return QE_EINVAL; }
  if (nprob < 0 || (nprob > 0 && (!probs || !psi_inout || !evals))) {
    set_error("qe_davidson_batch: bad problem list");
    return QE_EINVAL;
  }
  const int flags = precision & (QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  precision &= ~(QE_GAMMA | QE_NO_GAMMA | QE_RR_FP32);
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_davidson_batch: bad precision"); return QE_EINVAL; }
  if (!(tol > 0.0) || max_iter < 0) { set_error("qe_davidson_batch: tol must be > 0, max_iter >= 0"); return QE_EINVAL; }
  for (int p = 0; p < nprob; ++p) {
    DV_TRY(check_problem(&probs[p], "qe_davidson_batch"));
    if (probs[p].mem != QE_DEVICE) {
      set_error("qe_davidson_batch: problem %d: arrays must be device memory", p);
      return QE_EINVAL;
    }
    if (probs[p].nbnd > 0 && (!psi_inout[p] || !evals[p])) {
      set_error("qe_davidson_batch: problem %d: null psi/evals", p);
      return QE_EINVAL;
    }
    if (iters) iters[p] = 0;
    if (status) status[p] = QE_OK;
  }
  if (nprob == 0) return QE_OK;
  DV_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DV_TRY(ctx_begin(ctx, st));
  // one lockstep task per solve with bands; the Rayleigh-Ritz steps of a round
  // run on the context's side streams, so that the dense eigensolvers of
  // different solves overlap
  constexpr int kSide = 8;
  if (ctx->round_side.empty()) {
    for (int i = 0; i < kSide; ++i) {
      cudaStream_t x = nullptr;
      DV_CU(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      ctx->round_side.push_back(x);
    }
    for (int i = 0; i <= kSide; ++i) {
      cudaEvent_t e = nullptr;
      DV_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ctx->round_events.push_back(e);
    }
  }
  std::vector<int> ids;
  std::vector<DvTask*> tasks;
  auto cleanup = [&] {
    for (DvTask* t : tasks) dv_task_destroy(t, st);
    tasks.clear();
  };
  int worst = QE_OK;
  for (int p = 0; p < nprob; ++p) {
    if (probs[p].nbnd <= 0) continue;
    DvTask* t = nullptr;
    const int rc = dv_task_create(ctx, &probs[p], precision | flags, tol, max_iter, max_dim,
                                  psi_inout[p], st, &t);
    if (rc) { cleanup(); return rc; }
    ids.push_back(p);
    tasks.push_back(t);
  }
  while (true) {
    std::vector<DvTask*> live;
    for (DvTask* t : tasks)
      if (!dv_task_done(t)) live.push_back(t);
    if (live.empty()) break;
    const int rc = dv_round(ctx, live.data(), (int)live.size(), st, ctx->round_side.data(),
                            (int)ctx->round_side.size(), ctx->round_events.data());
    if (rc) { cleanup(); return rc; }
  }
  for (size_t i = 0; i < tasks.size(); ++i) {
    const int p = ids[i];
    int it = 0;
    const int rc = dv_task_result(ctx, tasks[i], psi_inout[p], evals[p], resid ? resid[p] : nullptr,
                                  &it, true, st);
    if (iters) iters[p] = it;
    if (status) status[p] = rc;
    if (rc != QE_OK && (worst == QE_OK || worst == QE_ENOCONV)) worst = rc;
  }
  cleanup();
  DV_TRY(tc_check(ctx, st));
  if (worst == QE_ENOCONV) set_error("qe_davidson_batch: some problems did not converge");
  return worst;
}

extern "C" int qe_cg(qe_ctx* ctx, const qe_problem* prob, int precision, double tol, int max_iter,
                     int max_sweeps, double* psi_inout, double* evals, double* resid, int* iters,
                     void* stream) {
  clear_error();
  if (!ctx) { set_error("qe_cg: null context"); return QE_EINVAL; }
  DV_TRY(check_problem(prob, "qe_cg"));
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_cg: bad precision"); return QE_EINVAL; }
  if (!(tol > 0.0) || max_iter < 1 || max_sweeps < 0) {
    set_error("qe_cg: tol must be > 0, max_iter >= 1, max_sweeps >= 0");
    return QE_EINVAL;
  }
  const int nb = prob->nbnd;
  if (iters) *iters = 0;
  if (nb == 0) return QE_OK;
  if (!psi_inout || !evals) { set_error("qe_cg: null psi/evals"); return QE_EINVAL; }
  DV_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DV_TRY(ctx_begin(ctx, st));
  DvSolve v;
  // four scratch vectors past the bands in V and in HV
  DV_TRY(dv_setup(ctx, prob, precision, tol, max_iter, std::max(default_max_dim(nb), nb + 4),
                  ctx->dv_basis, ctx->dv_red, v, st, "qe_cg", false));
  DvState& S = v.S;
  S.vcache = nullptr;   // the CG keeps scratch rows in V past the bands: no kept slices
  if (S.max_dim < nb + 4) { set_error("qe_cg: %d bands need more plane waves", nb); return QE_EINVAL; }
  const size_t bytes = (size_t)nb * S.npw * sizeof(z);
  const cudaMemcpyKind in_kind = prob->mem == QE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind out_kind = prob->mem == QE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  DV_CU(cudaMemcpyAsync(S.V, psi_inout, bytes, in_kind, st));
  S.vrows = 0;   // V rewritten: its kept slices are stale
  CgRun run;
  const int rc = cg_run(ctx, v, tol, max_iter, max_sweeps, run, st);
  if (iters) *iters = run.iters;
  if (rc) return rc;
  DV_CU(cudaMemcpyAsync(psi_inout, S.Psi, bytes, out_kind, st));
  DV_CU(cudaMemcpyAsync(evals, S.e, nb * sizeof(double), out_kind, st));
  if (resid) DV_CU(cudaMemcpyAsync(resid, S.rn, nb * sizeof(double), out_kind, st));
  DV_TRY(dv_final_status(v, st, "qe_cg"));
  DV_TRY(tc_check(ctx, st));
  if (!run.conv) {
    set_error("qe_cg: not converged after %d sweeps", run.sweeps);
    return QE_ENOCONV;
  }
  return QE_OK;
}
