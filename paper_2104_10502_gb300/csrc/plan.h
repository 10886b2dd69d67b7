// Device-resident plan of one (lattice, k, cut-off, grid) and the kernel
// launchers that use it.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include <type_traits>

#include "common.h"
#include "fft_device.cuh"

namespace qe {

// Element type of the FP64 path's FFT: float-float pairs on the FP32 pipes
// (ff.cuh; FP64-accurate, ~2^-48 per operation); `double` runs it on the FP64
// pipe instead (QE_FFT_FP64PIPE).
using FftF64 = ff;
// Type of the SIMT projector products that go with an FFT element type.
template <typename T>
using GemmT = std::conditional_t<std::is_same<T, float>::value, float, double>;

// Plane size with a register-resident two-pass transform (plane2.cuh), or 0.
int sq_plane_size(const int grid[3]);
// n when lines of n points have the register-resident two-pass transform, else 0
int sq_line_size(int n);
// perm[p] = natural index held at line position p of that transform of length n.
std::vector<int> sq_order(int n);

struct DevPlan {
  double lat[9], k[3], ecut;
  int grid[3];
  int sq = 0;   // sq_plane_size(grid): x and y perms are sq_order(n) when non-zero
  int sqz = 0;  // sq_line_size(grid[2]): the z perm is sq_order(n) when non-zero
  PlanHost h;
  Radix rad[3];
  // device arrays (one allocation)
  void* block = nullptr;
  double* kin = nullptr;    // [npw]
  int* st_ptr = nullptr;    // [nst+1]
  int* st_g = nullptr;      // [npw]
  int* st_z = nullptr;      // [npw]
  int* st_of = nullptr;     // [npw]
  int* st_x = nullptr;      // [nst]
  int* st_y = nullptr;      // [nst]
  int* ax = nullptr;        // [nax]
  int* mg = nullptr;        // [npw] sphere index of -G (k = 0 plans only, else null)
  int* perm[3] = {nullptr, nullptr, nullptr};   // digit reversal per axis
  double* tw[3] = {nullptr, nullptr, nullptr};  // exp(-2 pi i t / N_axis), interleaved,
                                                // then as (cos, tan) (twiddles())
};

// Raise a kernel's dynamic shared-memory cap to the device's opt-in maximum
// minus its static shared memory.  Always the same value for a kernel, so
// concurrent host threads never lower it under each other's launch.
template <typename F>
inline void set_max_dynamic_smem(F* f) {
  int dev = 0, optin = 0;
  cudaFuncAttributes a;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(f)) != cudaSuccess)
    return;
  cudaFuncSetAttribute(reinterpret_cast<const void*>(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                       optin - (int)a.sharedSizeBytes);
}

// Optional per-kernel timing: CUDA events recorded on the launching stream
// around each kernel, folded into per-name totals on read.  Also counts
// launches (always, even when timing is off).
struct Prof {
  bool on = false;
  std::atomic<long long> launches{0};
  std::mutex mu;   // recs: the lockstep rounds record from several host threads
  struct Rec { const char* name; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<std::string> names;
  std::vector<long long> calls;
  std::vector<double> ms;
  void begin(const char* name, cudaStream_t st, cudaEvent_t* ev);
  void end(const char* name, cudaStream_t st, cudaEvent_t ev);
  int fold();   // synchronises on the recorded events
  void reset();
};
struct ProfScope {
  Prof* p; const char* name; cudaStream_t st; cudaEvent_t a = nullptr;
  ProfScope(Prof* p_, const char* n, cudaStream_t s) : p(p_), name(n), st(s) {
    if (p) p->begin(name, st, &a);
  }
  ~ProfScope() { if (p) p->end(name, st, a); }
};

// Grow-only device buffer, allocated and freed stream-ordered (cudaMallocAsync /
// cudaFreeAsync) on the owning context's current stream, so that growing or
// releasing it never synchronises the whole device.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  const cudaStream_t* sp = nullptr;   // owner's current stream
  int ensure(size_t nbytes);
  void release();
};

// ---- FFT stage descriptors ---------------------------------------------------------
// Launch shape of the FFT kernels for one grid: sticks per CTA of the z stages
// and threads per CTA of the z and plane stages (0 = default).  Any shape gives
// bit-identical results; the autotuner only picks the fastest.
struct FftShape {
  int spb = 0, zthreads = 0, pthreads = 0;
};
// Tuned shape for this plan's grid at this element size (defaults if untuned).
FftShape tuned_shape(const DevPlan& P, size_t elem_bytes);

// One problem's share of the local + kinetic stages: plan, operands, bands.
template <typename T>
struct FftJob {
  Radix r1, r2, r3;
  const int *st_ptr, *st_g, *st_z, *st_of, *st_x, *st_y, *ax;
  const double *tw1, *tw2, *tw3, *kin;
  // digit reversal per axis, and whether the transforms of an axis may drop the
  // padding outside [0, K] + [N - K, N) in their stage of span N (zero input of
  // the first inverse stage, unread output of the last forward stage; radix 4
  // first, 4K < N)
  const int *pm1, *pm2, *pm3;
  int pr1, pr2, pr3;
  const double* psi;
  double* hpsi;
  const T* vp;
  cx<T>* W;
  int nst, nax, npw, nb, b0, spb, nsb, stage_v;   // stage_v: V plane staged in shared memory
  // pair: FFT band b carries the real-space-real bands 2b and 2b+1 of the
  // job's nbr bands as psi_2b + i psi_2b+1 (k = 0; sticks in mirror pairs);
  // self_st: the self-mirror stick
  int pair, nbr, self_st;
  // sq: N when the planes are N x N with a register-resident two-pass plane
  // transform (plane2.cuh; x and y in its order, the plan's perm[0], perm[1]),
  // 0 for the stage-by-stage transform; sqz: the same for the z lines of the
  // sticks (z in its order, the plan's perm[2])
  int sq, sqz;
  double inv_n;
};

// pair != 0 on a k = 0 plan: bands taken two per FFT (they must be real in r,
// psi(-G) = conj psi(G); the result is H applied to that part of each band).
template <typename T>
FftJob<T> make_job(const DevPlan& P, const double* psi, double* hpsi, const T* vp, void* W, int b0,
                   int nb, const FftShape& sh, int pair = 0);
template <typename T>
int default_spb(int n3);   // sticks per z tile of the stage-by-stage z lines
template <typename T>
size_t zsm_bytes(int n3, int spb);
template <typename T>
size_t psm_bytes(const DevPlan& P);

// ---- launchers (return QE_OK or QE_ECUDA with the error message set) -------
// Vp[pz][py][px] = V[perm3[pz]][perm2[py]][perm1[px]] converted to T.
template <typename T>
int launch_vperm(const DevPlan& P, const double* vloc, T* vp, cudaStream_t st, Prof* pf);

// hpsi[b] = |k+G|^2 psi[b] + V_loc psi[b] for bands b0 .. b0+nbc-1.
// W: stick workspace of nbc * N3 * nst complex T (ceil(nbc / 2) * N3 * nst
// with pair, as make_job).
template <typename T>
int launch_local_kinetic(const DevPlan& P, const double* psi, double* hpsi, const T* vp,
                         void* W, int b0, int nbc, cudaStream_t st, Prof* pf, int pair = 0);

template <typename T>
int launch_local_kinetic_shape(const DevPlan& P, const double* psi, double* hpsi, const T* vp,
                               void* W, int b0, int nbc, const FftShape& sh, cudaStream_t st,
                               Prof* pf, int pair = 0);
template <typename T>
int launch_local_kinetic_batch(const FftJob<T>* jobs_dev, const int* prefix_dev, int njobs,
                               int* counters, size_t smem_z, size_t smem_p, int threads,
                               int zthreads, cudaStream_t st, Prof* pf);

// Charge density (sum of w |psi(r)|^2): bands b0 .. b0+nbc-1 of psi with device
// weights w[b] into the group accumulators acc [ngrp][N3][N2][N1] (digit-reversed
// positions; zeroed by the caller before the first launch); W as for
// launch_local_kinetic.  launch_density_finish writes rho [N3][N2][N1] (natural
// order) = scale * the sum of the groups.
// mode 1: acc += w Re psi(r) instead (the inverse transform of the bands to the grid).
template <typename T>
int launch_density(const DevPlan& P, const double* psi, const double* w, void* W, int b0, int nbc,
                   int ngrp, double* acc, cudaStream_t st, Prof* pf, int pair = 0, int mode = 0);
int launch_density_finish(const DevPlan& P, const double* acc, int ngrp, double scale, double* rho,
                          cudaStream_t st, Prof* pf);

// Size in bytes of the stick workspace for nbc bands.
size_t stick_bytes(const DevPlan& P, int nbc, size_t elem_bytes);

// ---- complex GEMMs (all matrices complex, interleaved doubles in memory) -----
// Split-K inner products: P[m][n] = sum_k conj(A[m][k]) B[n][k]; A [M][lda],
// B [N][ldb]; result written to C (double complex, [M][ldc]; real_out: Im C = 0).
// `part` is a scratch of gemm_inner_scratch(M, N, K) bytes.
template <typename T>
int gemm_inner(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
               double* C, int ldc, void* part, size_t part_bytes, cudaStream_t st, Prof* pf,
               bool real_out = false);
size_t gemm_inner_scratch(int M, int N, int K, size_t elem_bytes);
// As gemm_inner, with as many K splits as fit in part_bytes (>= 1).
template <typename T>
int gemm_inner_bounded(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                       double* C, int ldc, void* part, size_t part_bytes, cudaStream_t st, Prof* pf);

// C[n][m] = beta * C[n][m] + sum_k A[k][m] B[k][n]; A [K][lda], B [K][ldb],
// C [N][ldc]; beta in {0, 1}.
template <typename T>
int gemm_outer(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
               double* C, int ldc, int beta, cudaStream_t st, Prof* pf);

// C[n][m] = beta * C[n][m] + (alpha_neg ? -1 : 1) * sum_k A[k][m] B[k][n]
template <typename T>
int gemm_outer_ab(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                  double* C, int ldc, int alpha_neg, int beta, cudaStream_t st, Prof* pf);

// ---- tensor-core (tcgen05, TF32x3) path of the mixed-precision nonlocal term ----
// Real split-precision GEMM on padded K-major operands (tcgemm.cu).
int tc_gemm_tf32x3(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int Mp,
                   int Np, int Kp, int nsplit, float* C, int* status, cudaStream_t st, Prof* pf);
int tc_gemm_splits(int Mp, int Np, int Kp);
// General complex products on the tensor cores, FP32-accurate (TF32 x3), for the
// mixed path: inner C[m][n] = sum_k conj(A[m][k]) B[n][k] (A, B rows of length
// K, contiguous); outer C[n][m] (+)= (-) sum_k A[k][m] B[k][n] (A [K][M], B
// [K][N] dense).  Work of tc_*_bytes(); a bounded wait that ran out writes a
// non-zero code to *status.
size_t tc_inner_bytes(int M, int N, int K);
size_t tc_outer_bytes(int M, int N, int K);
// real_out: only Re C, written as (Re C, 0) (the k = 0 real-in-r products), with
// half the GEMM columns.
int tc_inner(const double* A, const double* B, int M, int N, int K, double* C, int ldc, void* work,
             size_t work_bytes, int* status, cudaStream_t st, Prof* pf, bool real_out = false);
int tc_outer(const double* A, const double* B, int M, int N, int K, double* C, int ldc,
             int alpha_neg, int beta, void* work, size_t work_bytes, int* status, cudaStream_t st,
             Prof* pf);
// tc_outer for a real-valued B (zero imaginary parts; the k = 0 mode's Ritz
// vectors and Gram blocks): half the tensor-core work; work of tc_outer_real_bytes().
size_t tc_outer_real_bytes(int M, int N, int K);
int tc_outer_real(const double* A, const double* B, int M, int N, int K, double* C, int ldc,
                  int alpha_neg, int beta, void* work, size_t work_bytes, int* status,
                  cudaStream_t st, Prof* pf);
// hpsi += beta^T D (conj(beta) psi^T) on the tensor cores; work of nonlocal_tc_bytes().
size_t nonlocal_tc_bytes(int np, int nb, int npw);
size_t nonlocal_tc_beta_bytes(int np, int npw);
int nonlocal_tc(const double* beta, const double* dmat, const double* psi, double* hpsi, int np,
                int nb, int npw, void* bpack, bool pack_beta, void* work, size_t work_bytes,
                int* status, cudaStream_t st, Prof* pf, bool real_p = false);

// Q[i][n] = sum_j D[i][j] P[j][n] (D real [np][np], P complex [np][nb]).
// Q = D P (D real [np][np], P complex [np][nb]); real_p: Q = D Re(P) (bands real in r
// with real projectors at k = 0, where P is real up to rounding).
int dmul(const double* D, const double* P, double* Q, int np, int nb, cudaStream_t st, Prof* pf,
         bool real_p = false);

// ---- projectors generated on the fly (betagen.cu) ------------------------------
// beta_{I,n,c}(G) = e^{-i q.R_I} (-i)^{l_n} Y_{l_n c}(q) F_n(G), q = k + G, with
// the structure factor from per-atom, per-axis phase tables (the separable
// e^{-iG.R_I} = prod_c e^{-i 2 pi m_c f_Ic}) times e^{-i k.R_I}, the real solid
// harmonic Y_00 = 1/(2 sqrt pi), Y_1c = sqrt(3/4pi) q_c, and the caller's radial
// table F_n(G).  Projector order: atom-major; per atom, per radial function n
// its 2 l_n + 1 components.
constexpr int kGenMaxRad = 8;
struct GenProj {
  int natom = 0, nper = 0, nrad = 0, npw = 0, np = 0;
  const int* mill = nullptr;        // [npw][3] signed Miller indices of the sphere
  const double* tab = nullptr;      // phase tables, complex: atom I, axis c, m in [-half_c, half_c]
  int toff[3] = {0, 0, 0}, half[3] = {0, 0, 0}, tstride = 0;
  const double* ekr = nullptr;      // [natom] complex e^{-i k.R_I}
  const double* radial = nullptr;   // [nrad][npw] F_n(G)
  int l[kGenMaxRad] = {}, off[kGenMaxRad] = {};
  double b[9] = {}, k[3] = {};
};
// The two Ozaki slicings of the generated beta (rows for the inner product,
// columns for the outer one) into bslices (nonlocal_oz_beta_bytes), as
// nonlocal_oz's own slicing of a stored beta would lay them out; form4: the
// columns as separate real and imaginary rows (the k = 0 band-pair products,
// nonlocal_oz_real_outer).
int oz_gen_beta(const GenProj& g, void* bslices, void* scratch, cudaStream_t st, Prof* pf,
                bool form4 = false);
// Bytes of oz_gen_beta's scratch (the exponent bounds).
size_t oz_gen_scratch_bytes(const GenProj& g);
// The generated beta as values, complex [np][npw] (the SIMT and TF32 paths).
int gen_beta_values(const GenProj& g, double* beta, cudaStream_t st, Prof* pf);

// hpsi += beta^T D (conj(beta) psi^T) with FP64-accurate products on the BF16
// tensor cores (ozgemm.cu); beta slices in bslices (nonlocal_oz_beta_bytes),
// work of nonlocal_oz_bytes().
size_t nonlocal_oz_bytes(int np, int nb, int npw);
size_t nonlocal_oz_beta_bytes(int np, int npw);
// Whether nonlocal_oz with real_p keeps beta's column slices in the real-K form
// (a real Q = D Re P: half the outer product's work); the kept slices of one
// form do not serve the other.
bool nonlocal_oz_real_outer(bool real_p, int np);
int nonlocal_oz(const double* beta, const double* dmat, const double* psi, double* hpsi, int np,
                int nb, int npw, void* bslices, bool slice_beta, void* work, size_t work_bytes,
                int* status, cudaStream_t st, Prof* pf, bool real_p = false);
// FP64 complex products on the tensor cores (default) or on the DFMA pipe
// (environment QE_FP64_GEMM=simt).
bool fp64_gemm_on_tensor_cores();
// ... and large enough for them to pay (M N K >= 2^22 complex multiply-adds).
bool oz_worth(long long M, long long N, long long K);
// General FP64-accurate complex products on the tensor cores (ozgemm.cu), with
// the semantics of gemm_inner / gemm_outer_ab; scratch of oz_*_scratch bytes;
// a bounded wait that ran out writes a non-zero code to *status.
size_t oz_inner_scratch(int M, int N, int K);
size_t oz_outer_scratch(int M, int N, int K);
// real: C = (Re of the inner product, 0), half the tensor-core work.
int oz_inner(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
             int ldc, void* scratch, size_t scratch_bytes, int* status, cudaStream_t st, Prof* pf,
             bool real = false);
int oz_outer(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
             int ldc, int alpha_neg, int beta, void* scratch, size_t scratch_bytes, int* status,
             cudaStream_t st, Prof* pf);
// Row slices of an append-only matrix kept across products (the Davidson
// basis): oz_cache_rows slices rows [r0, r1) into `mem` (oz_cache_bytes);
// oz_inner_cached is oz_inner with A = the first M kept rows.
size_t oz_cache_bytes(int rows_cap, int K);
int oz_cache_rows(const double* src, int ld, int r0, int r1, int K, int rows_cap, void* mem,
                  cudaStream_t st, Prof* pf);
size_t oz_inner_cached_scratch(int M, int N, int K);
int oz_inner_cached(const void* mem, int rows_cap, int M, const double* B, int ldb, int N, int K,
                    double* C, int ldc, void* scratch, size_t scratch_bytes, int* status,
                    cudaStream_t st, Prof* pf, bool real = false);
// oz_outer with a real B (imaginary parts ignored): half the tensor-core work.
size_t oz_outer_real_scratch(int M, int N, int K);
int oz_outer_real(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                  double* C, int ldc, int alpha_neg, int beta, void* scratch, size_t scratch_bytes,
                  int* status, cudaStream_t st, Prof* pf);

}  // namespace qe
