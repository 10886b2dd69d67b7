// Local-potential and kinetic part of H|psi> (Sec. 3.3 of the paper: the
// local-potential and kinetic-energy contributions; FFTXlib of Sec. 3.2.1):
//
//   psi(r_j) = sum_G c_G e^{iG.r_j},   (H c)_G = |k+G|^2 c_G + (1/N) sum_j e^{-iG.r_j} V(r_j) psi(r_j)
//
// as a pruned 3D FFT in three stages per block of bands:
//   zinv   scatter the sphere onto its sticks (x, y columns) and run the
//          inverse z transform of each stick (DIF, z left digit-reversed);
//   plane  one CTA per (z plane, band): scatter the sticks into the plane,
//          inverse y transform of the columns that hold sticks, inverse x
//          transform of every row, multiply by V (read through the digit
//          reversal), forward x and y transforms (DIT), gather the sticks;
//   zfwd   forward z transform of each stick (DIT, natural order out),
//          gather onto the sphere, scale by 1/N and add |k+G|^2 c_G.
// Sticks live in a workspace laid out [band][z][stick] so that every kernel
// reads and writes it with consecutive threads on consecutive sticks.
//
// Each stage is a device "tile" function driven by a job descriptor (one
// problem: plan, operands, band range).  A single problem launches the tiles
// as a grid; a batch of problems with different cells, grids, plane-wave
// counts and band counts runs each stage as ONE persistent launch whose CTAs
// pull (problem, band, tile) items from an atomic work counter.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fft_device.cuh"
#include "plan.h"
#include "plane2.cuh"

namespace qe {

static int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

// Twiddle table slots per entry in a tile's shared memory: float-float entries
// take two elements (the (c, c) and (-t, t) pairs, fft_device.cuh), others one
// (c, t) or w.
template <typename T>
__host__ __device__ constexpr int tw_slots() { return std::is_same<T, ff>::value ? 2 : 1; }
template <typename T>
__device__ __forceinline__ void tw_put(cx<T>* tw, int i, double a, double b) {
  if constexpr (std::is_same<T, ff>::value) {
    const ff c(a), t(b);
    tw[2 * i] = {f2_of(c.hi, c.hi), f2_of(c.lo, c.lo)};
    tw[2 * i + 1] = {f2_of(-t.hi, t.hi), f2_of(-t.lo, t.lo)};
  } else {
    tw[i] = {T(a), T(b)};
  }
}

template <typename T>
__global__ void k_vperm(const double* __restrict__ v, T* __restrict__ vp, int n1, int n2, int n3,
                        const int* __restrict__ p1, const int* __restrict__ p2,
                        const int* __restrict__ p3) {
  const size_t total = (size_t)n1 * n2 * n3;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int px = (int)(i % n1);
    const int py = (int)((i / n1) % n2);
    const int pz = (int)(i / ((size_t)n1 * n2));
    vp[i] = T(v[((size_t)p3[pz] * n2 + p2[py]) * n1 + p1[px]]);
  }
}

// ---- tiles ----------------------------------------------------------------------
// z lines with the register-resident two-pass transform (plane2.cuh): stick l
// of the tile is the line at line + l with element stride spb; consecutive
// threads take consecutive sticks.  Each ends with a barrier.
template <typename T, int N>
__device__ __forceinline__ void sq_z_inverse(const FftJob<T>& J, cx<T>* line, int spb, int ns,
                                             const cx<T>* tab) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B;
  const FastDiv fns(ns);
  for (int it = threadIdx.x; it < ns * B; it += blockDim.x) {
    const int n2 = fns.div(it), l = it - n2 * ns;
    if (J.pr3) sq_inv1<T, N, true>(line + l, spb, n2, tab);
    else sq_inv1<T, N, false>(line + l, spb, n2, tab);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ns * A; it += blockDim.x) {
    const int k1 = fns.div(it), l = it - k1 * ns;
    cx<T>* p = line + l;
    cx<T> o[B];
    sq_inv2_regs<T, N>(p, spb, k1, tab, o);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) p[(B * k1 + k2) * spb] = o[k2];
  }
  __syncthreads();
}

template <typename T, int N>
__device__ __forceinline__ void sq_z_forward(const FftJob<T>& J, cx<T>* line, int spb, int ns,
                                             const cx<T>* tab) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B;
  const FastDiv fns(ns);
  for (int it = threadIdx.x; it < ns * A; it += blockDim.x) {
    const int k1 = fns.div(it), l = it - k1 * ns;
    cx<T>* p = line + l;
    cx<T> in[B], f[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) in[k2] = p[(B * k1 + k2) * spb];
    sq_fwd1_regs<T, N>(in, k1, tab, f);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) p[(B * k1 + m2) * spb] = f[m2];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ns * B; it += blockDim.x) {
    const int m2 = fns.div(it), l = it - m2 * ns;
    if (J.pr3) sq_fwd2<T, N, true>(line + l, spb, m2, tab);
    else sq_fwd2<T, N, false>(line + l, spb, m2, tab);
  }
  __syncthreads();
}

#define QE_SQZ_DISPATCH(CALL) \
  switch (J.sqz) {            \
    case 96: CALL(96); break; \
    case 48: CALL(48); break; \
    case 32: CALL(32); break; \
    default: break;           \
  }

template <typename T>
__device__ void zinv_tile(const FftJob<T>& J, int b, int sblk, unsigned char* smem) {
  cx<T>* line = reinterpret_cast<cx<T>*>(smem);
  const int n3 = J.r3.n, spb = J.spb, nst = J.nst;
  cx<T>* tw = line + (size_t)n3 * spb;
  const int s0 = sblk * spb;
  const int ns = min(spb, nst - s0);
  for (int i = threadIdx.x; i < n3 * spb; i += blockDim.x) line[i] = cx_zero<T>();
  if (J.sqz) {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sq_tw_put<T>(tw, i, J.tw3[2 * i], J.tw3[2 * i + 1]);
  } else {
    const double* tw3 = J.tw3 + (ct_twiddles<T>() ? 2 * n3 : 0);
    for (int i = threadIdx.x; i < n3; i += blockDim.x) tw_put<T>(tw, i, tw3[2 * i], tw3[2 * i + 1]);
  }
  __syncthreads();
  const int e0 = J.st_ptr[s0], e1 = J.st_ptr[s0 + ns];
  if (J.pair) {
    // bands 2b and 2b+1 (real in r) as one complex band psi_2b + i psi_2b+1
    const double2* pa = reinterpret_cast<const double2*>(J.psi) + (size_t)(J.b0 + 2 * b) * J.npw;
    const bool hb = 2 * b + 1 < J.nbr;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int g = J.st_g[e];
      const double2 a = pa[g];
      const double2 c = hb ? pa[(size_t)J.npw + g] : make_double2(0.0, 0.0);
      line[J.st_z[e] * spb + (J.st_of[e] - s0)] = cx_from<T>(a.x - c.y, a.y + c.x);
    }
  } else {
    const double2* ps = reinterpret_cast<const double2*>(J.psi) + (size_t)(J.b0 + b) * J.npw;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const double2 c = ps[J.st_g[e]];
      line[J.st_z[e] * spb + (J.st_of[e] - s0)] = cx_from<T>(c.x, c.y);
    }
  }
  __syncthreads();
  if (J.sqz) {
#define QE_SQZ_INV(n) sq_z_inverse<T, n>(J, line, spb, ns, tw)
    QE_SQZ_DISPATCH(QE_SQZ_INV)
#undef QE_SQZ_INV
  } else {
    fft_lines<T, +1, false>(line, spb, 1, nullptr, ns, true, J.r3, tw, J.pm3, J.pr3);
  }
  cx<T>* Wb = J.W + (size_t)b * n3 * nst;
  const FastDiv fns(ns);
  for (int i = threadIdx.x; i < n3 * ns; i += blockDim.x) {
    const int pz = fns.div(i), l = i - pz * ns;
    Wb[(size_t)pz * nst + s0 + l] = line[pz * spb + l];
  }
}

// The plane stage fuses radix stages in pairs in single precision (its FP32
// butterflies are issue-bound); in FP64 the kernel is bound by the FP64 pipe
// itself and fusing measured slower (15.8 against 15.2 ms per C1 call).
template <typename T>
constexpr bool kFusePlane = sizeof(T) == 4;

// Launch bounds of the plane stage.  FP32: two CTAs of 256 threads per SM and
// up to 128 registers for the fused stage pairs (capping registers for a third
// CTA makes the fused butterflies spill).
template <typename T> struct PlaneLB { static constexpr int threads = 512, minb = 1, dflt = 256; };
template <> struct PlaneLB<float> { static constexpr int threads = 256, minb = 2, dflt = 256; };
// float-float planes: 16 warps per SM (one CTA) hide the dependent FP32 chains of
// the float-float operations better than 8
template <> struct PlaneLB<ff> { static constexpr int threads = 512, minb = 1, dflt = 512; };

// Row stride of a plane in shared memory: odd, so that the lines of one pass that
// consecutive threads take (rows in the x pass, columns in the y pass) fall in
// different banks.
__host__ __device__ inline int plane_ld(int n1) { return n1 | 1; }

// FP32 planes also stage their V_loc plane in shared memory with cp.async,
// issued first and waited for only before the multiply, so that its L2 latency
// hides behind the inverse transforms -- when two CTAs per SM still fit (FP64
// planes are FP64-pipe bound and their shared memory is full).
template <typename T>
constexpr bool kStageV = sizeof(T) == 4;
constexpr size_t kStageVMaxBytes = 113 * 1024;

// Byte offset of the staged V plane: after the plane, the twiddles and the
// active-column table, rounded up to 16 bytes.
template <typename T>
__host__ __device__ inline size_t plane_v_offset(int n1, int n2, int nax) {
  const size_t b = ((size_t)plane_ld(n1) * n2 + (size_t)(n1 + n2) * tw_slots<T>()) * sizeof(cx<T>) +
                   (size_t)nax * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- square planes with the register-resident two-pass transform (plane2.cuh) ----------
// Shared memory: the plane (row stride N | 1), the twiddle table of length N,
// the active-column table.
// With the padding skipped along both axes (pr1 and pr2), the inverse passes
// read only the columns and rows outside [N/4, 3N/4) before anything writes
// there: the y pass reads the outer rows of the active columns, the x pass the
// outer columns of every row after the y pass has filled the active columns --
// so only the outer columns of every row need zeros (half the plane).
template <typename T, int N>
__device__ __forceinline__ void sq_setup(const FftJob<T>& J, cx<T>* plane, cx<T>* tab, int* ax) {
  constexpr int ld = N | 1, Q = N / 4, W = N - 2 * Q;   // outer columns: [0, Q) and [N - Q, N)
  if (J.pr1 && J.pr2) {
    for (int i = threadIdx.x; i < 2 * Q * N; i += blockDim.x) {
      const int y = i / (2 * Q), c = i - y * (2 * Q);
      plane[y * ld + (c < Q ? c : c + W)] = cx_zero<T>();
    }
  } else {
    for (int i = threadIdx.x; i < ld * N; i += blockDim.x) plane[i] = cx_zero<T>();
  }
  for (int t = threadIdx.x; t < N; t += blockDim.x) sq_tw_put<T>(tab, t, J.tw1[2 * t], J.tw1[2 * t + 1]);
  for (int i = threadIdx.x; i < J.nax; i += blockDim.x) ax[i] = J.ax[i];
}

// Inverse y transforms of the active columns (sticks scattered beforehand);
// ends with a barrier.
template <typename T, int N>
__device__ __forceinline__ void sq_inverse_y(const FftJob<T>& J, cx<T>* plane, const cx<T>* tab,
                                             const int* ax) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B, ld = N | 1;
  const int nax = J.nax, nt = blockDim.x;
  const FastDiv fax(nax);
  for (int it = threadIdx.x; it < nax * B; it += nt) {
    const int n2 = fax.div(it), l = it - n2 * nax;
    if (J.pr2) sq_inv1<T, N, true>(plane + ax[l], ld, n2, tab);
    else sq_inv1<T, N, false>(plane + ax[l], ld, n2, tab);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nax * A; it += nt) {
    const int k1 = fax.div(it), l = it - k1 * nax;
    cx<T>* p = plane + ax[l];
    cx<T> o[B];
    sq_inv2_regs<T, N>(p, ld, k1, tab, o);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) p[(B * k1 + k2) * ld] = o[k2];
  }
  __syncthreads();
}

// The above, then the inverse x pass 1 of every row; ends with a barrier.
template <typename T, int N>
__device__ __forceinline__ void sq_inverse_yx1(const FftJob<T>& J, cx<T>* plane, const cx<T>* tab,
                                               const int* ax) {
  constexpr int B = SqSplit<N>::B, ld = N | 1;
  const int nt = blockDim.x;
  sq_inverse_y<T, N>(J, plane, tab, ax);
  const FastDiv fn(N);
  for (int it = threadIdx.x; it < N * B; it += nt) {
    const int n2 = fn.div(it), y = it - n2 * N;
    if (J.pr1) sq_inv1<T, N, true>(plane + y * ld, 1, n2, tab);
    else sq_inv1<T, N, false>(plane + y * ld, 1, n2, tab);
  }
  __syncthreads();
}

// The x step of a plane pair with rows owned by warps: inverse pass 1, then
// inverse pass 2 x V x forward pass 1, then forward pass 2, each row's three
// phases in one warp, so that only __syncwarp separates them (no block barrier,
// no warp waiting for the slowest row of the plane).  Lane j of a round takes
// row y0 + j mod R: with 16-byte elements and the odd row stride the lanes of
// one access spread over all banks.  R = N / warps rows per warp.
template <typename T, int N>
__device__ __forceinline__ void sq_x_step_warp_rows(const FftJob<T>& J, cx<T>* plane, const cx<T>* tab,
                                                    const T* vz, int R, const FastDiv& fR) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B, ld = N | 1;
  const int lane = threadIdx.x & 31, y0 = (threadIdx.x >> 5) * R;
  for (int it = lane; it < R * B; it += 32) {
    const int n2 = fR.div(it), y = y0 + (it - n2 * R);
    if (J.pr1) sq_inv1<T, N, true>(plane + y * ld, 1, n2, tab);
    else sq_inv1<T, N, false>(plane + y * ld, 1, n2, tab);
  }
  __syncwarp();
  for (int it = lane; it < R * A; it += 32) {
    const int k1 = fR.div(it), y = y0 + (it - k1 * R);
    cx<T>* p = plane + y * ld;
    const T* vr = vz + (size_t)y * N + B * k1;
    T vv[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) vv[k2] = vr[k2];
    cx<T> o[B], f[B];
    sq_inv2_regs<T, N>(p, 1, k1, tab, o);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) o[k2] = cscale(o[k2], vv[k2]);
    sq_fwd1_regs<T, N>(o, k1, tab, f);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) p[B * k1 + m2] = f[m2];
  }
  __syncwarp();
  for (int it = lane; it < R * B; it += 32) {
    const int m2 = fR.div(it), y = y0 + (it - m2 * R);
    if (J.pr1) sq_fwd2<T, N, true>(plane + y * ld, 1, m2, tab);
    else sq_fwd2<T, N, false>(plane + y * ld, 1, m2, tab);
  }
  __syncthreads();
}

template <typename T, int N>
__device__ void plane_tile_sq(const FftJob<T>& J, int b, int pz, unsigned char* smem) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B, ld = N | 1;
  const int n3 = J.r3.n, nst = J.nst, nax = J.nax, nt = blockDim.x;
  cx<T>* plane = reinterpret_cast<cx<T>*>(smem);
  cx<T>* tab = plane + ld * N;
  int* ax = reinterpret_cast<int*>(tab + N * sq_tw_slots<T>());
  // V is read from L2 in the x step (staging it in shared memory with cp.async,
  // as the stage-by-stage FP32 plane does, measured slower here: 0.41 -> 0.45 ms
  // per 64-band C1 launch)
  const T* vz = J.vp + (size_t)pz * N * N;
  sq_setup<T, N>(J, plane, tab, ax);
  __syncthreads();
  cx<T>* Wp = J.W + ((size_t)b * n3 + pz) * nst;
  for (int s0 = threadIdx.x; s0 < nst; s0 += 4 * nt) {
    int off[4];
    cx<T> val[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * nt;
      if (s < nst) { off[u] = J.st_y[s] * ld + J.st_x[s]; val[u] = Wp[s]; }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (s0 + u * nt < nst) plane[off[u]] = val[u];
  }
  __syncthreads();
  const FastDiv fax(nax), fn(N);
  const int nw = nt >> 5;
  if (N % nw == 0) {
    // x rows owned by warps
    sq_inverse_y<T, N>(J, plane, tab, ax);
    const FastDiv fR(N / nw);
    sq_x_step_warp_rows<T, N>(J, plane, tab, vz, N / nw, fR);
  } else {
  sq_inverse_yx1<T, N>(J, plane, tab, ax);
  // x: inverse pass 2, times V, forward pass 1 on the same B values of a row
  for (int it = threadIdx.x; it < N * A; it += nt) {
    const int k1 = fn.div(it), y = it - k1 * N;
    cx<T>* p = plane + y * ld;
    const T* vr = vz + (size_t)y * N + B * k1;
    T vv[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) vv[k2] = vr[k2];
    cx<T> o[B], f[B];
    sq_inv2_regs<T, N>(p, 1, k1, tab, o);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) o[k2] = cscale(o[k2], vv[k2]);
    sq_fwd1_regs<T, N>(o, k1, tab, f);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) p[B * k1 + m2] = f[m2];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < N * B; it += nt) {
    const int m2 = fn.div(it), y = it - m2 * N;
    if (J.pr1) sq_fwd2<T, N, true>(plane + y * ld, 1, m2, tab);
    else sq_fwd2<T, N, false>(plane + y * ld, 1, m2, tab);
  }
  __syncthreads();
  }
  // y forward on the active columns
  for (int it = threadIdx.x; it < nax * A; it += nt) {
    const int k1 = fax.div(it), l = it - k1 * nax;
    cx<T>* p = plane + ax[l];
    cx<T> in[B], f[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) in[k2] = p[(B * k1 + k2) * ld];
    sq_fwd1_regs<T, N>(in, k1, tab, f);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) p[(B * k1 + m2) * ld] = f[m2];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nax * B; it += nt) {
    const int m2 = fax.div(it), l = it - m2 * nax;
    if (J.pr2) sq_fwd2<T, N, true>(plane + ax[l], ld, m2, tab);
    else sq_fwd2<T, N, false>(plane + ax[l], ld, m2, tab);
  }
  __syncthreads();
  for (int s0 = threadIdx.x; s0 < nst; s0 += 4 * nt) {
    int off[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * nt;
      if (s < nst) off[u] = J.st_y[s] * ld + J.st_x[s];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (s0 + u * nt < nst) Wp[s0 + u * nt] = plane[off[u]];
  }
}

// Sizes with a register-resident plane transform (plane2.cuh SqSplit).
#define QE_SQ_DISPATCH(CALL)                                  \
  switch (J.sq) {                                             \
    case 96: CALL(96); return;                                \
    case 48: CALL(48); return;                                \
    case 32: CALL(32); return;                                \
    default: break;                                           \
  }

// Launch bounds of the square-plane kernel.  FP32: at most 85 registers a
// thread (72 used: the register-resident passes hold one line's 8 or 12
// values), so that three CTAs of 256 threads (76 KB of shared memory each)
// share an SM -- 24 warps where the general plane kernel, at 123 registers,
// fits 16.  C1 mixed: 0.413 -> 0.381 ms per 68-band launch (384 threads:
// 0.393).
// Float-float and float64 planes: 384 threads (12 warps, 8 rows of the x step
// each: whole rounds of every pass; 0.644 -> 0.590 ms per 32-band C1 launch
// against 512 threads with block barriers between the x passes).
template <typename T> struct SqLB { static constexpr int threads = 512, minb = 1, dflt = 384; };
template <> struct SqLB<float> { static constexpr int threads = 384, minb = 2, dflt = 256; };

template <typename T, int N>
__global__ void __launch_bounds__(SqLB<T>::threads, SqLB<T>::minb) k_plane_sq(const FftJob<T> J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  plane_tile_sq<T, N>(J, blockIdx.y, blockIdx.x, smem_raw);
}

template <typename T>
__device__ void plane_tile(const FftJob<T>& J, int b, int pz, unsigned char* smem) {
#define QE_SQ_PLANE(n) plane_tile_sq<T, n>(J, b, pz, smem)
  QE_SQ_DISPATCH(QE_SQ_PLANE)
#undef QE_SQ_PLANE
  const int n1 = J.r1.n, n2 = J.r2.n, n3 = J.r3.n, nst = J.nst, nax = J.nax;
  const int ld = plane_ld(n1), nt = blockDim.x;
  cx<T>* plane = reinterpret_cast<cx<T>*>(smem);
  cx<T>* tw1 = plane + (size_t)ld * n2;
  cx<T>* tw2 = tw1 + (size_t)n1 * tw_slots<T>();
  int* ax = reinterpret_cast<int*>(tw2 + (size_t)n2 * tw_slots<T>());
  const T* v = J.vp + (size_t)pz * n1 * n2;
  T* sv = reinterpret_cast<T*>(smem + plane_v_offset<T>(n1, n2, nax));
  const bool stage = kStageV<T> && J.stage_v;
  if (stage) {
    const int nv = n1 * n2;
    if ((reinterpret_cast<size_t>(v) & 15) == 0) {
      const int n16 = nv / 4;
      for (int i = threadIdx.x; i < n16; i += nt) cp_async16(sv + 4 * i, v + 4 * i);
      for (int i = 4 * n16 + threadIdx.x; i < nv; i += nt) cp_async4(sv + i, v + i);
    } else {
      for (int i = threadIdx.x; i < nv; i += nt) cp_async4(sv + i, v + i);
    }
  }
  for (int i = threadIdx.x; i < ld * n2; i += nt) plane[i] = cx_zero<T>();
  {
    const double* t1 = J.tw1 + (ct_twiddles<T>() ? 2 * n1 : 0);
    const double* t2 = J.tw2 + (ct_twiddles<T>() ? 2 * n2 : 0);
    for (int i = threadIdx.x; i < n1; i += nt) tw_put<T>(tw1, i, t1[2 * i], t1[2 * i + 1]);
    for (int i = threadIdx.x; i < n2; i += nt) tw_put<T>(tw2, i, t2[2 * i], t2[2 * i + 1]);
  }
  for (int i = threadIdx.x; i < nax; i += nt) ax[i] = J.ax[i];
  __syncthreads();
  // scatter the sticks of this plane: four loads in flight per thread
  cx<T>* Wp = J.W + ((size_t)b * n3 + pz) * nst;
  for (int s0 = threadIdx.x; s0 < nst; s0 += 4 * nt) {
    int off[4];
    cx<T> val[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * nt;
      if (s < nst) { off[u] = J.st_y[s] * ld + J.st_x[s]; val[u] = Wp[s]; }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (s0 + u * nt < nst) plane[off[u]] = val[u];
  }
  __syncthreads();
  // y on the active columns, then x on every row; consecutive threads take
  // consecutive lines in both passes
  fft_lines<T, +1, false, kFusePlane<T>>(plane, ld, 0, ax, nax, true, J.r2, tw2, J.pm2, J.pr2);
  fft_lines<T, +1, false, kFusePlane<T>>(plane, 1, ld, nullptr, n2, true, J.r1, tw1, J.pm1, J.pr1);
  const FastDiv fn1(n1);
  if (stage) {
    cp_async_wait_all();
    __syncthreads();
    for (int i = threadIdx.x; i < n1 * n2; i += nt) {
      const int y = fn1.div(i), x = i - y * n1;
      plane[y * ld + x] = cscale(plane[y * ld + x], sv[i]);
    }
  } else {
    for (int i = threadIdx.x; i < n1 * n2; i += nt) {
      const int y = fn1.div(i), x = i - y * n1;
      plane[y * ld + x] = cscale(plane[y * ld + x], v[i]);
    }
  }
  __syncthreads();
  fft_lines<T, -1, true, kFusePlane<T>>(plane, 1, ld, nullptr, n2, true, J.r1, tw1, nullptr, J.pr1);
  fft_lines<T, -1, true, kFusePlane<T>>(plane, ld, 0, ax, nax, true, J.r2, tw2, nullptr, J.pr2);
  for (int s0 = threadIdx.x; s0 < nst; s0 += 4 * nt) {
    int off[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * nt;
      if (s < nst) off[u] = J.st_y[s] * ld + J.st_x[s];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (s0 + u * nt < nst) Wp[s0 + u * nt] = plane[off[u]];
  }
}

template <typename T>
__device__ void zfwd_tile(const FftJob<T>& J, int b, int sblk, unsigned char* smem) {
  cx<T>* line = reinterpret_cast<cx<T>*>(smem);
  const int n3 = J.r3.n, spb = J.spb, nst = J.nst;
  cx<T>* tw = line + (size_t)n3 * spb;
  const int s0 = sblk * spb;
  const int ns = min(spb, nst - s0);
  if (J.sqz) {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sq_tw_put<T>(tw, i, J.tw3[2 * i], J.tw3[2 * i + 1]);
  } else {
    const double* tw3 = J.tw3 + (ct_twiddles<T>() ? 2 * n3 : 0);
    for (int i = threadIdx.x; i < n3; i += blockDim.x) tw_put<T>(tw, i, tw3[2 * i], tw3[2 * i + 1]);
  }
  const cx<T>* Wb = J.W + (size_t)b * n3 * nst;
  const FastDiv fns(ns);
  for (int i = threadIdx.x; i < n3 * ns; i += blockDim.x) {
    const int pz = fns.div(i), l = i - pz * ns;
    line[pz * spb + l] = Wb[(size_t)pz * nst + s0 + l];
  }
  __syncthreads();
  if (J.sqz) {
#define QE_SQZ_FWD(n) sq_z_forward<T, n>(J, line, spb, ns, tw)
    QE_SQZ_DISPATCH(QE_SQZ_FWD)
#undef QE_SQZ_FWD
  } else {
    fft_lines<T, -1, true>(line, spb, 1, nullptr, ns, true, J.r3, tw, nullptr, J.pr3);
  }
  const int e0 = J.st_ptr[s0], e1 = J.st_ptr[s0 + ns];
  if (J.pair) {
    // W = F(V (a + i b)) with a, b real in r: F(V a)_G = (W_G + conj W_-G) / 2,
    // F(V b)_G = (W_G - conj W_-G) / 2i.  -G sits in the mirror stick (the
    // pair partner l ^ 1 of this tile, or the self-mirror stick itself) at -z.
    const double2* pa = reinterpret_cast<const double2*>(J.psi) + (size_t)(J.b0 + 2 * b) * J.npw;
    double2* ha = reinterpret_cast<double2*>(J.hpsi) + (size_t)(J.b0 + 2 * b) * J.npw;
    const bool hb = 2 * b + 1 < J.nbr;
    const double h = 0.5 * J.inv_n;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int g = J.st_g[e], z = J.st_z[e], s = J.st_of[e], l = s - s0;
      const int lm = s == J.self_st ? l : (l ^ 1);
      const int zm = z == 0 ? 0 : n3 - z;
      double wx, wy, mx, my;
      cx_to<T>(line[z * spb + l], wx, wy);
      cx_to<T>(line[zm * spb + lm], mx, my);
      const double kg = J.kin[g];
      const double2 a = pa[g];
      ha[g] = make_double2((wx + mx) * h + kg * a.x, (wy - my) * h + kg * a.y);
      if (hb) {
        const double2 c = pa[(size_t)J.npw + g];
        ha[(size_t)J.npw + g] = make_double2((wy + my) * h + kg * c.x, (mx - wx) * h + kg * c.y);
      }
    }
    return;
  }
  const double2* ps = reinterpret_cast<const double2*>(J.psi) + (size_t)(J.b0 + b) * J.npw;
  double2* hp = reinterpret_cast<double2*>(J.hpsi) + (size_t)(J.b0 + b) * J.npw;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int g = J.st_g[e];
    double cr, ci;
    cx_to<T>(line[J.st_z[e] * spb + (J.st_of[e] - s0)], cr, ci);
    const double2 p = ps[g];
    const double kg = J.kin[g];
    hp[g] = make_double2(cr * J.inv_n + kg * p.x, ci * J.inv_n + kg * p.y);
  }
}

// ---- one problem: tiles mapped on the grid ----------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_zinv(const FftJob<T> J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zinv_tile<T>(J, blockIdx.y, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(PlaneLB<T>::threads, PlaneLB<T>::minb) k_plane(const FftJob<T> J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  plane_tile<T>(J, blockIdx.y, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(512) k_zfwd(const FftJob<T> J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zfwd_tile<T>(J, blockIdx.y, blockIdx.x, smem_raw);
}

// ---- a batch of problems: persistent CTAs over a work queue ------------------------
// Items of job j are [prefix[j], prefix[j+1]); item i of a job maps to
// (band, tile) = (i / tiles, i % tiles).  counter must be zero at launch.
template <typename T, int STAGE>
struct BatchLB {
  static constexpr int threads = STAGE == 1 ? PlaneLB<T>::threads : 512;
  static constexpr int minb = STAGE == 1 ? PlaneLB<T>::minb : 1;
};

template <typename T, int STAGE>
__global__ void __launch_bounds__(BatchLB<T, STAGE>::threads, BatchLB<T, STAGE>::minb) k_fft_batch(const FftJob<T>* __restrict__ jobs,
                                                   const int* __restrict__ prefix, int njobs,
                                                   int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FftJob<T> sJ;
  __shared__ int item, cur;
  if (threadIdx.x == 0) cur = -1;
  const int total = prefix[njobs];
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = item;
    if (it >= total) break;
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= it) lo = mid;
      else hi = mid;
    }
    if (lo != cur) {   // stage the job descriptor in shared memory
      const int* src = reinterpret_cast<const int*>(&jobs[lo]);
      int* dst = reinterpret_cast<int*>(&sJ);
      for (int w = threadIdx.x; w < (int)(sizeof(FftJob<T>) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) cur = lo;
    }
    const int local = it - prefix[lo];
    const int tiles = STAGE == 1 ? sJ.r3.n : sJ.nsb;
    const int b = local / tiles, t = local - b * tiles;
    if (STAGE == 0) zinv_tile<T>(sJ, b, t, smem_raw);
    else if (STAGE == 1) plane_tile<T>(sJ, b, t, smem_raw);
    else zfwd_tile<T>(sJ, b, t, smem_raw);
  }
}

// ---- charge density: inverse transforms only, w |psi(r)|^2 summed over bands ----------
// rho(r) = (1 / Omega) sum_nk w_nk |psi_nk(r)|^2 (Sec. 3.3, charge-density
// generation).  After the z stage (zinv_tile), CTA (plane pz, group grp) runs
// the inverse y and x transforms of each FFT band of its group in turn and adds
// w |psi|^2 of its plane into per-thread registers (elements t, t + nt, ...;
// every band in the same order), then adds the sum into acc[grp][pz][...]
// (digit-reversed positions in all three axes, like the permuted potential).
// One CTA owns each (group, plane) slice in a launch, so the sums are
// deterministic; launches for more bands or k points accumulate in turn.
// Pair mode (k = 0): FFT band b carries the real-in-r bands 2b and 2b+1 as
// a + i b, so |a|^2 = Re^2 and |b|^2 = Im^2 with their own weights.
constexpr int kDensRegs = 24;
constexpr int kDensThreads = 512;

// The density tile on a square plane with the register-resident transform:
// the same band loop and sums as dens_plane_tile, the inverse transforms of
// plane2.cuh (its x and y order is the plan's).
template <typename T, int N>
__device__ void dens_plane_tile_sq(const FftJob<T>& J, int grp, int ngrp, int pz,
                                   const double* __restrict__ w, double* __restrict__ acc,
                                   int mode, unsigned char* smem) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B, ld = N | 1, n12 = N * N;
  const int n3 = J.r3.n, nst = J.nst, nt = blockDim.x;
  cx<T>* plane = reinterpret_cast<cx<T>*>(smem);
  cx<T>* tab = plane + ld * N;
  int* ax = reinterpret_cast<int*>(tab + N * sq_tw_slots<T>());
  sq_setup<T, N>(J, plane, tab, ax);
  const int bpg = (J.nb + ngrp - 1) / ngrp;
  const int b0 = grp * bpg, b1 = min(J.nb, b0 + bpg);
  const bool in_regs = n12 <= kDensRegs * nt;
  double racc[kDensRegs];
#pragma unroll
  for (int k = 0; k < kDensRegs; ++k) racc[k] = 0.0;
  double* accp = acc + ((size_t)grp * n3 + pz) * n12;
  const FastDiv fn(N);
  for (int b = b0; b < b1; ++b) {
    __syncthreads();
    if (b > b0)
      for (int i = threadIdx.x; i < ld * N; i += nt) plane[i] = cx_zero<T>();
    __syncthreads();
    const cx<T>* Wp = J.W + ((size_t)b * n3 + pz) * nst;
    for (int s = threadIdx.x; s < nst; s += nt) plane[J.st_y[s] * ld + J.st_x[s]] = Wp[s];
    __syncthreads();
    sq_inverse_yx1<T, N>(J, plane, tab, ax);
    for (int it = threadIdx.x; it < N * A; it += nt) {
      const int k1 = fn.div(it), y = it - k1 * N;
      cx<T>* p = plane + y * ld;
      cx<T> o[B];
      sq_inv2_regs<T, N>(p, 1, k1, tab, o);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) p[B * k1 + k2] = o[k2];
    }
    __syncthreads();
    double wa, wb = 0.0;
    if (J.pair) {
      wa = w[J.b0 + 2 * b];
      if (2 * b + 1 < J.nbr) wb = w[J.b0 + 2 * b + 1];
    } else {
      wa = w[J.b0 + b];
    }
    if (in_regs) {
#pragma unroll
      for (int k = 0; k < kDensRegs; ++k) {
        const int i = threadIdx.x + k * nt;
        if (i < n12) {
          const int y = fn.div(i), x = i - y * N;
          double re, im;
          cx_to<T>(plane[y * ld + x], re, im);
          racc[k] += mode ? wa * re : (J.pair ? wa * re * re + wb * im * im : wa * (re * re + im * im));
        }
      }
    } else {
      for (int i = threadIdx.x; i < n12; i += nt) {
        const int y = fn.div(i), x = i - y * N;
        double re, im;
        cx_to<T>(plane[y * ld + x], re, im);
        accp[i] += mode ? wa * re : (J.pair ? wa * re * re + wb * im * im : wa * (re * re + im * im));
      }
    }
  }
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kDensRegs; ++k) {
      const int i = threadIdx.x + k * nt;
      if (i < n12) accp[i] += racc[k];
    }
  }
}

template <typename T>
__device__ void dens_plane_tile(const FftJob<T>& J, int grp, int ngrp, int pz,
                                const double* __restrict__ w, double* __restrict__ acc,
                                int mode, unsigned char* smem) {
#define QE_SQ_DENS(n) dens_plane_tile_sq<T, n>(J, grp, ngrp, pz, w, acc, mode, smem)
  QE_SQ_DISPATCH(QE_SQ_DENS)
#undef QE_SQ_DENS
  const int n1 = J.r1.n, n2 = J.r2.n, n3 = J.r3.n, nst = J.nst, nax = J.nax;
  const int ld = plane_ld(n1), nt = blockDim.x, n12 = n1 * n2;
  cx<T>* plane = reinterpret_cast<cx<T>*>(smem);
  cx<T>* tw1 = plane + (size_t)ld * n2;
  cx<T>* tw2 = tw1 + (size_t)n1 * tw_slots<T>();
  int* ax = reinterpret_cast<int*>(tw2 + (size_t)n2 * tw_slots<T>());
  {
    const double* t1 = J.tw1 + (ct_twiddles<T>() ? 2 * n1 : 0);
    const double* t2 = J.tw2 + (ct_twiddles<T>() ? 2 * n2 : 0);
    for (int i = threadIdx.x; i < n1; i += nt) tw_put<T>(tw1, i, t1[2 * i], t1[2 * i + 1]);
    for (int i = threadIdx.x; i < n2; i += nt) tw_put<T>(tw2, i, t2[2 * i], t2[2 * i + 1]);
  }
  for (int i = threadIdx.x; i < nax; i += nt) ax[i] = J.ax[i];
  const int bpg = (J.nb + ngrp - 1) / ngrp;
  const int b0 = grp * bpg, b1 = min(J.nb, b0 + bpg);
  const bool in_regs = n12 <= kDensRegs * nt;
  double racc[kDensRegs];
#pragma unroll
  for (int k = 0; k < kDensRegs; ++k) racc[k] = 0.0;
  double* accp = acc + ((size_t)grp * n3 + pz) * n12;
  const FastDiv fn1(n1);
  for (int b = b0; b < b1; ++b) {
    __syncthreads();
    for (int i = threadIdx.x; i < ld * n2; i += nt) plane[i] = cx_zero<T>();
    __syncthreads();
    const cx<T>* Wp = J.W + ((size_t)b * n3 + pz) * nst;
    for (int s = threadIdx.x; s < nst; s += nt) plane[J.st_y[s] * ld + J.st_x[s]] = Wp[s];
    __syncthreads();
    fft_lines<T, +1, false, kFusePlane<T>>(plane, ld, 0, ax, nax, true, J.r2, tw2, J.pm2, J.pr2);
    fft_lines<T, +1, false, kFusePlane<T>>(plane, 1, ld, nullptr, n2, true, J.r1, tw1, J.pm1, J.pr1);
    // weights of this FFT band's real bands (pair) or of the band itself
    double wa, wb = 0.0;
    if (J.pair) {
      wa = w[J.b0 + 2 * b];
      if (2 * b + 1 < J.nbr) wb = w[J.b0 + 2 * b + 1];
    } else {
      wa = w[J.b0 + b];
    }
    if (in_regs) {
#pragma unroll
      for (int k = 0; k < kDensRegs; ++k) {
        const int i = threadIdx.x + k * nt;
        if (i < n12) {
          const int y = fn1.div(i), x = i - y * n1;
          double re, im;
          cx_to<T>(plane[y * ld + x], re, im);
          racc[k] += mode ? wa * re : (J.pair ? wa * re * re + wb * im * im : wa * (re * re + im * im));
        }
      }
    } else {
      for (int i = threadIdx.x; i < n12; i += nt) {
        const int y = fn1.div(i), x = i - y * n1;
        double re, im;
        cx_to<T>(plane[y * ld + x], re, im);
        accp[i] += mode ? wa * re : (J.pair ? wa * re * re + wb * im * im : wa * (re * re + im * im));
      }
    }
  }
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kDensRegs; ++k) {
      const int i = threadIdx.x + k * nt;
      if (i < n12) accp[i] += racc[k];
    }
  }
}

// mode 0: acc += w |psi(r)|^2 (the density); mode 1: acc += w Re psi(r) (the
// inverse transform of one band to the grid)
template <typename T>
__global__ void __launch_bounds__(kDensThreads) k_dens_plane(const FftJob<T> J, int ngrp,
                                                            const double* __restrict__ w,
                                                            double* __restrict__ acc, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dens_plane_tile<T>(J, blockIdx.y, ngrp, blockIdx.x, w, acc, mode, smem_raw);
}

// rho[perm3[pz]][perm2[py]][perm1[px]] = scale * sum_g acc[g][pz][py][px]
__global__ void k_dens_finish(const double* __restrict__ acc, int ngrp, int n1, int n2, int n3,
                              const int* __restrict__ p1, const int* __restrict__ p2,
                              const int* __restrict__ p3, double scale, double* __restrict__ rho) {
  const size_t total = (size_t)n1 * n2 * n3;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int px = (int)(i % n1);
    const int py = (int)((i / n1) % n2);
    const int pz = (int)(i / ((size_t)n1 * n2));
    double s = 0.0;
    for (int g = 0; g < ngrp; ++g) s += acc[(size_t)g * total + i];
    rho[((size_t)p3[pz] * n2 + p2[py]) * n1 + p1[px]] = scale * s;
  }
}

// ---- host side ---------------------------------------------------------------------
int sq_line_size(int n) {
  switch (n) {
    case 96: case 48: case 32: return n;
    default: return 0;
  }
}

int sq_plane_size(const int grid[3]) {
  if (grid[0] != grid[1]) return 0;
  return sq_line_size(grid[0]);
}

std::vector<int> sq_order(int n) {
  int A = 0, B = 0;
  switch (n) {
    case 96: A = SqSplit<96>::A; B = SqSplit<96>::B; break;
    case 48: A = SqSplit<48>::A; B = SqSplit<48>::B; break;
    case 32: A = SqSplit<32>::A; B = SqSplit<32>::B; break;
    default: return {};
  }
  std::vector<int> perm(n);
  for (int p = 0; p < n; ++p) perm[p] = p / B + A * (p % B);   // position B k1 + k2 holds k1 + A k2
  return perm;
}

size_t stick_bytes(const DevPlan& P, int nbc, size_t elem_bytes) {
  return (size_t)nbc * P.grid[2] * P.h.nst * elem_bytes;
}

// z lines with the two-pass transform: 16 sticks and 128 threads per CTA (C1,
// float-float: z stage 0.124 -> 0.113 ms per 32 bands; 32 sticks or 256
// threads leave a third of the threads idle in one pass of the two)
constexpr int kSqzSticks = 16, kSqzThreads = 128;

template <typename T>
int default_spb(int n3) {
  int spb = (int)(49152 / ((size_t)n3 * sizeof(cx<T>)));
  if (spb > 32) spb = 32;
  if (spb < 1) spb = 1;
  return spb;
}

template <typename T>
size_t zsm_bytes(int n3, int spb) {
  return ((size_t)n3 * spb + (size_t)n3 * tw_slots<T>()) * sizeof(cx<T>);
}

template <typename T>
static bool plane_stages_v(const DevPlan& P) {
  return kStageV<T> && P.sq == 0 && plane_v_offset<T>(P.grid[0], P.grid[1], P.h.nax) +
                               (size_t)P.grid[0] * P.grid[1] * sizeof(T) <= kStageVMaxBytes;
}

template <typename T>
size_t psm_bytes(const DevPlan& P) {
  const size_t base = ((size_t)plane_ld(P.grid[0]) * P.grid[1] +
                       (size_t)(P.grid[0] + P.grid[1]) * tw_slots<T>()) * sizeof(cx<T>) +
                      (size_t)P.h.nax * sizeof(int);
  return plane_stages_v<T>(P) ? plane_v_offset<T>(P.grid[0], P.grid[1], P.h.nax) +
                                    (size_t)P.grid[0] * P.grid[1] * sizeof(T)
                              : base;
}

template <typename T>
FftJob<T> make_job(const DevPlan& P, const double* psi, double* hpsi, const T* vp, void* W, int b0,
                   int nb, const FftShape& sh, int pair) {
  FftJob<T> J;
  std::memset(&J, 0, sizeof(J));
  J.r1 = P.rad[0];
  J.r2 = P.rad[1];
  J.r3 = P.rad[2];
  J.st_ptr = P.st_ptr;
  J.st_g = P.st_g;
  J.st_z = P.st_z;
  J.st_of = P.st_of;
  J.st_x = P.st_x;
  J.st_y = P.st_y;
  J.ax = P.ax;
  J.tw1 = P.tw[0];
  J.tw2 = P.tw[1];
  J.tw3 = P.tw[2];
  J.pm1 = P.perm[0];
  J.pm2 = P.perm[1];
  J.pm3 = P.perm[2];
  J.pr1 = P.rad[0].r[0] == 4 && 4 * P.h.half[0] < P.grid[0];
  J.pr2 = P.rad[1].r[0] == 4 && 4 * P.h.half[1] < P.grid[1];
  J.pr3 = P.rad[2].r[0] == 4 && 4 * P.h.half[2] < P.grid[2];
  J.kin = P.kin;
  J.psi = psi;
  J.hpsi = hpsi;
  J.vp = vp;
  J.W = reinterpret_cast<cx<T>*>(W);
  J.nst = P.h.nst;
  J.nax = P.h.nax;
  J.npw = P.h.npw;
  J.pair = pair && P.h.gamma ? 1 : 0;
  J.nbr = nb;
  J.nb = J.pair ? (nb + 1) / 2 : nb;   // FFT bands
  J.self_st = J.pair ? P.h.nst - 1 : -1;
  J.b0 = b0;
  J.spb = sh.spb > 0 ? sh.spb : (P.sqz ? kSqzSticks : default_spb<T>(P.grid[2]));
  if (J.pair) J.spb = std::max(2, J.spb & ~1);   // a tile holds whole mirror pairs
  J.nsb = (J.nst + J.spb - 1) / J.spb;
  J.inv_n = 1.0 / ((double)P.grid[0] * P.grid[1] * P.grid[2]);
  J.stage_v = plane_stages_v<T>(P) ? 1 : 0;
  J.sq = P.sq;
  J.sqz = P.sqz;
  return J;
}

template <typename T>
int launch_vperm(const DevPlan& P, const double* vloc, T* vp, cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, "k_vperm", st);
  const size_t total = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  k_vperm<T><<<blocks, 256, 0, st>>>(vloc, vp, P.grid[0], P.grid[1], P.grid[2], P.perm[0],
                                     P.perm[1], P.perm[2]);
  return check_launch("k_vperm");
}

template <typename T>
int launch_local_kinetic_shape(const DevPlan& P, const double* psi, double* hpsi, const T* vp,
                               void* Wv, int b0, int nbc, const FftShape& sh, cudaStream_t st,
                               Prof* pf, int pair) {
  const FftJob<T> J = make_job<T>(P, psi, hpsi, vp, Wv, b0, nbc, sh, pair);
  const size_t zsm = zsm_bytes<T>(P.grid[2], J.spb);
  const size_t psm = psm_bytes<T>(P);
  if (psm > 227 * 1024) {
    set_error("FFT plane %d x %d does not fit in shared memory at this precision", P.grid[0],
              P.grid[1]);
    return QE_EINVAL;
  }
  // The cap is a per-function device attribute shared by every thread of the
  // process: always set the same (largest) value so that concurrent callers
  // with different plane sizes cannot lower it under each other's launch.
  set_max_dynamic_smem(k_plane<T>);
  set_max_dynamic_smem(k_plane_sq<T, 96>);
  set_max_dynamic_smem(k_plane_sq<T, 48>);
  set_max_dynamic_smem(k_plane_sq<T, 32>);
  set_max_dynamic_smem(k_zinv<T>);
  set_max_dynamic_smem(k_zfwd<T>);
  const int zt = sh.zthreads > 0 ? sh.zthreads : (J.sqz ? kSqzThreads : 256);
  const int pt = std::min(sh.pthreads > 0 ? sh.pthreads : PlaneLB<T>::dflt, PlaneLB<T>::threads);
  const int pts = std::min(sh.pthreads > 0 ? sh.pthreads : SqLB<T>::dflt, SqLB<T>::threads);
  dim3 gz(J.nsb, J.nb);
  int rc;
  {
    ProfScope ps(pf, "k_zinv", st);
    k_zinv<T><<<gz, zt, zsm, st>>>(J);
    rc = check_launch("k_zinv");
  }
  if (rc) return rc;
  {
    ProfScope ps(pf, "k_plane", st);
    const dim3 gp(P.grid[2], J.nb);
    switch (J.sq) {
      case 96: k_plane_sq<T, 96><<<gp, pts, psm, st>>>(J); break;
      case 48: k_plane_sq<T, 48><<<gp, pts, psm, st>>>(J); break;
      case 32: k_plane_sq<T, 32><<<gp, pts, psm, st>>>(J); break;
      default: k_plane<T><<<gp, pt, psm, st>>>(J); break;
    }
    rc = check_launch("k_plane");
  }
  if (rc) return rc;
  ProfScope ps(pf, "k_zfwd", st);
  k_zfwd<T><<<gz, zt, zsm, st>>>(J);
  return check_launch("k_zfwd");
}

template <typename T>
int launch_local_kinetic(const DevPlan& P, const double* psi, double* hpsi, const T* vp, void* Wv,
                         int b0, int nbc, cudaStream_t st, Prof* pf, int pair) {
  return launch_local_kinetic_shape<T>(P, psi, hpsi, vp, Wv, b0, nbc, tuned_shape(P, sizeof(T)),
                                       st, pf, pair);
}

// Batched local + kinetic: every stage is one persistent launch over all jobs.
// prefix_dev holds two prefix arrays of njobs + 1 items (stick-block items, then
// plane items); counters (3 ints) are zeroed here; smem_* are the largest
// per-item needs over the jobs.
template <typename T>
int launch_local_kinetic_batch(const FftJob<T>* jobs_dev, const int* prefix_dev, int njobs,
                               int* counters, size_t smem_z, size_t smem_p, int threads, int zthreads,
                               cudaStream_t st, Prof* pf) {
  if (smem_p > 227 * 1024) {
    set_error("batched FFT: a plane does not fit in shared memory at this precision");
    return QE_EINVAL;
  }
  set_max_dynamic_smem(k_fft_batch<T, 0>);
  set_max_dynamic_smem(k_fft_batch<T, 1>);
  set_max_dynamic_smem(k_fft_batch<T, 2>);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemsetAsync(counters, 0, 3 * sizeof(int), st) != cudaSuccess) {
    set_error("batched FFT: memset failed");
    return QE_ECUDA;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_batch<T, 0>, zthreads, smem_z);
  {
    ProfScope ps(pf, "k_zinv_batch", st);
    k_fft_batch<T, 0><<<nsm * std::max(1, occ), zthreads, smem_z, st>>>(jobs_dev, prefix_dev, njobs,
                                                                       counters);
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_batch<T, 1>, threads, smem_p);
  {
    ProfScope ps(pf, "k_plane_batch", st);
    k_fft_batch<T, 1><<<nsm * std::max(1, occ), threads, smem_p, st>>>(
        jobs_dev, prefix_dev + (njobs + 1), njobs, counters + 1);
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_batch<T, 2>, zthreads, smem_z);
  {
    ProfScope ps(pf, "k_zfwd_batch", st);
    k_fft_batch<T, 2><<<nsm * std::max(1, occ), zthreads, smem_z, st>>>(jobs_dev, prefix_dev, njobs,
                                                                       counters + 2);
  }
  return check_launch("batched FFT");
}

// Density of bands b0 .. b0+nbc-1 of psi (weights w, device, indexed by band)
// into the group accumulators acc [ngrp][N3][N2][N1]: z stage into W, then the
// inverse planes.  pair: k = 0 bands real in r, two per FFT.
template <typename T>
int launch_density(const DevPlan& P, const double* psi, const double* w, void* Wv, int b0, int nbc,
                   int ngrp, double* acc, cudaStream_t st, Prof* pf, int pair, int mode) {
  const FftShape sh = tuned_shape(P, sizeof(T));
  const FftJob<T> J = make_job<T>(P, psi, nullptr, nullptr, Wv, b0, nbc, sh, pair);
  const size_t zsm = zsm_bytes<T>(P.grid[2], J.spb);
  const size_t psm = ((size_t)plane_ld(P.grid[0]) * P.grid[1] +
                      (size_t)(P.grid[0] + P.grid[1]) * tw_slots<T>()) * sizeof(cx<T>) +
                     (size_t)P.h.nax * sizeof(int);
  if (psm > 227 * 1024) {
    set_error("FFT plane %d x %d does not fit in shared memory at this precision", P.grid[0],
              P.grid[1]);
    return QE_EINVAL;
  }
  set_max_dynamic_smem(k_zinv<T>);
  set_max_dynamic_smem(k_dens_plane<T>);
  const int zt = sh.zthreads > 0 ? sh.zthreads : (J.sqz ? kSqzThreads : 256);
  int rc;
  {
    ProfScope ps(pf, "k_zinv", st);
    k_zinv<T><<<dim3(J.nsb, J.nb), zt, zsm, st>>>(J);
    rc = check_launch("k_zinv");
  }
  if (rc) return rc;
  ProfScope ps(pf, "k_dens_plane", st);
  k_dens_plane<T><<<dim3(P.grid[2], ngrp), kDensThreads, psm, st>>>(J, ngrp, w, acc, mode);
  return check_launch("k_dens_plane");
}

int launch_density_finish(const DevPlan& P, const double* acc, int ngrp, double scale, double* rho,
                          cudaStream_t st, Prof* pf) {
  ProfScope ps(pf, "k_dens_finish", st);
  const size_t total = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  k_dens_finish<<<blocks, 256, 0, st>>>(acc, ngrp, P.grid[0], P.grid[1], P.grid[2], P.perm[0],
                                        P.perm[1], P.perm[2], scale, rho);
  return check_launch("k_dens_finish");
}

#define QE_FFT_INSTANTIATE(T)                                                                  \
  template int launch_vperm<T>(const DevPlan&, const double*, T*, cudaStream_t, Prof*);            \
  template int launch_local_kinetic<T>(const DevPlan&, const double*, double*, const T*, void*,    \
                                       int, int, cudaStream_t, Prof*, int);                        \
  template int launch_local_kinetic_shape<T>(const DevPlan&, const double*, double*, const T*,     \
                                             void*, int, int, const FftShape&, cudaStream_t,       \
                                             Prof*, int);                                          \
  template int launch_local_kinetic_batch<T>(const FftJob<T>*, const int*, int, int*, size_t,      \
                                             size_t, int, int, cudaStream_t, Prof*);               \
  template FftJob<T> make_job<T>(const DevPlan&, const double*, double*, const T*, void*, int,     \
                                 int, const FftShape&, int);                                       \
  template size_t zsm_bytes<T>(int, int);                                                          \
  template int default_spb<T>(int);                                                                \
  template size_t psm_bytes<T>(const DevPlan&);                                                    \
  template int launch_density<T>(const DevPlan&, const double*, const double*, void*, int, int,    \
                                 int, double*, cudaStream_t, Prof*, int, int);
QE_FFT_INSTANTIATE(double)
QE_FFT_INSTANTIATE(float)
QE_FFT_INSTANTIATE(ff)
#undef QE_FFT_INSTANTIATE

}  // namespace qe
