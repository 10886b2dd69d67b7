// Local-potential and kinetic part of H|psi> (Sec. 3.3 of the paper: the
// local-potential and kinetic-energy contributions; FFTXlib of Sec. 3.2.1):
//
//   psi(r_j) = sum_G c_G e^{iG.r_j},   (H c)_G = |k+G|^2 c_G + (1/N) sum_j e^{-iG.r_j} V(r_j) psi(r_j)
//
// as a pruned 3D FFT in three kernels per block of bands:
//   k_zinv   scatter the sphere onto its sticks (x, y columns) and run the
//            inverse z transform of each stick (DIF, z left digit-reversed);
//   k_plane  one CTA per (z plane, band): scatter the sticks into the plane,
//            inverse y transform of the columns that hold sticks, inverse x
//            transform of every row, multiply by V (read through the digit
//            reversal), forward x and y transforms (DIT), gather the sticks;
//   k_zfwd   forward z transform of each stick (DIT, natural order out),
//            gather onto the sphere, scale by 1/N and add |k+G|^2 c_G.
// Sticks live in a workspace laid out [band][z][stick] so that every kernel
// reads and writes it with consecutive threads on consecutive sticks.
#include <algorithm>
#include <cstdio>

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

template <typename T>
__global__ void __launch_bounds__(256)
k_zinv(const double* __restrict__ psi, int npw, int b0, const int* __restrict__ st_ptr,
       const int* __restrict__ st_g, const int* __restrict__ st_z, const int* __restrict__ st_of,
       int nst, Radix r3, const double* __restrict__ tw3, cx<T>* __restrict__ W, int spb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw);
  const int n3 = r3.n;
  cx<T>* tw = line + (size_t)n3 * spb;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nst - s0);
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < n3 * spb; i += blockDim.x) line[i] = {T(0), T(0)};
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = {T(tw3[2 * i]), T(tw3[2 * i + 1])};
  __syncthreads();
  const double2* ps = reinterpret_cast<const double2*>(psi) + (size_t)(b0 + b) * npw;
  const int e0 = st_ptr[s0], e1 = st_ptr[s0 + ns];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double2 c = ps[st_g[e]];
    line[st_z[e] * spb + (st_of[e] - s0)] = {T(c.x), T(c.y)};
  }
  __syncthreads();
  fft_lines<T, +1, false>(line, spb, 1, nullptr, ns, true, r3, tw);
  cx<T>* Wb = W + (size_t)b * n3 * nst;
  for (int i = threadIdx.x; i < n3 * ns; i += blockDim.x) {
    const int pz = i / ns, l = i - pz * ns;
    Wb[(size_t)pz * nst + s0 + l] = line[pz * spb + l];
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_plane(cx<T>* __restrict__ W, int nst, const int* __restrict__ st_x, const int* __restrict__ st_y,
        const int* __restrict__ ax_g, int nax, Radix r1, Radix r2, const double* __restrict__ tw1g,
        const double* __restrict__ tw2g, const T* __restrict__ vp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = r1.n, n2 = r2.n, n3 = gridDim.x;
  cx<T>* plane = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw1 = plane + (size_t)n1 * n2;
  cx<T>* tw2 = tw1 + n1;
  int* ax = reinterpret_cast<int*>(tw2 + n2);
  const int pz = blockIdx.x, b = blockIdx.y;
  for (int i = threadIdx.x; i < n1 * n2; i += blockDim.x) plane[i] = {T(0), T(0)};
  for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = {T(tw1g[2 * i]), T(tw1g[2 * i + 1])};
  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = {T(tw2g[2 * i]), T(tw2g[2 * i + 1])};
  for (int i = threadIdx.x; i < nax; i += blockDim.x) ax[i] = ax_g[i];
  __syncthreads();
  cx<T>* Wp = W + ((size_t)b * n3 + pz) * nst;
  for (int s = threadIdx.x; s < nst; s += blockDim.x) plane[st_y[s] * n1 + st_x[s]] = Wp[s];
  __syncthreads();
  fft_lines<T, +1, false>(plane, n1, 0, ax, nax, true, r2, tw2);        // y, active columns
  fft_lines<T, +1, false>(plane, 1, n1, nullptr, n2, false, r1, tw1);   // x, every row
  const T* v = vp + (size_t)pz * n1 * n2;
  for (int i = threadIdx.x; i < n1 * n2; i += blockDim.x) plane[i] = cscale(plane[i], v[i]);
  __syncthreads();
  fft_lines<T, -1, true>(plane, 1, n1, nullptr, n2, false, r1, tw1);
  fft_lines<T, -1, true>(plane, n1, 0, ax, nax, true, r2, tw2);
  for (int s = threadIdx.x; s < nst; s += blockDim.x) Wp[s] = plane[st_y[s] * n1 + st_x[s]];
}

template <typename T>
__global__ void __launch_bounds__(256)
k_zfwd(const cx<T>* __restrict__ W, int nst, const int* __restrict__ st_ptr,
       const int* __restrict__ st_g, const int* __restrict__ st_z, const int* __restrict__ st_of,
       Radix r3, const double* __restrict__ tw3, const double* __restrict__ psi,
       const double* __restrict__ kin, double* __restrict__ hpsi, int npw, int b0, double inv_n,
       int spb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw);
  const int n3 = r3.n;
  cx<T>* tw = line + (size_t)n3 * spb;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nst - s0);
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = {T(tw3[2 * i]), T(tw3[2 * i + 1])};
  const cx<T>* Wb = W + (size_t)b * n3 * nst;
  for (int i = threadIdx.x; i < n3 * ns; i += blockDim.x) {
    const int pz = i / ns, l = i - pz * ns;
    line[pz * spb + l] = Wb[(size_t)pz * nst + s0 + l];
  }
  __syncthreads();
  fft_lines<T, -1, true>(line, spb, 1, nullptr, ns, true, r3, tw);
  const double2* ps = reinterpret_cast<const double2*>(psi) + (size_t)(b0 + b) * npw;
  double2* hp = reinterpret_cast<double2*>(hpsi) + (size_t)(b0 + b) * npw;
  const int e0 = st_ptr[s0], e1 = st_ptr[s0 + ns];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int g = st_g[e];
    const cx<T> c = line[st_z[e] * spb + (st_of[e] - s0)];
    const double2 p = ps[g];
    const double kg = kin[g];
    hp[g] = make_double2((double)c.x * inv_n + kg * p.x, (double)c.y * inv_n + kg * p.y);
  }
}

size_t stick_bytes(const DevPlan& P, int nbc, size_t elem_bytes) {
  return (size_t)nbc * P.grid[2] * P.h.nst * elem_bytes;
}

template <typename T>
static int sticks_per_block(int n3) {
  int spb = (int)(49152 / ((size_t)n3 * sizeof(cx<T>)));
  if (spb > 32) spb = 32;
  if (spb < 1) spb = 1;
  return spb;
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
int launch_local_kinetic(const DevPlan& P, const double* psi, double* hpsi, const T* vp, void* Wv,
                         int b0, int nbc, cudaStream_t st, Prof* pf) {
  cx<T>* W = reinterpret_cast<cx<T>*>(Wv);
  const int n1 = P.grid[0], n2 = P.grid[1], n3 = P.grid[2];
  const int nst = P.h.nst;
  const int spb = sticks_per_block<T>(n3);
  const size_t zsm = ((size_t)n3 * spb + n3) * sizeof(cx<T>);
  const size_t psm = ((size_t)n1 * n2 + n1 + n2) * sizeof(cx<T>) + (size_t)P.h.nax * sizeof(int);
  if (psm > 227 * 1024) {
    set_error("FFT plane %d x %d does not fit in shared memory at this precision", n1, n2);
    return QE_EINVAL;
  }
  // The cap is a per-function device attribute shared by every thread of the
  // process: always set the same (largest) value so that concurrent callers
  // with different plane sizes cannot lower it under each other's launch.
  set_max_dynamic_smem(k_plane<T>);
  set_max_dynamic_smem(k_zinv<T>);
  set_max_dynamic_smem(k_zfwd<T>);
  dim3 gz((nst + spb - 1) / spb, nbc);
  int rc;
  {
  ProfScope ps(pf, "k_zinv", st);
  k_zinv<T><<<gz, 256, zsm, st>>>(psi, P.h.npw, b0, P.st_ptr, P.st_g, P.st_z, P.st_of, nst,
                                  P.rad[2], P.tw[2], W, spb);
  rc = check_launch("k_zinv");
  }
  if (rc) return rc;
  dim3 gp(n3, nbc);
  {
  ProfScope ps(pf, "k_plane", st);
  k_plane<T><<<gp, 256, psm, st>>>(W, nst, P.st_x, P.st_y, P.ax, P.h.nax, P.rad[0], P.rad[1],
                                   P.tw[0], P.tw[1], vp);
  rc = check_launch("k_plane");
  }
  if (rc) return rc;
  ProfScope ps(pf, "k_zfwd", st);
  const double inv_n = 1.0 / ((double)n1 * n2 * n3);
  k_zfwd<T><<<gz, 256, zsm, st>>>(W, nst, P.st_ptr, P.st_g, P.st_z, P.st_of, P.rad[2], P.tw[2],
                                  psi, P.kin, hpsi, P.h.npw, b0, inv_n, spb);
  return check_launch("k_zfwd");
}

template int launch_vperm<double>(const DevPlan&, const double*, double*, cudaStream_t, Prof*);
template int launch_vperm<float>(const DevPlan&, const double*, float*, cudaStream_t, Prof*);
template int launch_local_kinetic<double>(const DevPlan&, const double*, double*, const double*,
                                          void*, int, int, cudaStream_t, Prof*);
template int launch_local_kinetic<float>(const DevPlan&, const double*, double*, const float*,
                                         void*, int, int, cudaStream_t, Prof*);

}  // namespace qe
