// Charge density of bands over k points (Sec. 3.3 of the paper lists
// charge-density generation among the kernels that run on the GPU):
//
//   rho(r_j) = (1 / Omega) sum_k sum_n w_nk |psi_nk(r_j)|^2,
//   psi_nk(r_j) = sum_G c_nk(G) e^{iG.r_j}   (the e^{ik.r} factor has modulus 1)
//
// per k point: the z stage of the H|psi> FFT (scatter onto the sticks, inverse
// z transforms), then one CTA per (z plane, band group) running the inverse y
// and x transforms of its bands and summing w |psi|^2 (fft.cu); the groups'
// sums over all k points are added in a fixed order and un-permuted at the end.
// The sum over k, the only reduction across k points on this path, runs inside
// these accumulations on the one GPU.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "plan.h"

namespace qe {

constexpr int kDensGroups = 8;   // band groups per plane: partial sums added in a fixed order

template <typename T>
static int density_k(qe_ctx* ctx, const DevPlan& P, const double* psi, const double* w, int nb,
                     bool pair, double* acc, cudaStream_t st) {
  const size_t per_band = stick_bytes(P, 1, 2 * sizeof(T));
  const int per_fft = pair ? 2 : 1;
  int nfb = (int)std::max<size_t>(1, ctx->stick_budget / std::max<size_t>(per_band, 1));
  nfb = std::min(nfb, (nb + per_fft - 1) / per_fft);
  const int nbc = nfb * per_fft;
  int rc = ctx->sticks.ensure(stick_bytes(P, nfb, 2 * sizeof(T)));
  if (rc) return rc;
  for (int b0 = 0; b0 < nb; b0 += nbc) {
    rc = launch_density<T>(P, psi, w, ctx->sticks.p, b0, std::min(nbc, nb - b0), kDensGroups, acc,
                           st, &ctx->prof, pair ? 1 : 0);
    if (rc) return rc;
  }
  return QE_OK;
}

}  // namespace qe

using namespace qe;

#define DN_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define DN_CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error("%s: %s", #x, cudaGetErrorString(e_)); return QE_ECUDA; } } while (0)

// rho (device, [N3][N2][N1]) of the bands; arguments as qe_density's (already
// checked), `precision` without flags, `pair` from QE_GAMMA.
static int density_into(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
                        const double* kpts, const int* nbnd, const double* const* psi,
                        const double* const* weights, int precision, bool pair, double* drho,
                        int mem, cudaStream_t st) {
  const size_t ngrid = (size_t)grid[0] * grid[1] * grid[2];
  std::vector<DevPlan*> plans(nk, nullptr);
  const double zero_k[3] = {0.0, 0.0, 0.0};
  DevPlan* P0 = nullptr;
  DN_TRY(get_plan(ctx, lat, nk > 0 ? kpts : zero_k, ecut, grid, &P0));
  for (int i = 0; i < nk; ++i) DN_TRY(get_plan(ctx, lat, kpts + 3 * i, ecut, grid, &plans[i]));
  size_t nw = 0;
  for (int i = 0; i < nk; ++i) nw += (size_t)nbnd[i];
  DN_TRY(ctx->dens_acc.ensure((size_t)kDensGroups * ngrid * sizeof(double)));
  DN_TRY(ctx->dens_w.ensure(std::max<size_t>(nw, 1) * sizeof(double)));
  std::vector<double> wh(std::max<size_t>(nw, 1), 0.0);
  for (int i = 0, o = 0; i < nk; o += nbnd[i], ++i)
    if (nbnd[i] > 0) std::memcpy(wh.data() + o, weights[i], (size_t)nbnd[i] * sizeof(double));
  DN_CU(cudaMemcpyAsync(ctx->dens_w.p, wh.data(), wh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  double* acc = (double*)ctx->dens_acc.p;
  DN_CU(cudaMemsetAsync(acc, 0, (size_t)kDensGroups * ngrid * sizeof(double), st));
  size_t wo = 0;
  for (int i = 0; i < nk; ++i) {
    const int nb = nbnd[i];
    const DevPlan& P = *plans[i];
    const double* wk = (const double*)ctx->dens_w.p + wo;
    wo += (size_t)nb;
    if (nb == 0) continue;
    const double* dpsi = psi[i];
    if (mem == QE_HOST) {
      const size_t bytes = (size_t)nb * P.h.npw * 2 * sizeof(double);
      DN_TRY(ctx->h_psi.ensure(bytes));
      DN_CU(cudaMemcpyAsync(ctx->h_psi.p, psi[i], bytes, cudaMemcpyHostToDevice, st));
      dpsi = (const double*)ctx->h_psi.p;
    }
    const bool pr = pair && P.h.gamma;
    DN_TRY(precision == QE_FP64 ? density_k<FftF64>(ctx, P, dpsi, wk, nb, pr, acc, st)
                                : density_k<float>(ctx, P, dpsi, wk, nb, pr, acc, st));
  }
  return launch_density_finish(*P0, acc, kDensGroups, 1.0 / cell_volume(lat), drho, st, &ctx->prof);
}

static int density_args(const double lat[9], const int grid[3], int nk, const double* kpts,
                        const int* nbnd, const double* const* psi, const double* const* weights,
                        int mem, const char* who) {
  if (!lat || !grid || nk < 0 || (nk > 0 && (!kpts || !nbnd || !psi || !weights))) {
    set_error("%s: invalid argument", who);
    return QE_EINVAL;
  }
  if (mem != QE_HOST && mem != QE_DEVICE) { set_error("%s: bad mem flag", who); return QE_EINVAL; }
  for (int c = 0; c < 3; ++c)
    if (grid[c] < 1) { set_error("%s: grid must be positive", who); return QE_EINVAL; }
  for (int i = 0; i < nk; ++i) {
    if (nbnd[i] < 0) { set_error("%s: negative band count at k point %d", who, i); return QE_EINVAL; }
    if (nbnd[i] > 0 && (!psi[i] || !weights[i])) {
      set_error("%s: null psi/weights at k point %d", who, i);
      return QE_EINVAL;
    }
  }
  return QE_OK;
}

extern "C" int qe_density(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
                          const double* kpts, const int* nbnd, const double* const* psi,
                          const double* const* weights, int precision, double* rho, int mem,
                          void* stream) {
  clear_error();
  if (!ctx || !rho) { set_error("qe_density: invalid argument"); return QE_EINVAL; }
  DN_TRY(density_args(lat, grid, nk, kpts, nbnd, psi, weights, mem, "qe_density"));
  const bool pair = (precision & QE_GAMMA) != 0;
  precision &= ~QE_GAMMA;
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_density: bad precision"); return QE_EINVAL; }
  DN_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DN_TRY(ctx_begin(ctx, st));
  const size_t ngrid = (size_t)grid[0] * grid[1] * grid[2];
  double* drho = rho;
  if (mem == QE_HOST) {
    DN_TRY(ctx->h_v.ensure(ngrid * sizeof(double)));
    drho = (double*)ctx->h_v.p;
  }
  DN_TRY(density_into(ctx, lat, ecut, grid, nk, kpts, nbnd, psi, weights, precision, pair, drho, mem, st));
  if (mem == QE_HOST) {
    DN_CU(cudaMemcpyAsync(rho, drho, ngrid * sizeof(double), cudaMemcpyDeviceToHost, st));
    DN_CU(cudaStreamSynchronize(st));
  }
  return QE_OK;
}

// ---- one self-consistency step of the local potential -------------------------------
// Sec. 3.3 lists electronic self-consistency among the GPU-accelerated
// functionalities.  From rho of the bands: rho~(G) on the density sphere
// |G|^2 <= 4 ecut (the local part of H applied to the G = 0 plane wave with
// V = rho is exactly (1/N) sum_j e^{-iG.r_j} rho(r_j)), V_H(G) = 8 pi rho~(G) /
// |G|^2 (G = 0 dropped), its inverse transform to the grid (the density
// stage's mode 1), the Slater exchange -2 (3 rho / pi)^{1/3} and the mixing
// V_new = (1 - alpha) V_in + alpha (V_ext + V_H + v_x).  The sum over k of the
// density is the only reduction across k points; every step runs on the GPU.
namespace qe {

__global__ void k_poisson(const double2* __restrict__ rg, const double* __restrict__ kin, int n,
                          double2* __restrict__ vg) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const double q2 = kin[g];
  const double f = q2 > 0.0 ? 25.132741228718345907701147066236 / q2 : 0.0;   // 8 pi / |G|^2
  vg[g] = make_double2(f * rg[g].x, f * rg[g].y);
}

__global__ void k_scf_mix(const double* __restrict__ rho, const double* __restrict__ vh,
                          const double* __restrict__ vext, const double* __restrict__ vin,
                          double alpha, size_t n, double* __restrict__ vnew) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double vx = -2.0 * cbrt(0.95492965855137201461 * fmax(rho[i], 0.0));   // 3 / pi
    vnew[i] = (1.0 - alpha) * vin[i] + alpha * (vext[i] + vh[i] + vx);
  }
}

template <typename T>
static int scf_potential(qe_ctx* ctx, const DevPlan& Pd, const double* rho, double* e0, double* rg,
                         double* vg, const double* w1, double* vh, cudaStream_t st) {
  const size_t ngrid = (size_t)Pd.grid[0] * Pd.grid[1] * Pd.grid[2];
  ctx->last_op = qe_ctx::LastOp{};   // the permuted potential below is rho's
  DN_TRY(ctx->vp.ensure(ngrid * sizeof(T)));
  DN_TRY(launch_vperm<T>(Pd, rho, (T*)ctx->vp.p, st, &ctx->prof));
  DN_TRY(ctx->sticks.ensure(stick_bytes(Pd, 1, 2 * sizeof(T))));
  DN_TRY(launch_local_kinetic<T>(Pd, e0, rg, (const T*)ctx->vp.p, ctx->sticks.p, 0, 1, st, &ctx->prof));
  const int npw = Pd.h.npw;
  k_poisson<<<(npw + 255) / 256, 256, 0, st>>>(reinterpret_cast<const double2*>(rg), Pd.kin, npw,
                                               reinterpret_cast<double2*>(vg));
  DN_CU(cudaGetLastError());
  double* acc = (double*)ctx->dens_acc.p;
  DN_CU(cudaMemsetAsync(acc, 0, (size_t)kDensGroups * ngrid * sizeof(double), st));
  DN_TRY(launch_density<T>(Pd, vg, w1, ctx->sticks.p, 0, 1, kDensGroups, acc, st, &ctx->prof, 0, 1));
  return launch_density_finish(Pd, acc, kDensGroups, 1.0, vh, st, &ctx->prof);
}

}  // namespace qe

extern "C" int qe_scf_step(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
                           const double* kpts, const int* nbnd, const double* const* psi,
                           const double* const* weights, const double* vext, const double* vin,
                           double alpha, int precision, double* vnew, double* rho_out, int mem,
                           void* stream) {
  clear_error();
  if (!ctx || !vext || !vin || !vnew) { set_error("qe_scf_step: invalid argument"); return QE_EINVAL; }
  DN_TRY(density_args(lat, grid, nk, kpts, nbnd, psi, weights, mem, "qe_scf_step"));
  const bool pair = (precision & QE_GAMMA) != 0;
  precision &= ~QE_GAMMA;
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_scf_step: bad precision"); return QE_EINVAL; }
  DN_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DN_TRY(ctx_begin(ctx, st));
  const size_t ngrid = (size_t)grid[0] * grid[1] * grid[2];
  // the density sphere at k = 0 (fails with QE_EINVAL when the grid cannot hold it)
  DevPlan* Pd = nullptr;
  const double k0[3] = {0.0, 0.0, 0.0};
  DN_TRY(get_plan(ctx, lat, k0, 4.0 * ecut, grid, &Pd));
  const int npwd = Pd->h.npw;
  // work: rho, V_H, three host-array stagings (V_ext, V_in, V_new) [ngrid]; the
  // G = 0 unit vector, rho~ and V_H~ [npwd] complex; the weight 1
  const size_t gb = (ngrid * sizeof(double) + 255) & ~(size_t)255;
  const size_t sb = ((size_t)npwd * 16 + 255) & ~(size_t)255;
  DN_TRY(ctx->scf_work.ensure(5 * gb + 3 * sb + 256));
  char* base = static_cast<char*>(ctx->scf_work.p);
  double* drho = reinterpret_cast<double*>(base);
  double* dvh = reinterpret_cast<double*>(base + gb);
  double* dvext = reinterpret_cast<double*>(base + 2 * gb);
  double* dvin = reinterpret_cast<double*>(base + 3 * gb);
  double* dvnew = reinterpret_cast<double*>(base + 4 * gb);
  double* e0 = reinterpret_cast<double*>(base + 5 * gb);
  double* rg = reinterpret_cast<double*>(base + 5 * gb + sb);
  double* vg = reinterpret_cast<double*>(base + 5 * gb + 2 * sb);
  double* w1 = reinterpret_cast<double*>(base + 5 * gb + 3 * sb);
  const double one[2] = {1.0, 0.0};
  DN_CU(cudaMemsetAsync(e0, 0, (size_t)npwd * 16, st));
  DN_CU(cudaMemcpyAsync(e0, one, sizeof(one), cudaMemcpyHostToDevice, st));   // G = 0 is first
  DN_CU(cudaMemcpyAsync(w1, one, sizeof(double), cudaMemcpyHostToDevice, st));
  if (mem == QE_HOST) {
    DN_CU(cudaMemcpyAsync(dvext, vext, ngrid * sizeof(double), cudaMemcpyHostToDevice, st));
    DN_CU(cudaMemcpyAsync(dvin, vin, ngrid * sizeof(double), cudaMemcpyHostToDevice, st));
  } else {
    dvext = const_cast<double*>(vext);
    dvin = const_cast<double*>(vin);
    dvnew = vnew;
    if (rho_out) drho = rho_out;
  }
  DN_TRY(density_into(ctx, lat, ecut, grid, nk, kpts, nbnd, psi, weights, precision, pair, drho, mem, st));
  DN_TRY(precision == QE_FP64 ? scf_potential<FftF64>(ctx, *Pd, drho, e0, rg, vg, w1, dvh, st)
                              : scf_potential<float>(ctx, *Pd, drho, e0, rg, vg, w1, dvh, st));
  const int blocks = (int)std::min<size_t>((ngrid + 255) / 256, 152 * 16);
  k_scf_mix<<<blocks, 256, 0, st>>>(drho, dvh, dvext, dvin, alpha, ngrid, dvnew);
  DN_CU(cudaGetLastError());
  if (mem == QE_HOST) {
    DN_CU(cudaMemcpyAsync(vnew, dvnew, ngrid * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (rho_out) DN_CU(cudaMemcpyAsync(rho_out, drho, ngrid * sizeof(double), cudaMemcpyDeviceToHost, st));
    DN_CU(cudaStreamSynchronize(st));
  }
  return QE_OK;
}
