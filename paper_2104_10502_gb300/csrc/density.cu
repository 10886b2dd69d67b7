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

extern "C" int qe_density(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
                          const double* kpts, const int* nbnd, const double* const* psi,
                          const double* const* weights, int precision, double* rho, int mem,
                          void* stream) {
  clear_error();
  if (!ctx || !lat || !grid || !rho || nk < 0 || (nk > 0 && (!kpts || !nbnd || !psi || !weights))) {
    set_error("qe_density: invalid argument");
    return QE_EINVAL;
  }
  const bool pair = (precision & QE_GAMMA) != 0;
  precision &= ~QE_GAMMA;
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_density: bad precision"); return QE_EINVAL; }
  if (mem != QE_HOST && mem != QE_DEVICE) { set_error("qe_density: bad mem flag"); return QE_EINVAL; }
  for (int c = 0; c < 3; ++c)
    if (grid[c] < 1) { set_error("qe_density: grid must be positive"); return QE_EINVAL; }
  for (int i = 0; i < nk; ++i) {
    if (nbnd[i] < 0) { set_error("qe_density: negative band count at k point %d", i); return QE_EINVAL; }
    if (nbnd[i] > 0 && (!psi[i] || !weights[i])) {
      set_error("qe_density: null psi/weights at k point %d", i);
      return QE_EINVAL;
    }
  }
  DN_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  DN_TRY(ctx_begin(ctx, st));
  const size_t ngrid = (size_t)grid[0] * grid[1] * grid[2];
  // plans first (they validate the grid), so that nothing is queued for a bad call
  std::vector<DevPlan*> plans(nk, nullptr);
  const double zero_k[3] = {0.0, 0.0, 0.0};
  DevPlan* P0 = nullptr;
  DN_TRY(get_plan(ctx, lat, nk > 0 ? kpts : zero_k, ecut, grid, &P0));
  for (int i = 0; i < nk; ++i) DN_TRY(get_plan(ctx, lat, kpts + 3 * i, ecut, grid, &plans[i]));
  // accumulators and the weights of every band (host arrays, copied once)
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
  double* drho = rho;
  if (mem == QE_HOST) {
    DN_TRY(ctx->h_v.ensure(ngrid * sizeof(double)));
    drho = (double*)ctx->h_v.p;
  }
  DN_TRY(launch_density_finish(*P0, acc, kDensGroups, 1.0 / cell_volume(lat), drho, st, &ctx->prof));
  if (mem == QE_HOST) {
    DN_CU(cudaMemcpyAsync(rho, drho, ngrid * sizeof(double), cudaMemcpyDeviceToHost, st));
    DN_CU(cudaStreamSynchronize(st));
  }
  return QE_OK;
}
