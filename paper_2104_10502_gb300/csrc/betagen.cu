// H|psi> with projectors generated on the fly (the paper's Sec. 3.2.2 item
// (viii), calculation of pseudopotential terms; Sec. 4 names memory per card as
// the bound on system size): instead of a stored beta [nproj][npw] the caller
// gives what defines it -- atom positions, the radial table F_n(|k+G|) of each
// radial function and its angular momentum -- and the library forms
//   beta_{I,n,c}(G) = e^{-i (k+G).R_I} (-i)^{l_n} Y_{l_n c}(k+G) F_n(G)
// where the products need it: straight into the FP64 path's BF16 slices
// (ozgemm.cu, oz_gen_beta), with the structure factor from per-atom, per-axis
// phase tables e^{-i 2 pi m f_Ic} (f the fractional coordinates) and one
// factor e^{-i k.R_I}.  No beta array is stored or read: a C1 call moves the
// 2.2 MB of tables instead of the 281 MB beta (and, from host memory, copies no
// beta at all).
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "plan.h"

namespace qe {

static int gen_setup(qe_ctx* ctx, const DevPlan& P, const qe_problem* pr, const qe_projectors* pj,
                     cudaStream_t st, GenProj& g) {
  const PlanHost& h = P.h;
  g.npw = h.npw;
  g.natom = pj->natom;
  g.nrad = pj->nrad;
  int nper = 0;
  for (int n = 0; n < pj->nrad; ++n) {
    g.l[n] = pj->l[n];
    g.off[n] = nper;
    nper += 2 * pj->l[n] + 1;
  }
  g.nper = nper;
  g.np = nper * pj->natom;
  // signed Miller indices of the sphere (kept per plan)
  if (ctx->gen_mill_plan != &P || !ctx->gen_mill.p) {
    std::vector<int> mill(3 * (size_t)h.npw);
    for (int G = 0; G < h.npw; ++G) {
      const int s = h.g_st[G];
      const int slot[3] = {h.st_x[s], h.st_y[s], h.g_z[G]};
      for (int c = 0; c < 3; ++c)
        mill[3 * (size_t)G + c] = 2 * slot[c] <= h.n[c] ? slot[c] : slot[c] - h.n[c];
    }
    int rc = ctx->gen_mill.ensure(mill.size() * sizeof(int));
    if (rc) return rc;
    if (cudaMemcpyAsync(ctx->gen_mill.p, mill.data(), mill.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("qe_hpsi_gen: upload failed");
      return QE_ECUDA;
    }
    ctx->gen_mill_plan = &P;
  }
  g.mill = (const int*)ctx->gen_mill.p;
  // reciprocal vectors, k, and the phase tables
  reciprocal(pr->lat, g.b);
  std::memcpy(g.k, pr->k, sizeof(g.k));
  int stride = 0;
  for (int c = 0; c < 3; ++c) {
    g.half[c] = h.half[c];
    g.toff[c] = stride;
    stride += 2 * h.half[c] + 1;
  }
  g.tstride = stride;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> tab(2 * ((size_t)stride * pj->natom + pj->natom));
  double* ekr = tab.data() + 2 * (size_t)stride * pj->natom;
  for (int I = 0; I < pj->natom; ++I) {
    const double* R = pj->tau + 3 * I;
    for (int c = 0; c < 3; ++c) {
      // fractional coordinate along a_c: R . b_c / (2 pi)
      const double f = (R[0] * g.b[3 * c] + R[1] * g.b[3 * c + 1] + R[2] * g.b[3 * c + 2]) / two_pi;
      for (int m = -h.half[c]; m <= h.half[c]; ++m) {
        const double ph = -two_pi * m * f;
        double* t = tab.data() + 2 * ((size_t)I * stride + g.toff[c] + m + h.half[c]);
        t[0] = std::cos(ph);
        t[1] = std::sin(ph);
      }
    }
    const double kr = pr->k[0] * R[0] + pr->k[1] * R[1] + pr->k[2] * R[2];
    ekr[2 * I] = std::cos(-kr);
    ekr[2 * I + 1] = std::sin(-kr);
  }
  int rc = ctx->gen_tab.ensure(tab.size() * sizeof(double));
  if (rc) return rc;
  if (cudaMemcpyAsync(ctx->gen_tab.p, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                      st) != cudaSuccess) {
    set_error("qe_hpsi_gen: upload failed");
    return QE_ECUDA;
  }
  g.tab = (const double*)ctx->gen_tab.p;
  g.ekr = (const double*)ctx->gen_tab.p + 2 * (size_t)stride * pj->natom;
  // radial table
  const size_t nrb = (size_t)pj->nrad * h.npw * sizeof(double);
  if (pr->mem == QE_HOST) {
    if ((rc = ctx->gen_rad.ensure(std::max<size_t>(nrb, 8)))) return rc;
    if (nrb && cudaMemcpyAsync(ctx->gen_rad.p, pj->radial, nrb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("qe_hpsi_gen: upload failed");
      return QE_ECUDA;
    }
    g.radial = (const double*)ctx->gen_rad.p;
  } else {
    g.radial = pj->radial;
  }
  return QE_OK;
}

}  // namespace qe

using namespace qe;

#define BG_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define BG_CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error("%s: %s", #x, cudaGetErrorString(e_)); return QE_ECUDA; } } while (0)

extern "C" int qe_hpsi_gen(qe_ctx* ctx, const qe_problem* prob, const qe_projectors* pj,
                           int precision, const double* psi, double* hpsi, void* stream) {
  clear_error();
  if (!ctx || !prob || !pj) { set_error("qe_hpsi_gen: null argument"); return QE_EINVAL; }
  if (prob->mem != QE_HOST && prob->mem != QE_DEVICE) { set_error("qe_hpsi_gen: bad mem flag"); return QE_EINVAL; }
  if (prob->nbnd < 0 || !prob->vloc_r) { set_error("qe_hpsi_gen: invalid problem"); return QE_EINVAL; }
  for (int c = 0; c < 3; ++c)
    if (prob->grid[c] < 1) { set_error("qe_hpsi_gen: grid must be positive"); return QE_EINVAL; }
  if (pj->natom < 0 || pj->nrad < 0 || pj->nrad > kGenMaxRad || (pj->natom > 0 && !pj->tau) ||
      (pj->nrad > 0 && (!pj->l || !pj->radial))) {
    set_error("qe_hpsi_gen: invalid projector description (at most %d radial functions)", kGenMaxRad);
    return QE_EINVAL;
  }
  int nper = 0;
  for (int n = 0; n < pj->nrad; ++n) {
    if (pj->l[n] != 0 && pj->l[n] != 1) { set_error("qe_hpsi_gen: l must be 0 or 1"); return QE_EINVAL; }
    nper += 2 * pj->l[n] + 1;
  }
  if (prob->nproj != nper * pj->natom) {
    set_error("qe_hpsi_gen: nproj %d, but the projectors described number %d", prob->nproj,
              nper * pj->natom);
    return QE_EINVAL;
  }
  if (prob->nproj > 0 && !prob->dmat) { set_error("qe_hpsi_gen: dmat is null"); return QE_EINVAL; }
  const bool pair = (precision & QE_GAMMA) != 0;
  const bool fp64_pipe = (precision & QE_FFT_FP64PIPE) != 0;
  precision &= ~(QE_GAMMA | QE_FFT_FP64PIPE);
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_hpsi_gen: bad precision"); return QE_EINVAL; }
  const int nb = prob->nbnd;
  if (nb > 0 && (!psi || !hpsi)) { set_error("qe_hpsi_gen: null psi/hpsi"); return QE_EINVAL; }
  BG_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  BG_TRY(ctx_begin(ctx, st));
  DevPlan* P = nullptr;
  BG_TRY(get_plan(ctx, prob->lat, prob->k, prob->ecutwfc, prob->grid, &P));
  const size_t ngrid = (size_t)P->grid[0] * P->grid[1] * P->grid[2];
  const size_t nel = (size_t)nb * P->h.npw * 2;
  // operator: V and D (copied when they are host arrays), beta generated
  OpView op;
  op.nproj = prob->nproj;
  op.tag = ++ctx->op_tag;
  const double* dpsi = psi;
  double* dhpsi = hpsi;
  if (prob->mem == QE_HOST) {
    const size_t nd = (size_t)prob->nproj * prob->nproj;
    BG_TRY(ctx->h_v.ensure(ngrid * sizeof(double)));
    BG_TRY(ctx->h_d.ensure(std::max<size_t>(nd, 1) * sizeof(double)));
    BG_CU(cudaMemcpyAsync(ctx->h_v.p, prob->vloc_r, ngrid * sizeof(double), cudaMemcpyHostToDevice, st));
    if (nd) BG_CU(cudaMemcpyAsync(ctx->h_d.p, prob->dmat, nd * sizeof(double), cudaMemcpyHostToDevice, st));
    op.vloc = (const double*)ctx->h_v.p;
    op.dmat = (const double*)ctx->h_d.p;
    if (nb > 0) {
      BG_TRY(ctx->h_psi.ensure(nel * sizeof(double)));
      BG_TRY(ctx->h_hpsi.ensure(nel * sizeof(double)));
      BG_CU(cudaMemcpyAsync(ctx->h_psi.p, psi, nel * sizeof(double), cudaMemcpyHostToDevice, st));
      dpsi = (const double*)ctx->h_psi.p;
      dhpsi = (double*)ctx->h_hpsi.p;
    }
  } else {
    op.vloc = prob->vloc_r;
    op.dmat = prob->dmat;
  }
  GenProj g;
  BG_TRY(gen_setup(ctx, *P, prob, pj, st, g));
  op.gen = &g;
  ctx->last_op = qe_ctx::LastOp{};   // the prepared operator forms are this call's
  BG_TRY(hpsi_core(ctx, *P, op, precision, dpsi, dhpsi, nb, st, pair, fp64_pipe));
  if (prob->mem == QE_HOST) {
    if (nb > 0) BG_CU(cudaMemcpyAsync(hpsi, dhpsi, nel * sizeof(double), cudaMemcpyDeviceToHost, st));
    BG_CU(cudaStreamSynchronize(st));
    BG_TRY(tc_check(ctx, st));
  }
  return QE_OK;
}
