// The context behind the opaque qe_ctx handle.
#pragma once

#include <memory>
#include <vector>

#include "plan.h"

struct qe_ctx {
  int device = 0;
  qe::Prof prof;
  std::vector<std::unique_ptr<qe::DevPlan>> plans;
  // H|psi> workspaces
  size_t stick_budget = (size_t)64 << 20;  // stick buffer per band chunk (kept L2-sized)
  qe::DevBuf sticks, vp, part, proj, projd;
  // device copies of host arrays
  qe::DevBuf h_v, h_beta, h_d, h_psi, h_hpsi;
  // Davidson workspaces
  qe::DevBuf dv_basis, dv_hbasis, dv_red, dv_small, dv_vec;
};

namespace qe {

struct OpView {
  int nproj = 0;
  const double* vloc = nullptr;
  const double* beta = nullptr;
  const double* dmat = nullptr;
};

int get_plan(qe_ctx* ctx, const double lat[9], const double k[3], double ecut, const int grid[3],
             DevPlan** out);
int check_problem(const qe_problem* pr, const char* who);
int resolve_operator(qe_ctx* ctx, const qe_problem* pr, const DevPlan& P, OpView& op,
                     cudaStream_t st);
// H psi for nb bands already on the device.
int hpsi_core(qe_ctx* ctx, const DevPlan& P, const OpView& op, int precision, const double* psi,
              double* hpsi, int nb, cudaStream_t st);

}  // namespace qe
