// H|psi> for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a memory
// pool or arena owned by someone else, under a framework's allocator that must
// see every allocation, or at a point where a device allocation would
// synchronise the device or fail (for example while another component holds
// all free memory).  qe_hpsi needs workspace (the stick buffer of the FFT, the
// permuted potential, the split-K partial sums, the projections) and takes it
// from the context's grow-only buffers, which allocate on first use.  The entry
// point in this file instead takes every byte of workspace from one fixed,
// file-scope device array of kNoAllocBytes (64 MiB) that the CUDA runtime
// places when the library's module is loaded on a GPU; every GPU that loads
// the library holds that array until the process exits.
//
// The caller still owns and passes the inputs (psi, V_loc, beta, D) and the
// output (hpsi), all in device memory.  Nothing here calls cudaMalloc,
// cudaFree or any allocating library routine; host-side set-up (the sphere and
// its maps) uses ordinary host memory.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ctx.h"
#include "plan.h"

namespace qe {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static std::vector<void*> g_noalloc_addr;   // device address of the array, per device

// The plan (sphere maps, twiddles, digit reversals) that the array holds on
// each device: a call with the same cell, k, cut-off and grid finds it there
// and copies nothing from the host.
struct NoallocPlanKey {
  bool valid = false;
  double lat[9], k[3], ecut;
  int grid[3];
  bool same(const qe_problem* pr) const {
    return valid && std::memcmp(lat, pr->lat, sizeof(lat)) == 0 &&
           std::memcmp(k, pr->k, sizeof(k)) == 0 && ecut == pr->ecutwfc &&
           std::memcmp(grid, pr->grid, sizeof(grid)) == 0;
  }
};
static std::vector<NoallocPlanKey> g_noalloc_plan;   // per device

// Once per device, with that device current: the array's device address.  The
// host-side symbol is only a stand-in and must never be handed to a kernel.
static int noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if ((int)g_noalloc_addr.size() <= dev) g_noalloc_addr.resize(dev + 1, nullptr);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("qe_hpsi_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return QE_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return QE_OK;
}

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
static int hpsi_noalloc_impl(const qe_problem* pr, const double* psi, double* hpsi,
                             cudaStream_t st, unsigned char* base, int dev) {
  DevPlan P;   // device pointers below point into the fixed array; P.block stays null
  std::memcpy(P.lat, pr->lat, sizeof(P.lat));
  std::memcpy(P.k, pr->k, sizeof(P.k));
  P.ecut = pr->ecutwfc;
  std::memcpy(P.grid, pr->grid, sizeof(P.grid));
  int rc = build_plan_host(pr->lat, pr->k, pr->ecutwfc, pr->grid, P.h);
  if (rc) return rc;
  const PlanHost& h = P.h;
  std::vector<int> perm[3];
  std::vector<double> tw[3];
  for (int c = 0; c < 3; ++c) {
    make_radix(P.grid[c], P.rad[c]);
    perm[c] = digit_reversal(P.rad[c]);
    tw[c] = twiddles(P.grid[c]);
  }
  P.sq = sq_plane_size(P.grid);
  if (P.sq) perm[0] = perm[1] = sq_order(P.sq);
  P.sqz = sq_line_size(P.grid[2]);
  if (P.sqz) perm[2] = sq_order(P.sqz);
  const int nb = pr->nbnd, np = pr->nproj, npw = h.npw;
  const size_t ngrid = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  // layout: plan image | permuted V | projections x2 | stick buffer | split-K partials
  size_t nd = h.npw;
  for (int c = 0; c < 3; ++c) nd += tw[c].size();
  size_t ni = (h.nst + 1) + 3 * (size_t)h.npw + 2 * (size_t)h.nst + h.nax;
  for (int c = 0; c < 3; ++c) ni += P.grid[c];
  const size_t plan_bytes = up256(nd * sizeof(double) + ni * sizeof(int));
  const size_t vp_bytes = up256(ngrid * sizeof(T));
  const size_t proj_bytes = up256((size_t)np * nb * 2 * sizeof(double));
  const size_t per_band = stick_bytes(P, 1, 2 * sizeof(T));
  const size_t one_split = np > 0 ? up256((size_t)np * nb * 2 * sizeof(T)) : 0;
  const size_t fixed = plan_bytes + vp_bytes + 2 * proj_bytes;
  const size_t need = fixed + up256(per_band) + one_split + 256;
  if (need > kNoAllocBytes) {
    set_error("qe_hpsi_noalloc: problem needs %zu bytes of workspace, the fixed array holds %zu "
              "(use qe_hpsi)", need, kNoAllocBytes);
    return QE_EINVAL;
  }
  const size_t room = kNoAllocBytes - fixed - one_split - 256;
  int nbc = (int)std::min<size_t>(room / per_band, ((size_t)64 << 20) / per_band);
  nbc = std::max(1, std::min(nbc, nb));
  const size_t stick_sz = up256((size_t)nbc * per_band);
  unsigned char* p_plan = base;
  T* vp = reinterpret_cast<T*>(base + plan_bytes);
  double* proj = reinterpret_cast<double*>(base + plan_bytes + vp_bytes);
  double* projd = reinterpret_cast<double*>(base + plan_bytes + vp_bytes + proj_bytes);
  void* sticks = base + fixed;
  void* part = base + fixed + stick_sz;
  const size_t part_bytes = kNoAllocBytes - fixed - stick_sz;

  // plan image: doubles first, then ints (same order as the context's plans)
  std::vector<char> img(plan_bytes, 0);
  double* dp = reinterpret_cast<double*>(img.data());
  size_t od = 0;
  auto put_d = [&](const double* s, size_t n) { std::memcpy(dp + od, s, n * sizeof(double)); size_t o = od; od += n; return o; };
  const size_t o_kin = put_d(h.kin.data(), h.npw);
  size_t o_tw[3];
  for (int c = 0; c < 3; ++c) o_tw[c] = put_d(tw[c].data(), tw[c].size());
  int* ip = reinterpret_cast<int*>(img.data() + nd * sizeof(double));
  size_t oi = 0;
  auto put_i = [&](const int* s, size_t n) { std::memcpy(ip + oi, s, n * sizeof(int)); size_t o = oi; oi += n; return o; };
  const size_t o_ptr = put_i(h.st_ptr.data(), h.nst + 1);
  const size_t o_g = put_i(h.st_g.data(), h.npw);
  const size_t o_z = put_i(h.st_z.data(), h.npw);
  const size_t o_of = put_i(h.st_of.data(), h.npw);
  const size_t o_x = put_i(h.st_x.data(), h.nst);
  const size_t o_y = put_i(h.st_y.data(), h.nst);
  const size_t o_ax = put_i(h.ax.data(), h.nax);
  size_t o_perm[3];
  for (int c = 0; c < 3; ++c) o_perm[c] = put_i(perm[c].data(), perm[c].size());
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_plan.size() <= dev) g_noalloc_plan.resize(dev + 1);
    NoallocPlanKey& key = g_noalloc_plan[dev];
    if (!key.same(pr)) {
      key.valid = false;
      cudaError_t e = cudaMemcpyAsync(p_plan, img.data(), plan_bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) {
        set_error("qe_hpsi_noalloc: plan upload: %s", cudaGetErrorString(e));
        return QE_ECUDA;
      }
      std::memcpy(key.lat, pr->lat, sizeof(key.lat));
      std::memcpy(key.k, pr->k, sizeof(key.k));
      key.ecut = pr->ecutwfc;
      std::memcpy(key.grid, pr->grid, sizeof(key.grid));
      key.valid = true;
    }
  }
  double* dd = reinterpret_cast<double*>(p_plan);
  int* di = reinterpret_cast<int*>(p_plan + nd * sizeof(double));
  P.kin = dd + o_kin;
  for (int c = 0; c < 3; ++c) { P.tw[c] = dd + o_tw[c]; P.perm[c] = di + o_perm[c]; }
  P.st_ptr = di + o_ptr;
  P.st_g = di + o_g;
  P.st_z = di + o_z;
  P.st_of = di + o_of;
  P.st_x = di + o_x;
  P.st_y = di + o_y;
  P.ax = di + o_ax;

  rc = launch_vperm<T>(P, pr->vloc_r, vp, st, nullptr);
  if (rc) return rc;
  for (int b0 = 0; b0 < nb; b0 += nbc) {
    rc = launch_local_kinetic<T>(P, psi, hpsi, vp, sticks, b0, std::min(nbc, nb - b0), st, nullptr);
    if (rc) return rc;
  }
  if (np > 0) {
    rc = gemm_inner_bounded<GemmT<T>>(pr->beta, npw, psi, npw, np, nb, npw, proj, nb, part,
                                      part_bytes, st, nullptr);
    if (rc) return rc;
    rc = dmul(pr->dmat, proj, projd, np, nb, st, nullptr);
    if (rc) return rc;
    rc = gemm_outer<GemmT<T>>(pr->beta, npw, projd, nb, npw, nb, np, hpsi, npw, 1, st, nullptr);
    if (rc) return rc;
  }
  return QE_OK;
}

}  // namespace qe

extern "C" int qe_hpsi_noalloc(const qe_problem* prob, int precision, const double* psi,
                               double* hpsi, void* stream) {
  qe::clear_error();
  int rc = qe::check_problem(prob, "qe_hpsi_noalloc");
  if (rc) return rc;
  if (prob->mem != QE_DEVICE) {
    qe::set_error("qe_hpsi_noalloc: every array must be device memory (mem = QE_DEVICE)");
    return QE_EINVAL;
  }
  if (precision != QE_FP64 && precision != QE_MIXED) {
    qe::set_error("qe_hpsi_noalloc: bad precision");
    return QE_EINVAL;
  }
  if (prob->nbnd == 0) return QE_OK;
  if (!psi || !hpsi) {
    qe::set_error("qe_hpsi_noalloc: null psi/hpsi");
    return QE_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    qe::set_error("qe_hpsi_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return QE_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Under capture the plan check below would run once, at capture time, while
  // the graph may be replayed after other calls replaced the array's plan.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    qe::set_error("qe_hpsi_noalloc: cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    return QE_ECUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) {
    qe::set_error("qe_hpsi_noalloc: not callable while the stream is being captured");
    return QE_EINVAL;
  }
  void* base = nullptr;
  rc = qe::noalloc_scratch(dev, &base);
  if (rc) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  if (precision == QE_FP64) return qe::hpsi_noalloc_impl<qe::FftF64>(prob, psi, hpsi, st, b, dev);
  return qe::hpsi_noalloc_impl<float>(prob, psi, hpsi, st, b, dev);
}
