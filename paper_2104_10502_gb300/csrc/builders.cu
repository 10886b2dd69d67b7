// Synthetic pseudopotential terms on the GPU (Sec. 3.2.2 item (viii) of the
// paper, "calculation of pseudopotential terms"): a Gaussian local potential
// sampled on the FFT grid and Gaussian-times-solid-harmonic Kleinman-Bylander
// projectors in the plane-wave basis.  Definitions are in qegb.h.
#include <cmath>
#include <vector>

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

struct Lat { double a[9]; };

__global__ void k_vloc(int n1, int n2, int n3, Lat L, const double* __restrict__ tau, int natom,
                       double amp, double inv2s2, double* __restrict__ v) {
  const size_t total = (size_t)n1 * n2 * n3;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j0 = (int)(i % n1), j1 = (int)((i / n1) % n2), j2 = (int)(i / ((size_t)n1 * n2));
    const double f0 = (double)j0 / n1, f1 = (double)j1 / n2, f2 = (double)j2 / n3;
    double r[3];
    for (int c = 0; c < 3; ++c) r[c] = f0 * L.a[c] + f1 * L.a[3 + c] + f2 * L.a[6 + c];
    double s = 0.0;
    for (int I = 0; I < natom; ++I) {
      for (int t0 = -1; t0 <= 1; ++t0)
        for (int t1 = -1; t1 <= 1; ++t1)
          for (int t2 = -1; t2 <= 1; ++t2) {
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
              const double d = r[c] - tau[3 * I + c] - (t0 * L.a[c] + t1 * L.a[3 + c] + t2 * L.a[6 + c]);
              d2 += d * d;
            }
            s += exp(-d2 * inv2s2);
          }
    }
    v[i] = amp * s;
  }
}

// One thread per (plane wave, atom): writes the 4 * nrad projectors of the atom.
__global__ void k_beta(const double* __restrict__ q, int npw, const double* __restrict__ tau,
                       int natom, const double* __restrict__ widths, int nrad, double pref,
                       double* __restrict__ beta) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = blockIdx.y;
  if (g >= npw) return;
  const double qx = q[3 * g], qy = q[3 * g + 1], qz = q[3 * g + 2];
  const double q2 = qx * qx + qy * qy + qz * qz;
  const double qr = qx * tau[3 * I] + qy * tau[3 * I + 1] + qz * tau[3 * I + 2];
  double sn, cs;
  sincos(qr, &sn, &cs);            // e^{-i q.R} = cs - i sn
  const double sqpi = 1.7724538509055160273;   // sqrt(pi)
  const double y00 = 0.28209479177387814347;   // 1 / (2 sqrt(pi))
  const double y1 = 0.48860251190291992159;    // sqrt(3 / (4 pi))
  for (int n = 0; n < nrad; ++n) {
    const double w = widths[n];
    const double gw = exp(-0.5 * w * w * q2);
    const double n0 = sqrt(4.0 / (sqpi * w * w * w));
    const double n1 = sqrt(8.0 / (3.0 * sqpi * w * w * w * w * w));
    const int row = (I * nrad + n) * 4;
    // s: real amplitude times e^{-i q.R}
    const double as = pref * n0 * w * w * w * y00 * gw;
    double2* b = reinterpret_cast<double2*>(beta);
    b[(size_t)row * npw + g] = make_double2(as * cs, -as * sn);
    // p: (-i) amplitude q_c times e^{-i q.R}:  (-i)(cs - i sn) = -sn - i cs
    const double ap = pref * n1 * w * w * w * w * w * y1 * gw;
    const double qc[3] = {qx, qy, qz};
    for (int c = 0; c < 3; ++c) {
      const double a = ap * qc[c];
      b[(size_t)(row + 1 + c) * npw + g] = make_double2(-a * sn, -a * cs);
    }
  }
}

int build_vloc(const double lat[9], const int grid[3], int natom, const double* tau_h, double amp,
               double sigma, double* v_dev, cudaStream_t st) {
  double* tau_d = nullptr;
  if (natom > 0) {
    if (cudaMallocAsync(&tau_d, sizeof(double) * 3 * natom, st) != cudaSuccess) {
      cudaGetLastError();
      set_error("qe_vloc_gaussian: cudaMallocAsync failed");
      return QE_ENOMEM;
    }
    cudaMemcpyAsync(tau_d, tau_h, sizeof(double) * 3 * natom, cudaMemcpyHostToDevice, st);
  }
  Lat L;
  for (int i = 0; i < 9; ++i) L.a[i] = lat[i];
  const size_t total = (size_t)grid[0] * grid[1] * grid[2];
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
  k_vloc<<<blocks, 256, 0, st>>>(grid[0], grid[1], grid[2], L, tau_d, natom, amp,
                                 1.0 / (2.0 * sigma * sigma), v_dev);
  int rc = check_launch("k_vloc");
  cudaStreamSynchronize(st);
  if (tau_d) cudaFreeAsync(tau_d, st);
  return rc;
}

int build_beta(const double lat[9], const double k[3], double ecut, int natom, const double* tau_h,
               int nrad, const double* widths_h, double* beta_dev, int* npw_out, cudaStream_t st) {
  Sphere S;
  int rc = build_sphere(lat, k, ecut, S);
  if (rc) return rc;
  double b[9];
  reciprocal(lat, b);
  std::vector<double> q(3 * (size_t)S.npw);
  for (int i = 0; i < S.npw; ++i)
    for (int c = 0; c < 3; ++c)
      q[3 * i + c] = k[c] + S.miller[3 * i] * b[c] + S.miller[3 * i + 1] * b[3 + c] +
                     S.miller[3 * i + 2] * b[6 + c];
  *npw_out = S.npw;
  if (natom == 0 || nrad == 0) return QE_OK;
  double *q_d = nullptr, *tau_d = nullptr, *w_d = nullptr;
  const size_t nb = sizeof(double) * (q.size() + 3 * (size_t)natom + nrad);
  void* blk = nullptr;
  if (cudaMallocAsync(&blk, nb, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("qe_beta_gaussian: cudaMallocAsync failed");
    return QE_ENOMEM;
  }
  q_d = (double*)blk;
  tau_d = q_d + q.size();
  w_d = tau_d + 3 * (size_t)natom;
  cudaMemcpyAsync(q_d, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(tau_d, tau_h, sizeof(double) * 3 * natom, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(w_d, widths_h, sizeof(double) * nrad, cudaMemcpyHostToDevice, st);
  const double pref = pow(2.0 * M_PI, 1.5) / sqrt(cell_volume(lat));
  dim3 g((S.npw + 127) / 128, natom);
  k_beta<<<g, 128, 0, st>>>(q_d, S.npw, tau_d, natom, w_d, nrad, pref, beta_dev);
  rc = check_launch("k_beta");
  cudaStreamSynchronize(st);
  cudaFreeAsync(blk, st);
  return rc;
}

}  // namespace qe
