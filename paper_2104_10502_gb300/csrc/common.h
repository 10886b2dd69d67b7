// Internal declarations shared by the translation units of libqegb.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "qegb.h"

namespace qe {

// ---- errors -----------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

// ---- plane-wave sphere (host, float64, no contraction) ------------------------
struct Sphere {
  int npw = 0;
  std::vector<int> miller;   // [npw][3]
  std::vector<double> kin;   // |k+G|^2
};
void reciprocal(const double lat[9], double b[9]);
double cell_volume(const double lat[9]);
int build_sphere(const double lat[9], const double k[3], double ecut, Sphere& out);

// ---- mixed-radix plans for one FFT axis ---------------------------------------
constexpr int kMaxStages = 16;
constexpr int kMaxFftLen = 1024;
struct Radix {
  int n = 0;
  int nst = 0;
  int r[kMaxStages];   // radix of stage s (DIF order)
  int L[kMaxStages];   // sub-transform length entering stage s
};
// Factor n into radices 4, 2, 3, 5 (in that order).  False if n has another factor.
bool make_radix(int n, Radix& out);
// perm[p] = natural index held at stored position p after the DIF stages.
std::vector<int> digit_reversal(const Radix& rp);
// table[t] = exp(-2 pi i t / n), t < n, interleaved (re, im), then the same
// twiddles as (cos, tan) pairs at table[n + t] (quarter turns: (2^-60, +-2^60))
std::vector<double> twiddles(int n);

// ---- host-side plan (maps of the sphere onto sticks and planes) --------------
struct PlanHost {
  int npw = 0, nst = 0, nax = 0;
  int n[3] = {0, 0, 0};
  int half[3] = {0, 0, 0};        // max |Miller index| of the sphere per axis
  std::vector<double> kin;        // [npw]
  std::vector<int> st_ptr;        // [nst + 1] CSR over sticks
  std::vector<int> st_g;          // [npw] sphere index, stick-major
  std::vector<int> st_z;          // [npw] z slot (natural)
  std::vector<int> st_of;         // [npw] stick of CSR entry
  std::vector<int> st_x, st_y;    // [nst] natural x and y slots of each stick
  std::vector<int> ax;            // [nax] x slots holding at least one stick
  std::vector<int> g_st;          // [npw] stick of plane wave g
  std::vector<int> g_z;           // [npw] natural z slot of plane wave g
  // k = 0: the sphere is symmetric under G -> -G.  gamma = 1 when the sticks
  // are ordered in mirror pairs (2i, 2i+1) = ((x, y), (-x, -y)) with the
  // self-mirror stick (0, 0) last; mg[g] is the sphere index of -G.
  int gamma = 0;
  std::vector<int> mg;            // [npw] when gamma
};
int build_plan_host(const double lat[9], const double k[3], double ecut,
                    const int grid[3], PlanHost& out);

}  // namespace qe
