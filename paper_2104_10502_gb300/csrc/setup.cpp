// Host-side set-up: plane-wave sphere, stick/plane maps, FFT radix plans.
//
// The sphere is the plane-wave basis of Sec. 3.2.2 item (vi) of the paper
// ("generation of plane waves and of their mapping to FFT grids").  This file
// must be compiled without floating-point contraction (-ffp-contract=off): the
// order of the plane waves is decided by a float64 value whose exact evaluation
// is part of the interface (see qe_gsphere in qegb.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <tuple>

#include "common.h"

namespace qe {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

static const double kTwoPi = 2.0 * 3.14159265358979323846;

static void cross(const double* u, const double* v, double* c) {
  c[0] = u[1] * v[2] - u[2] * v[1];
  c[1] = u[2] * v[0] - u[0] * v[2];
  c[2] = u[0] * v[1] - u[1] * v[0];
}

double cell_volume(const double lat[9]) {
  double c[3];
  cross(lat + 3, lat + 6, c);
  return std::fabs((lat[0] * c[0] + lat[1] * c[1]) + lat[2] * c[2]);
}

void reciprocal(const double lat[9], double b[9]) {
  double c1[3], c2[3], c3[3];
  cross(lat + 3, lat + 6, c1);
  cross(lat + 6, lat + 0, c2);
  cross(lat + 0, lat + 3, c3);
  const double vol = (lat[0] * c1[0] + lat[1] * c1[1]) + lat[2] * c1[2];
  const double fac = kTwoPi / vol;
  for (int c = 0; c < 3; ++c) {
    b[0 + c] = c1[c] * fac;
    b[3 + c] = c2[c] * fac;
    b[6 + c] = c3[c] * fac;
  }
}

int build_sphere(const double lat[9], const double k[3], double ecut, Sphere& out) {
  if (!(ecut > 0.0) || !std::isfinite(ecut)) {
    set_error("qe_gsphere: ecut must be positive and finite");
    return QE_EINVAL;
  }
  if (cell_volume(lat) <= 0.0) {
    set_error("qe_gsphere: singular lattice");
    return QE_EINVAL;
  }
  double b[9];
  reciprocal(lat, b);
  const double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  const double gmax = std::sqrt(ecut) + kn;
  int lim[3];
  for (int i = 0; i < 3; ++i) {
    const double an = std::sqrt(lat[3 * i] * lat[3 * i] + lat[3 * i + 1] * lat[3 * i + 1] +
                                lat[3 * i + 2] * lat[3 * i + 2]);
    lim[i] = (int)std::floor(gmax * an / kTwoPi) + 1;
    if (lim[i] > 4096) {
      set_error("qe_gsphere: sphere too large (|m_%d| up to %d)", i + 1, lim[i]);
      return QE_EINVAL;
    }
  }
  const double thr = ecut * (1.0 + 1e-12);
  struct E { double kin; int m1, m2, m3; };
  std::vector<E> v;
  for (int m1 = -lim[0]; m1 <= lim[0]; ++m1)
    for (int m2 = -lim[1]; m2 <= lim[1]; ++m2)
      for (int m3 = -lim[2]; m3 <= lim[2]; ++m3) {
        double q[3];
        for (int c = 0; c < 3; ++c)
          q[c] = ((k[c] + (double)m1 * b[0 + c]) + (double)m2 * b[3 + c]) + (double)m3 * b[6 + c];
        const double kin = (q[0] * q[0] + q[1] * q[1]) + q[2] * q[2];
        if (kin <= thr) v.push_back({kin, m1, m2, m3});
      }
  std::sort(v.begin(), v.end(), [](const E& a, const E& b2) {
    return std::tie(a.kin, a.m1, a.m2, a.m3) < std::tie(b2.kin, b2.m1, b2.m2, b2.m3);
  });
  out.npw = (int)v.size();
  out.miller.resize(3 * v.size());
  out.kin.resize(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    out.miller[3 * i] = v[i].m1;
    out.miller[3 * i + 1] = v[i].m2;
    out.miller[3 * i + 2] = v[i].m3;
    out.kin[i] = v[i].kin;
  }
  return QE_OK;
}

bool make_radix(int n, Radix& out) {
  out = Radix();
  out.n = n;
  if (n < 1 || n > kMaxFftLen) return false;
  int m = n;
  while (m % 4 == 0) { out.r[out.nst++] = 4; m /= 4; }
  for (int p : {2, 3, 5})
    while (m % p == 0) { out.r[out.nst++] = p; m /= p; }
  if (m != 1) return false;
  int L = n;
  for (int s = 0; s < out.nst; ++s) { out.L[s] = L; L /= out.r[s]; }
  return true;
}

std::vector<int> digit_reversal(const Radix& rp) {
  std::vector<int> perm(rp.n);
  for (int k = 0; k < rp.n; ++k) {
    int pos = 0, base = 1;
    for (int s = 0; s < rp.nst; ++s) {
      const int q = (k / base) % rp.r[s];
      base *= rp.r[s];
      pos += q * (rp.L[s] / rp.r[s]);
    }
    perm[pos] = k;
  }
  return perm;
}

std::vector<double> twiddles(int n) {
  std::vector<double> t(4 * (size_t)n);
  const long double pi = 3.141592653589793238462643383279502884L;
  const double q = 0x1p-60;
  for (int j = 0; j < n; ++j) {
    const long double a = -2.0L * pi * (long double)j / (long double)n;
    const long double c = cosl(a), s = sinl(a);
    t[2 * j] = (double)c;
    t[2 * j + 1] = (double)s;
    // (cos a, tan a); a quarter turn (|c| below any other angle's 2 pi / n) as
    // (2^-60, +-2^60)
    const bool quarter = fabsl(c) < 1e-9L;
    t[2 * (size_t)n + 2 * j] = quarter ? q : (double)c;
    t[2 * (size_t)n + 2 * j + 1] = quarter ? (s > 0 ? 1.0 / q : -1.0 / q) : (double)(s / c);
  }
  return t;
}

static inline int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

int build_plan_host(const double lat[9], const double k[3], double ecut,
                    const int grid[3], PlanHost& P) {
  Sphere S;
  int rc = build_sphere(lat, k, ecut, S);
  if (rc) return rc;
  if (S.npw == 0) { set_error("empty plane-wave sphere"); return QE_EINVAL; }
  int mx[3] = {0, 0, 0};
  for (int i = 0; i < S.npw; ++i)
    for (int c = 0; c < 3; ++c) mx[c] = std::max(mx[c], std::abs(S.miller[3 * i + c]));
  for (int c = 0; c < 3; ++c) {
    if (grid[c] < 2 * mx[c] + 1) {
      set_error("grid axis %d: %d < %d (= 2 max|m| + 1)", c + 1, grid[c], 2 * mx[c] + 1);
      return QE_EINVAL;
    }
    Radix r;
    if (!make_radix(grid[c], r)) {
      set_error("grid axis %d: %d is not a product of 2, 3, 5 up to %d", c + 1, grid[c], kMaxFftLen);
      return QE_EINVAL;
    }
    P.n[c] = grid[c];
    P.half[c] = mx[c];
  }
  P.npw = S.npw;
  P.kin = S.kin;
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  // sticks: distinct (x, y) slots, ordered by x then y
  std::vector<long long> keys(S.npw);
  for (int i = 0; i < S.npw; ++i) {
    const int x = pmod(S.miller[3 * i], n1), y = pmod(S.miller[3 * i + 1], n2);
    keys[i] = (long long)x * n2 + y;
  }
  std::vector<long long> uk(keys);
  std::sort(uk.begin(), uk.end());
  uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
  // At k = 0 the sphere is symmetric under G -> -G: order the sticks in mirror
  // pairs, (x, y) next to (-x, -y), the self-mirror stick (0, 0) last, so that
  // a z tile of an even number of sticks holds both halves of every pair.
  std::vector<long long> order(uk);
  P.gamma = 0;
  if (k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0) {
    auto mirror = [&](long long key) {
      const int x = (int)(key / n2), y = (int)(key % n2);
      return (long long)((n1 - x) % n1) * n2 + (n2 - y) % n2;
    };
    std::vector<char> used(uk.size(), 0);
    std::vector<long long> ord;
    long long self = -1;
    bool ok = true;
    for (size_t s = 0; s < uk.size() && ok; ++s) {
      if (used[s]) continue;
      const long long m = mirror(uk[s]);
      if (m == uk[s]) {
        if (self >= 0) ok = false;
        self = uk[s];
        used[s] = 1;
        continue;
      }
      const auto it = std::lower_bound(uk.begin(), uk.end(), m);
      if (it == uk.end() || *it != m || used[it - uk.begin()]) { ok = false; break; }
      used[s] = used[it - uk.begin()] = 1;
      ord.push_back(uk[s]);
      ord.push_back(m);
    }
    if (ok && self >= 0) {
      ord.push_back(self);
      order = ord;
      P.gamma = 1;
    }
  }
  std::vector<int> pos(uk.size());   // sorted index -> stick index
  for (size_t s = 0; s < order.size(); ++s)
    pos[std::lower_bound(uk.begin(), uk.end(), order[s]) - uk.begin()] = (int)s;
  P.nst = (int)uk.size();
  P.st_x.resize(P.nst);
  P.st_y.resize(P.nst);
  for (int s = 0; s < P.nst; ++s) { P.st_x[s] = (int)(order[s] / n2); P.st_y[s] = (int)(order[s] % n2); }
  P.g_st.resize(S.npw);
  P.g_z.resize(S.npw);
  std::vector<int> cnt(P.nst + 1, 0);
  for (int i = 0; i < S.npw; ++i) {
    const int s = pos[std::lower_bound(uk.begin(), uk.end(), keys[i]) - uk.begin()];
    P.g_st[i] = s;
    P.g_z[i] = pmod(S.miller[3 * i + 2], n3);
    cnt[s + 1]++;
  }
  P.st_ptr.assign(P.nst + 1, 0);
  for (int s = 0; s < P.nst; ++s) P.st_ptr[s + 1] = P.st_ptr[s] + cnt[s + 1];
  P.st_g.resize(S.npw);
  P.st_z.resize(S.npw);
  P.st_of.resize(S.npw);
  std::vector<int> fill(P.st_ptr.begin(), P.st_ptr.end() - 1);
  for (int i = 0; i < S.npw; ++i) {
    const int s = P.g_st[i];
    const int e = fill[s]++;
    P.st_g[e] = i;
    P.st_z[e] = P.g_z[i];
    P.st_of[e] = s;
  }
  // active x columns, ascending (from the x-sorted stick keys)
  P.ax.clear();
  for (const long long key : uk) {
    const int x = (int)(key / n2);
    if (P.ax.empty() || P.ax.back() != x) P.ax.push_back(x);
  }
  P.nax = (int)P.ax.size();
  if (P.gamma) {
    // sphere index of -G for every G (Miller indices in a dense box)
    const int bx = 2 * mx[0] + 1, by = 2 * mx[1] + 1, bz = 2 * mx[2] + 1;
    std::vector<int> at((size_t)bx * by * bz, -1);
    auto cell = [&](int a, int b, int c) { return ((size_t)(a + mx[0]) * by + (b + mx[1])) * bz + (c + mx[2]); };
    for (int i = 0; i < S.npw; ++i) at[cell(S.miller[3 * i], S.miller[3 * i + 1], S.miller[3 * i + 2])] = i;
    P.mg.resize(S.npw);
    for (int i = 0; i < S.npw; ++i) {
      const int j = at[cell(-S.miller[3 * i], -S.miller[3 * i + 1], -S.miller[3 * i + 2])];
      if (j < 0) { P.gamma = 0; P.mg.clear(); break; }
      P.mg[i] = j;
    }
  }
  return QE_OK;
}

}  // namespace qe

extern "C" {

const char* qe_last_error(void) { return qe::g_err.c_str(); }

int qe_gsphere(const double lat[9], const double k[3], double ecut, const int grid[3],
               int* npw, int* miller, double* kin) {
  qe::clear_error();
  if (!lat || !k || !npw) { qe::set_error("qe_gsphere: null argument"); return QE_EINVAL; }
  qe::Sphere S;
  int rc = qe::build_sphere(lat, k, ecut, S);
  if (rc) return rc;
  if (grid) {
    for (int c = 0; c < 3; ++c) {
      int mx = 0;
      for (int i = 0; i < S.npw; ++i) mx = std::max(mx, std::abs(S.miller[3 * i + c]));
      if (grid[c] < 2 * mx + 1) {
        qe::set_error("qe_gsphere: grid axis %d: %d < %d", c + 1, grid[c], 2 * mx + 1);
        return QE_EINVAL;
      }
    }
  }
  if (!miller) { *npw = S.npw; return QE_OK; }
  if (*npw < S.npw) {
    qe::set_error("qe_gsphere: buffer holds %d plane waves, %d needed", *npw, S.npw);
    return QE_EINVAL;
  }
  *npw = S.npw;
  std::memcpy(miller, S.miller.data(), sizeof(int) * 3 * (size_t)S.npw);
  if (kin) std::memcpy(kin, S.kin.data(), sizeof(double) * (size_t)S.npw);
  return QE_OK;
}

}  // extern "C"
