// Autotuner of the FFT launch shapes: for each grid (N1, N2, N3) and precision
// it times a few candidate shapes (sticks per CTA, threads per CTA) of the z and
// plane stages and keeps the fastest.  Results live in a process-wide table and,
// when the environment variable QE_AUTOTUNE_CACHE names a file, in that file
// (one line per grid: "n1 n2 n3 elem spb zthreads pthreads").  Every shape
// gives bit-identical results, so tuning never changes an answer.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "plan.h"

namespace qe {

namespace {
using Key = std::tuple<int, int, int, int>;
std::mutex g_mu;
std::map<Key, FftShape> g_table;
bool g_loaded = false;

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("QE_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int n1, n2, n3, el, spb, zt, pt;
  while (std::fscanf(f, "%d %d %d %d %d %d %d", &n1, &n2, &n3, &el, &spb, &zt, &pt) == 7) {
    FftShape s;
    s.spb = spb;
    s.zthreads = zt;
    s.pthreads = pt;
    g_table[Key(n1, n2, n3, el)] = s;
  }
  std::fclose(f);
}
}  // namespace

// Untuned grids take the kernels' defaults, except the FP32 register-resident
// square plane: 384 threads, so that its x rows, owned by warps, come 8 to a
// warp and every x pass is whole rounds of 32 lanes (C1 mixed: 0.325 -> 0.276 ms
// per 68-band launch against the 256-thread default of its launch bounds).
FftShape tuned_shape(const DevPlan& P, size_t elem_bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_table.find(Key(P.grid[0], P.grid[1], P.grid[2], (int)elem_bytes));
  if (it != g_table.end()) return it->second;
  FftShape s;
  if (elem_bytes == sizeof(float) && P.sq != 0) s.pthreads = 384;
  return s;
}

void store_shape(const int grid[3], size_t elem_bytes, const FftShape& s) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  g_table[Key(grid[0], grid[1], grid[2], (int)elem_bytes)] = s;
  const char* path = std::getenv("QE_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (auto& kv : g_table)
    std::fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), kv.second.spb, kv.second.zthreads,
                 kv.second.pthreads);
  std::fclose(f);
}

bool has_shape(const int grid[3], size_t elem_bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  return g_table.count(Key(grid[0], grid[1], grid[2], (int)elem_bytes)) != 0;
}

}  // namespace qe
