/*
 * op_count.cpp -- the counting build of the CPU oracle (TEST INFRASTRUCTURE
 * ONLY): bh_oracle.c compiled as C++ with counting doubles (op_count.hpp),
 * plus the tally's reset and read-out.  Built into liboracle_count.so by
 * oracle.build_count(); only the benchmark's CPU-baseline leg and the tests
 * load it.
 */
// the oracle's system headers first, so that they are parsed with the real
// double; op_count.hpp then maps double to the counting type
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <cstdlib>
#include <cstring>

#define ORC_COUNTING 1
#include "op_count.hpp"
extern "C" {
#include "bh_oracle.c"
}
#undef double

namespace orc_count {
thread_local Tally t_tally;
thread_local int t_paused = 0;
static std::mutex g_mu;
static Tally g_tally;
static std::vector<std::atomic<uint64_t>> *g_seen = nullptr, *g_seen_occ = nullptr;

void flush() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int k = 0; k < kN; ++k) {
    g_tally.n[k] += t_tally.n[k];
    t_tally.n[k] = 0;
  }
}

void touch(long long rec, int occupied) {
  if (t_paused || !g_seen || rec < 0 || (size_t)(rec >> 6) >= g_seen->size()) return;
  (*g_seen)[rec >> 6].fetch_or(1ull << (rec & 63), std::memory_order_relaxed);
  if (occupied) (*g_seen_occ)[rec >> 6].fetch_or(1ull << (rec & 63), std::memory_order_relaxed);
}
}  // namespace orc_count

extern "C" {

/* Start a count: zero the tallies; n_records sizes the unique-record bitmaps
 * of the cube map (0: none). */
void orc_count_reset(long long n_records) {
  using namespace orc_count;
  std::lock_guard<std::mutex> lk(g_mu);
  memset(&g_tally, 0, sizeof g_tally);
  memset(&t_tally, 0, sizeof t_tally);
  delete g_seen;
  delete g_seen_occ;
  g_seen = g_seen_occ = nullptr;
  if (n_records > 0) {
    size_t w = (size_t)((n_records + 63) / 64);
    g_seen = new std::vector<std::atomic<uint64_t>>(w);
    g_seen_occ = new std::vector<std::atomic<uint64_t>>(w);
  }
}

/* Read the tallies: out[0..kN-1] by class (add, mul, div, sqrt, elementary
 * functions, comparisons, other, D/U/C/disc-table texel reads, cube records
 * read), out[kN] unique cube records read, out[kN+1] unique occupied ones. */
void orc_count_read(long long *out) {
  using namespace orc_count;
  flush();
  std::lock_guard<std::mutex> lk(g_mu);
  for (int k = 0; k < kN; ++k) out[k] = g_tally.n[k];
  long long u = 0, uo = 0;
  if (g_seen)
    for (size_t i = 0; i < g_seen->size(); ++i) {
      u += __builtin_popcountll((*g_seen)[i].load());
      uo += __builtin_popcountll((*g_seen_occ)[i].load());
    }
  out[kN] = u;
  out[kN + 1] = uo;
}
}
