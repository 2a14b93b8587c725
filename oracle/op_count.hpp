/*
 * op_count.hpp -- counting build of the CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Included by oracle/op_count.cpp, which compiles bh_oracle.c as C++ with
 * every `double` replaced by `cdouble`: a value type of the same size and
 * layout that tallies each operation the oracle performs on it, by class,
 * in per-thread counters.  The oracle's arithmetic and results are
 * unchanged; only the counting is added.  This gives the work the method
 * itself does per pixel (arithmetic, elementary functions, table reads),
 * independent of how the CUDA kernel is written.
 */
#pragma once
#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <type_traits>
#include <vector>

namespace orc_count {

enum Cls { kAdd, kMul, kDiv, kSqrt, kTransc, kCmp, kOther, kFetchD, kFetchU, kFetchC, kFetchDisc, kFetchCube, kN };

struct Tally {
  long long n[kN];
};
extern thread_local Tally t_tally;
extern thread_local int t_paused;
inline void tick(Cls c) {
  if (!t_paused) ++t_tally.n[c];
}
inline void tickn(Cls c, long long k) {
  if (!t_paused) t_tally.n[c] += k;
}
void flush();                        // add this thread's tally to the global one
void touch(long long rec, int occupied);  // a cube-map record read (unique-record bitmaps)

}  // namespace orc_count

struct cdouble {
  double v;
  cdouble() = default;
  constexpr cdouble(double x) : v(x) {}
  template <class T, class = typename std::enable_if<std::is_integral<T>::value>::type>
  constexpr cdouble(T x) : v((double)x) {}
  explicit operator double() const { return v; }
  explicit operator float() const { return (float)v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned() const { return (unsigned)v; }
  explicit operator unsigned short() const { return (unsigned short)v; }
  cdouble &operator+=(cdouble o) { orc_count::tick(orc_count::kAdd); v += o.v; return *this; }
  cdouble &operator-=(cdouble o) { orc_count::tick(orc_count::kAdd); v -= o.v; return *this; }
  cdouble &operator*=(cdouble o) { orc_count::tick(orc_count::kMul); v *= o.v; return *this; }
  cdouble &operator/=(cdouble o) { orc_count::tick(orc_count::kDiv); v /= o.v; return *this; }
};
static_assert(sizeof(cdouble) == sizeof(double), "cdouble must have double's layout");
static_assert(std::is_trivially_copyable<cdouble>::value, "cdouble must be trivially copyable");

inline cdouble operator+(cdouble a, cdouble b) { orc_count::tick(orc_count::kAdd); return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { orc_count::tick(orc_count::kAdd); return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { orc_count::tick(orc_count::kMul); return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { orc_count::tick(orc_count::kDiv); return cdouble(a.v / b.v); }
inline cdouble operator-(cdouble a) { orc_count::tick(orc_count::kOther); return cdouble(-a.v); }
inline bool operator<(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v < b.v; }
inline bool operator>(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v > b.v; }
inline bool operator<=(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v <= b.v; }
inline bool operator>=(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { orc_count::tick(orc_count::kCmp); return a.v != b.v; }

#define ORC_CD_F1(name, cls)                                       \
  inline cdouble name(cdouble a) {                                 \
    orc_count::tick(orc_count::cls);                               \
    return cdouble(std::name(a.v));                                \
  }
ORC_CD_F1(sqrt, kSqrt)
ORC_CD_F1(sin, kTransc)
ORC_CD_F1(cos, kTransc)
ORC_CD_F1(tan, kTransc)
ORC_CD_F1(asin, kTransc)
ORC_CD_F1(acos, kTransc)
ORC_CD_F1(atan, kTransc)
ORC_CD_F1(exp, kTransc)
ORC_CD_F1(exp2, kTransc)
ORC_CD_F1(expm1, kTransc)
ORC_CD_F1(log, kTransc)
ORC_CD_F1(log2, kTransc)
ORC_CD_F1(log1p, kTransc)
ORC_CD_F1(fabs, kOther)
ORC_CD_F1(floor, kOther)
ORC_CD_F1(ceil, kOther)
ORC_CD_F1(nearbyint, kOther)
#undef ORC_CD_F1
inline cdouble atan2(cdouble a, cdouble b) { orc_count::tick(orc_count::kTransc); return cdouble(std::atan2(a.v, b.v)); }
inline cdouble fmod(cdouble a, cdouble b) { orc_count::tick(orc_count::kDiv); return cdouble(std::fmod(a.v, b.v)); }
inline cdouble pow(cdouble a, cdouble b) { orc_count::tick(orc_count::kTransc); return cdouble(std::pow(a.v, b.v)); }
inline cdouble ldexp(cdouble a, int e) { orc_count::tick(orc_count::kOther); return cdouble(std::ldexp(a.v, e)); }
inline cdouble frexp(cdouble a, int *e) { orc_count::tick(orc_count::kOther); return cdouble(std::frexp(a.v, e)); }
inline bool isinf(cdouble a) { return std::isinf(a.v); }
inline bool isnan(cdouble a) { return std::isnan(a.v); }
inline bool isfinite(cdouble a) { return std::isfinite(a.v); }

#define ORC_COUNT_PAUSE() (++orc_count::t_paused)
#define ORC_COUNT_RESUME() (--orc_count::t_paused)
#define ORC_COUNT_FLUSH() orc_count::flush()
#define ORC_FETCH(cls, k) orc_count::tickn(orc_count::cls, (k))
#define ORC_TOUCH(rec, occupied) orc_count::touch((rec), (occupied))

#define double cdouble
