// FP64 operation count of the oracle's step, per cell-update.
//
// TEST INFRASTRUCTURE ONLY (an analysis of the oracle, not part of the
// library).  vlbm_oracle.c is compiled unchanged as C++ with `double`
// replaced by a stand-in that performs the same IEEE double operation and
// counts it: additions and subtractions, multiplications, divisions, square
// roots, comparisons, absolute values and the trigonometric calls of the
// inlet.  One realization of the jet (seed 0, m = 0, the paper's constants,
// Sec. 2.2-2.3) is advanced with the landing rule to each requested time;
// there the kinetic speed and one step (Sec. 2.1, Eqs. (vlbm1)-(vlbm5)) are
// counted and divided by the nx ny cell-updates of that step.
//
//   flop_count nx ny t1 [t2 ...]
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <vector>

namespace {
struct Counts {
  unsigned long long add, mul, div, sqrt, cmp, abs, trans;
};
Counts g_counts = {};
}  // namespace

struct CountedDouble {
  double v;
  CountedDouble() = default;
  constexpr CountedDouble(double x) : v(x) {}
  constexpr CountedDouble(int x) : v(x) {}
  constexpr CountedDouble(long x) : v((double)x) {}
  constexpr CountedDouble(unsigned x) : v(x) {}
  constexpr CountedDouble(unsigned long x) : v((double)x) {}
  constexpr CountedDouble(long long x) : v((double)x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator bool() const { return v != 0.0; }
  CountedDouble& operator+=(CountedDouble b) { ++g_counts.add; v += b.v; return *this; }
  CountedDouble& operator-=(CountedDouble b) { ++g_counts.add; v -= b.v; return *this; }
  CountedDouble& operator*=(CountedDouble b) { ++g_counts.mul; v *= b.v; return *this; }
  CountedDouble& operator/=(CountedDouble b) { ++g_counts.div; v /= b.v; return *this; }
  CountedDouble operator-() const { return CountedDouble(-v); }
};
using CD = CountedDouble;
inline CD operator+(CD a, CD b) { ++g_counts.add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++g_counts.add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++g_counts.mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++g_counts.div; return CD(a.v / b.v); }
inline bool operator<(CD a, CD b) { ++g_counts.cmp; return a.v < b.v; }
inline bool operator>(CD a, CD b) { ++g_counts.cmp; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { ++g_counts.cmp; return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { ++g_counts.cmp; return a.v >= b.v; }
inline bool operator==(CD a, CD b) { ++g_counts.cmp; return a.v == b.v; }
inline bool operator!=(CD a, CD b) { ++g_counts.cmp; return a.v != b.v; }
inline CD sqrt(CD a) { ++g_counts.sqrt; return CD(std::sqrt(a.v)); }
inline CD fabs(CD a) { ++g_counts.abs; return CD(std::fabs(a.v)); }
inline CD cos(CD a) { ++g_counts.trans; return CD(std::cos(a.v)); }
inline CD sin(CD a) { ++g_counts.trans; return CD(std::sin(a.v)); }
inline CD floor(CD a) { ++g_counts.trans; return CD(std::floor(a.v)); }
inline bool isfinite(CD a) { ++g_counts.cmp; return std::isfinite(a.v); }

#define double CountedDouble
#include "vlbm_oracle.c"
#undef double

int main(int argc, char** argv) {
  if (argc < 4) {
    fprintf(stderr, "usage: flop_count nx ny t1 [t2 ...]\n");
    return 1;
  }
  const int nx = atoi(argv[1]), ny = atoi(argv[2]);
  const double dx = 2.5 / nx;
  orc_grid g{nx, ny, CD(dx), CD(-0.5 * ny * dx)};
  orc_params P{CD(5.0 / 3.0), CD(0.0), CD(1.0), 2, CD(0.1), CD(0.0), CD(1e-13), BC_JET};
  orc_prim jet{CD(5.0), CD(800.0), CD(0.0), CD(0.4127)}, amb{CD(0.5), CD(0.0), CD(0.0), CD(0.4127)};
  const int K = 10;
  const size_t n = (size_t)nx * ny;
  std::vector<CD> amp(K), inlet(4 * (size_t)ny), u(4 * n), un(4 * n), f(16 * n), fn(16 * n);
  for (int k = 1; k <= K; ++k) amp[k - 1] = CD(0.1 * std::pow((double)k, -2.0));
  if (orc_inlet(&g, CD(5.0 / 3.0), &jet, &amb, CD(0.05), K, amp.data(), 0, 0, inlet.data())) return 2;
  CD a0;
  if (orc_init_state(&g, &P, inlet.data(), &amb, u.data(), f.data(), &a0)) return 2;
  double t = 0.0;
  for (int arg = 3; arg < argc; ++arg) {
    const double T = atof(argv[arg]);
    while (t < T) {
      CD a;
      if (orc_kinetic_speed(&g, &P, u.data(), &a)) return 3;
      double av = (double)a;
      if (av < dx / (T - t)) av = dx / (T - t);
      const bool landing = t + dx / av >= T * (1.0 - 1e-15);
      if (orc_step(&g, &P, CD(av), inlet.data(), u.data(), f.data(), un.data(), fn.data())) return 4;
      u.swap(un);
      f.swap(fn);
      t = landing ? T : t + dx / av;
    }
    g_counts = {};
    CD a;
    orc_kinetic_speed(&g, &P, u.data(), &a);
    orc_step(&g, &P, a, inlet.data(), u.data(), f.data(), un.data(), fn.data());
    const double c = (double)n;
    // the counted step's result, summed in storage order: equal to the plain
    // oracle's when the stand-in changes nothing but the counting
    double check = 0.0;
    for (size_t i = 0; i < 4 * n; ++i) check += un[i].v;
    printf("%d %d %.6g add %.2f mul %.2f div %.2f sqrt %.3f cmp %.2f abs %.2f trans %.3f check %.17g\n", nx, ny,
           T, g_counts.add / c, g_counts.mul / c, g_counts.div / c, g_counts.sqrt / c, g_counts.cmp / c,
           g_counts.abs / c, g_counts.trans / c, check);
  }
  return 0;
}
