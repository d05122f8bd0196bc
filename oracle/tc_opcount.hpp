// Operation-counting scalar for the oracle (TEST INFRASTRUCTURE ONLY).
//
// Cnt wraps a double and tallies every FP64 operation the oracle's method performs:
// add/sub, mul, div, sqrt and each call of exp, log and pow.  Instantiating the oracle's
// templates with R = Cnt yields the algorithmic operation count of one step, which is
// the numerator of the roofline fraction reported for the GPU kernels.
#pragma once
#include <cmath>

namespace oracle {

struct OpCount {
  unsigned long long add, mul, div, sqrt, exp, log, pow, cmp;
};
extern thread_local OpCount g_ops;

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
  explicit operator double() const { return v; }
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops.div; return Cnt(a.v / b.v); }
inline bool operator<(Cnt a, Cnt b) { ++g_ops.cmp; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { ++g_ops.cmp; return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { ++g_ops.cmp; return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { ++g_ops.cmp; return a.v >= b.v; }
inline bool operator==(Cnt a, Cnt b) { ++g_ops.cmp; return a.v == b.v; }
inline bool operator!=(Cnt a, Cnt b) { ++g_ops.cmp; return a.v != b.v; }
inline Cnt sqrt(Cnt a) { ++g_ops.sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt exp(Cnt a) { ++g_ops.exp; return Cnt(std::exp(a.v)); }
inline Cnt log(Cnt a) { ++g_ops.log; return Cnt(std::log(a.v)); }
inline Cnt pow(Cnt a, Cnt b) { ++g_ops.pow; return Cnt(std::pow(a.v, b.v)); }

}  // namespace oracle

namespace std {
inline bool isfinite(oracle::Cnt a) { return std::isfinite(a.v); }
}
