// Operation-counting scalar for the oracle's op-counting build.
//
// TEST INFRASTRUCTURE ONLY.  When the oracle is compiled with
// -DORACLE_COUNT_OPS its scalar type `real` becomes `Counted`, which holds a
// double and increments a global counter for every arithmetic operation it
// performs.  Comparisons are not counted (they decide branches, they are not
// floating-point work).  The counts give the algorithmic operation mix of one
// right-hand-side evaluation: additions/subtractions, multiplications,
// divisions, square roots and min/max/abs.
#pragma once
#include <cmath>

struct OracleOpCounts {
  unsigned long long add, mul, div, sqrt, minmax;
};
extern OracleOpCounts g_oracle_ops;

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}
  explicit operator double() const { return v; }
  Counted &operator+=(Counted b) { g_oracle_ops.add++; v += b.v; return *this; }
  Counted &operator-=(Counted b) { g_oracle_ops.add++; v -= b.v; return *this; }
  Counted &operator*=(Counted b) { g_oracle_ops.mul++; v *= b.v; return *this; }
  Counted &operator/=(Counted b) { g_oracle_ops.div++; v /= b.v; return *this; }
};

inline Counted operator+(Counted a, Counted b) { g_oracle_ops.add++; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { g_oracle_ops.add++; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { g_oracle_ops.mul++; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { g_oracle_ops.div++; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { return a.v != b.v; }

inline Counted o_sqrt(Counted a) { g_oracle_ops.sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted o_min(Counted a, Counted b) { g_oracle_ops.minmax++; return Counted(a.v < b.v ? a.v : b.v); }
inline Counted o_max(Counted a, Counted b) { g_oracle_ops.minmax++; return Counted(a.v > b.v ? a.v : b.v); }
inline Counted o_abs(Counted a) { g_oracle_ops.minmax++; return Counted(std::fabs(a.v)); }
inline double o_val(Counted a) { return a.v; }
inline bool o_isfinite(Counted a) { return std::isfinite(a.v); }
