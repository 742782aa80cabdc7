// Operation-counting scalar for the oracle's op-counting build.
//
// TEST INFRASTRUCTURE ONLY.  When the oracle is compiled with
// -DORACLE_COUNT_OPS its scalar type `real` becomes `Counted`, which holds a
// double and increments a global counter for every arithmetic operation it
// performs.  Comparisons are not counted (they decide branches, they are not
// floating-point work).  The counts give the algorithmic operation mix of one
// right-hand-side evaluation: additions/subtractions, multiplications,
// divisions, square roots and min/max/abs.  Every operation is also booked
// to the step of the method that is running (g_oracle_row, set by the
// oracle as it enters each step), so the mix is available per step.
#pragma once
#include <cmath>

struct OracleOpCounts {
  unsigned long long add, mul, div, sqrt, minmax;
};
extern OracleOpCounts g_oracle_ops;
// Per-step counts; index = the step's number (0 = not attributed).
enum { ORACLE_NROWS = 16 };
extern OracleOpCounts g_oracle_rows[ORACLE_NROWS];
extern int g_oracle_row;

#define OC_TALLY(field) (g_oracle_ops.field++, g_oracle_rows[g_oracle_row].field++)

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}
  explicit operator double() const { return v; }
  Counted &operator+=(Counted b) { OC_TALLY(add); v += b.v; return *this; }
  Counted &operator-=(Counted b) { OC_TALLY(add); v -= b.v; return *this; }
  Counted &operator*=(Counted b) { OC_TALLY(mul); v *= b.v; return *this; }
  Counted &operator/=(Counted b) { OC_TALLY(div); v /= b.v; return *this; }
};

inline Counted operator+(Counted a, Counted b) { OC_TALLY(add); return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { OC_TALLY(add); return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { OC_TALLY(mul); return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { OC_TALLY(div); return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { return a.v != b.v; }

inline Counted o_sqrt(Counted a) { OC_TALLY(sqrt); return Counted(std::sqrt(a.v)); }
inline Counted o_min(Counted a, Counted b) { OC_TALLY(minmax); return Counted(a.v < b.v ? a.v : b.v); }
inline Counted o_max(Counted a, Counted b) { OC_TALLY(minmax); return Counted(a.v > b.v ? a.v : b.v); }
inline Counted o_abs(Counted a) { OC_TALLY(minmax); return Counted(std::fabs(a.v)); }
inline double o_val(Counted a) { return a.v; }
inline bool o_isfinite(Counted a) { return std::isfinite(a.v); }
