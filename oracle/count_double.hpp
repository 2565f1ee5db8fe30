// Counting double for the oracle's operation tally.  TEST INFRASTRUCTURE
// ONLY (built by oracle/tally.py, never by the product library).
//
// The oracle's C source is compiled as C++ with this header forced in
// first and every `double` replaced by `cdouble`: a one-member struct with
// the size, alignment and calling convention of a double, whose arithmetic
// operators and math functions add one to a per-section counter before
// doing the plain double operation.  Results are therefore bit-identical
// to the plain build's, and the counters hold how many floating-point
// operations of each kind the oracle's direct formulation of the method
// performs.  Operations between two plain constants (e.g. 2.0 / 3.0) are
// folded by the compiler and not counted, as in the plain build.  The
// sections are set by the oracle's OR_SECTION markers.
#pragma once

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace tally {

enum Kind { ADD = 0, MUL = 1, DIV = 2, SQRT = 3, TRANS = 4, KINDS = 5 };
constexpr int SECTIONS = 16;
extern "C" {
extern long long or_tally[SECTIONS][KINDS];
extern int or_tally_section;
}
inline void hit(Kind k) { ++or_tally[or_tally_section][k]; }

struct cdouble {
  double v;
  cdouble() = default;
  constexpr cdouble(double x) : v(x) {}
  explicit constexpr operator double() const { return v; }
  cdouble &operator+=(cdouble o) { hit(ADD); v += o.v; return *this; }
  cdouble &operator-=(cdouble o) { hit(ADD); v -= o.v; return *this; }
  cdouble &operator*=(cdouble o) { hit(MUL); v *= o.v; return *this; }
  cdouble &operator/=(cdouble o) { hit(DIV); v /= o.v; return *this; }
  cdouble operator-() const { return cdouble(-v); }
  cdouble operator+() const { return *this; }
};
static_assert(sizeof(cdouble) == sizeof(double), "cdouble must be layout-compatible with double");

inline cdouble operator+(cdouble a, cdouble b) { hit(ADD); return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { hit(ADD); return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { hit(MUL); return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { hit(DIV); return cdouble(a.v / b.v); }
inline bool operator<(cdouble a, cdouble b) { return a.v < b.v; }
inline bool operator>(cdouble a, cdouble b) { return a.v > b.v; }
inline bool operator<=(cdouble a, cdouble b) { return a.v <= b.v; }
inline bool operator>=(cdouble a, cdouble b) { return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { return a.v != b.v; }

inline cdouble sqrt(cdouble a) { hit(SQRT); return cdouble(::sqrt(a.v)); }
inline cdouble pow(cdouble a, cdouble b) { hit(TRANS); return cdouble(::pow(a.v, b.v)); }
inline cdouble log(cdouble a) { hit(TRANS); return cdouble(::log(a.v)); }
inline cdouble exp(cdouble a) { hit(TRANS); return cdouble(::exp(a.v)); }
inline cdouble fabs(cdouble a) { return cdouble(::fabs(a.v)); }
inline cdouble fmax(cdouble a, cdouble b) { return cdouble(::fmax(a.v, b.v)); }
inline cdouble fmin(cdouble a, cdouble b) { return cdouble(::fmin(a.v, b.v)); }

}  // namespace tally

using tally::cdouble;
using tally::sqrt;
using tally::pow;
using tally::log;
using tally::exp;
using tally::fabs;
using tally::fmax;
using tally::fmin;

#define OR_SECTION(sec) (tally::or_tally_section = (sec))
#define double cdouble
