// Algorithmic work of each kernel launch (host only).
//
// Floating-point operations are counted, not estimated: the pointwise physics
// of physics.cuh (forward and adjoint) is instantiated on the host with a
// counting scalar type (every +, -, *, /, sqrt and |.| counts one flop, so a
// fused multiply-add counts two), and the contractions are counted from the
// loop structure of each kernel.  Bytes are the kernel's compulsory traffic:
// every input read once and every output written once.
#pragma once
#include <cmath>

// The counting type is host-only; the host-device physics templates are
// instantiated with it on the host only.
#pragma nv_diag_suppress 20011
#include <cstdint>

namespace dgx {

struct Count {
  double v;
  static int64_t ops;
  Count() : v(0) {}
  Count(double x) : v(x) {}
};
inline Count operator+(Count a, Count b) { ++Count::ops; return Count(a.v + b.v); }
inline Count operator-(Count a, Count b) { ++Count::ops; return Count(a.v - b.v); }
inline Count operator*(Count a, Count b) { ++Count::ops; return Count(a.v * b.v); }
inline Count operator/(Count a, Count b) { ++Count::ops; return Count(a.v / b.v); }
inline Count operator-(Count a) { return Count(-a.v); }
inline Count& operator+=(Count& a, Count b) { a = a + b; return a; }
inline Count& operator-=(Count& a, Count b) { a = a - b; return a; }
inline Count& operator*=(Count& a, Count b) { a = a * b; return a; }
inline bool operator>=(Count a, Count b) { return a.v >= b.v; }
inline bool operator>(Count a, Count b) { return a.v > b.v; }
inline bool operator<(Count a, Count b) { return a.v < b.v; }
inline bool operator!=(Count a, Count b) { return a.v != b.v; }
inline Count sqrt(Count a) { ++Count::ops; return Count(std::sqrt(a.v)); }
inline Count fabs(Count a) { ++Count::ops; return Count(std::fabs(a.v)); }

}  // namespace dgx
