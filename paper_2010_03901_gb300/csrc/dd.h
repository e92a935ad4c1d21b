// Double-double arithmetic (about 106 significand bits) for the plan-time
// computation of the FC matrices.  Error-free transformations after Knuth (TwoSum)
// and Dekker / the fused multiply-add (TwoProd); products and quotients follow
// the usual double-double recipes (Hida, Li & Bailey, "Library for double-double
// and quad-double arithmetic", 2000).  Only + - * fma of doubles are used, so the
// results are identical on every IEEE machine.  Compile the host code with
// -ffp-contract=off so that the compiler does not fuse the error terms away.
#pragma once
#include <cmath>

namespace fc2d {

struct dd {
  double hi, lo;
  dd() : hi(0), lo(0) {}
  dd(double h) : hi(h), lo(0) {}
  dd(double h, double l) : hi(h), lo(l) {}
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd(s, e);
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd(s, e);
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = std::fma(a, b, -p);
  return dd(p, e);
}
inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = a - b * dd(q1);
  double q2 = r.hi / b.hi;
  r = r - b * dd(q2);
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return q + dd(q3);
}
inline dd& operator+=(dd& a, dd b) { a = a + b; return a; }
inline dd& operator-=(dd& a, dd b) { a = a - b; return a; }
inline dd& operator*=(dd& a, dd b) { a = a * b; return a; }
inline bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline bool operator>(dd a, dd b) { return b < a; }
inline dd dd_abs(dd a) { return a.hi < 0 || (a.hi == 0 && a.lo < 0) ? -a : a; }
// sqrt by one Newton step on the double estimate (doubles the precision)
inline dd dd_sqrt(dd a) {
  if (a.hi <= 0) return dd(0.0);
  double x = 1.0 / std::sqrt(a.hi);
  double ax = a.hi * x;
  dd ax2 = dd(ax) * dd(ax);
  double corr = (a - ax2).hi * (x * 0.5);
  return two_sum(ax, corr);
}
inline double to_double(dd a) { return a.hi + a.lo; }

// pi to double-double precision: the double nearest pi and the double nearest the rest.
inline dd dd_pi() { return dd(3.141592653589793116e+00, 1.224646799147353207e-16); }

}  // namespace fc2d
