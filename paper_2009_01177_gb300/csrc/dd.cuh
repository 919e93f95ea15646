// dd.cuh -- double-double arithmetic for the second precision tier.
//
// A dd value is an unevaluated sum hi + lo with |lo| <= ulp(hi)/2, about
// 106 significant bits.  The operations are built from the standard
// error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2):  s + e == a + b exactly, any magnitudes;
//   FastTwoSum (Dekker 1971):      the same when |a| >= |b|;
//   TwoProd via FMA:               p + e == a * b exactly.
// The paper's own wide type is 128/256-bit fixed point (Sec. 5); this tier
// gives the ~2^-104 relative accuracy in the FP64 pipe instead.
#pragma once

namespace tor {

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return {s, e};
}

__device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }

// a * b with the cross terms (relative error ~ 2^-104)
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p = a.hi * b.hi;
  double e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  double p = a.hi * b;
  double e = fma(a.hi, b, -p);
  e = fma(a.lo, b, e);
  return fast_two_sum(p, e);
}

// a + b (the "sloppy" add: error bounded by ~2^-104 (|a| + |b|))
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

// s - (v0 u0 + v1 u1): the rank-2 Schur update of one entry
__device__ __forceinline__ dd dd_rank2_update(dd s, dd v0, dd u0, dd v1, dd u1) {
  double p0 = v0.hi * u0.hi;
  double e0 = fma(v0.hi, u0.hi, -p0);
  double p1 = v1.hi * u1.hi;
  double e1 = fma(v1.hi, u1.hi, -p1);
  dd q = two_sum(p0, p1);
  double c = e0 + e1;
  c = fma(v0.hi, u0.lo, c);
  c = fma(v0.lo, u0.hi, c);
  c = fma(v1.hi, u1.lo, c);
  c = fma(v1.lo, u1.hi, c);
  q.lo += c;
  dd r = two_sum(s.hi, -q.hi);
  r.lo += s.lo - q.lo;
  return fast_two_sum(r.hi, r.lo);
}

// a*d - b*b for the 2x2 pivot block
__device__ __forceinline__ dd dd_det2(dd a, dd b, dd d) {
  dd ad = dd_mul(a, d);
  dd bb = dd_mul(b, b);
  return dd_add(ad, dd_neg(bb));
}

// 1/sqrt(x) for x > 0: FP64 Newton seed, then one Newton step in dd
// (y <- y + y (1 - x y^2) / 2 doubles the ~53 correct bits).
__device__ __forceinline__ dd dd_rsqrt(dd x, double y0) {
  dd y = dd_from(y0);
  dd y2 = dd_mul(y, y);
  dd xy2 = dd_mul(x, y2);
  dd e = dd_add({1.0, 0.0}, dd_neg(xy2));   // small: |e| ~ 2^-52
  dd corr = dd_mul_d(dd_mul(y, e), 0.5);
  return dd_add(y, corr);
}

}  // namespace tor
