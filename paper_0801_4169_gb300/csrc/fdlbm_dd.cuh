#pragma once
// fdlbm_dd.cuh -- double-double arithmetic for the von Neumann tool (fdlbm_vn.cu).
//
// A value is an unevaluated sum hi + lo of two FP64 numbers with |lo| <= ulp(hi)/2, i.e. ~106
// significant bits. The building blocks are the error-free transformations:
//   two_sum  (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   two_prod (Dekker 1971, with a fused multiply-add): p + e = a * b exactly.
// The operations follow the "sloppy" double-double forms of Hida, Li and Bailey (QD library,
// 2001). Their error is a few units of 2^-106 relative to the operands' magnitudes, which is
// the normwise accuracy the eigenvalue computation needs.
//
// Every step uses the explicitly rounded intrinsics, so the compiler cannot contract or
// reorder the error terms.

namespace fdlbm {
namespace dd {

struct dd_t {
  double hi, lo;
};

__device__ __forceinline__ dd_t make(double x) { return {x, 0.0}; }

__device__ __forceinline__ dd_t two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dd_t quick_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd_t two_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  return {p, __fma_rn(a, b, -p)};
}

__device__ __forceinline__ dd_t add(dd_t a, dd_t b) {
  dd_t s = two_sum(a.hi, b.hi);
  s.lo = __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd_t neg(dd_t a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd_t sub(dd_t a, dd_t b) { return add(a, neg(b)); }
__device__ __forceinline__ dd_t add(dd_t a, double b) {
  dd_t s = two_sum(a.hi, b);
  s.lo = __dadd_rn(s.lo, a.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd_t mul(dd_t a, dd_t b) {
  dd_t p = two_prod(a.hi, b.hi);
  p.lo = __fma_rn(a.hi, b.lo, __fma_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd_t mul(dd_t a, double b) {
  dd_t p = two_prod(a.hi, b);
  p.lo = __fma_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd_t sqr(dd_t a) {
  dd_t p = two_prod(a.hi, a.hi);
  p.lo = __fma_rn(2.0 * a.hi, a.lo, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
// Multiplication by a power of two is exact.
__device__ __forceinline__ dd_t scale2(dd_t a, double p2) { return {a.hi * p2, a.lo * p2}; }

// 1/b: FP64 quotient refined by one Newton step, y = y0 + y0 (1 - b y0).
__device__ __forceinline__ dd_t rcp(dd_t b) {
  const double y0 = 1.0 / b.hi;
  const dd_t e = sub(make(1.0), mul(b, y0));
  return quick_two_sum(y0, __dmul_rn(e.hi, y0));
}
__device__ __forceinline__ dd_t div(dd_t a, dd_t b) {
  const double q1 = a.hi / b.hi;
  const dd_t r = sub(a, mul(b, q1));
  const double q2 = r.hi / b.hi;
  const dd_t r2 = sub(r, mul(b, q2));
  const double q3 = r2.hi / b.hi;
  return add(quick_two_sum(q1, q2), q3);
}
__device__ __forceinline__ dd_t div(dd_t a, double b) { return div(a, make(b)); }

// 1/sqrt(a), a > 0: FP64 estimate refined by one Newton step, y = y0 + y0 (1 - a y0^2) / 2.
__device__ __forceinline__ dd_t rsqrt(dd_t a) {
  const double y0 = 1.0 / ::sqrt(a.hi);
  const dd_t e = sub(make(1.0), mul(mul(a, y0), y0));
  return quick_two_sum(y0, __dmul_rn(0.5 * e.hi, y0));
}
// sqrt(a), a >= 0: x = sqrt(a_hi) corrected by (a - x^2) / (2x).
__device__ __forceinline__ dd_t sqrt(dd_t a) {
  if (a.hi <= 0.0) return make(0.0);
  const double x = ::sqrt(a.hi);
  const dd_t p = two_prod(x, x);
  const double r = __dadd_rn(__dsub_rn(__dsub_rn(a.hi, p.hi), p.lo), a.lo);
  return quick_two_sum(x, r / (2.0 * x));
}

// ---- complex double-double
struct cdd {
  dd_t re, im;
};
__device__ __forceinline__ cdd cmake(dd_t re, dd_t im) { return {re, im}; }
__device__ __forceinline__ cdd cadd(cdd a, cdd b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ cdd csub(cdd a, cdd b) { return {sub(a.re, b.re), sub(a.im, b.im)}; }
__device__ __forceinline__ cdd cconj(cdd a) { return {a.re, neg(a.im)}; }
__device__ __forceinline__ cdd cmul(cdd a, cdd b) {
  return {sub(mul(a.re, b.re), mul(a.im, b.im)), add(mul(a.re, b.im), mul(a.im, b.re))};
}
__device__ __forceinline__ cdd cmul(cdd a, dd_t b) { return {mul(a.re, b), mul(a.im, b)}; }
// conj(a) * b
__device__ __forceinline__ cdd cmulc(cdd a, cdd b) {
  return {add(mul(a.re, b.re), mul(a.im, b.im)), sub(mul(a.re, b.im), mul(a.im, b.re))};
}
__device__ __forceinline__ dd_t cabs2(cdd a) { return add(sqr(a.re), sqr(a.im)); }
// Principal square root: with r = |z|, t = sqrt((r + |x|)/2), the root is (t, y/2t) for x >= 0
// and (|y|/2t, sign(y) t) otherwise, which avoids cancellation in either half-plane.
__device__ __forceinline__ cdd csqrt(cdd z) {
  const dd_t r = sqrt(cabs2(z));
  if (r.hi == 0.0) return {make(0.0), make(0.0)};
  const dd_t ax = z.re.hi < 0.0 ? neg(z.re) : z.re;
  const dd_t t = sqrt(scale2(add(r, ax), 0.5));
  const dd_t q = div(z.im, scale2(t, 2.0));  // y / 2t
  if (z.re.hi >= 0.0) return {t, q};
  return {q.hi < 0.0 ? neg(q) : q, z.im.hi < 0.0 ? neg(t) : t};
}

// ---- sin and cos of an FP64 argument, to double-double accuracy.
// Argument reduction x = k pi/2 + r, |r| <= pi/4, with pi/2 split into three doubles (Cody and
// Waite's scheme carried in double-double), then the Taylor series of sin r and cos r to the
// r^27 and r^26 terms ((pi/4)^28 / 28! < 1e-31), summed by Horner's rule in r^2 with the
// coefficients 1/n! formed by exact-enough double-double division.
__device__ __forceinline__ void sincos_dd(double x, dd_t* s_out, dd_t* c_out) {
  const double P1 = 1.5707963267948966, P2 = 6.123233995736766e-17, P3 = -1.4973849048591698e-33;
  const double k = rint(x / P1);
  dd_t r = sub(make(x), two_prod(k, P1));
  r = sub(r, two_prod(k, P2));
  r = add(r, -k * P3);
  const dd_t r2 = sqr(r);
  // coefficients (-1)^m / (2m+1)! and (-1)^m / (2m)!, m = 0..13
  dd_t cs[14], cc[14];
  cs[0] = make(1.0);
  cc[0] = make(1.0);
  for (int m = 1; m < 14; ++m) {
    cc[m] = neg(div(cs[m - 1], (double)(2 * m)));
    cs[m] = div(cc[m], (double)(2 * m + 1));
  }
  dd_t ps = cs[13], pc = cc[13];
  for (int m = 12; m >= 0; --m) {
    ps = add(mul(ps, r2), cs[m]);
    pc = add(mul(pc, r2), cc[m]);
  }
  ps = mul(ps, r);
  const int q = ((int)k) & 3;
  dd_t s, c;
  if (q == 0) {
    s = ps;
    c = pc;
  } else if (q == 1) {
    s = pc;
    c = neg(ps);
  } else if (q == 2) {
    s = neg(ps);
    c = neg(pc);
  } else {
    s = neg(pc);
    c = ps;
  }
  *s_out = s;
  *c_out = c;
}

}  // namespace dd
}  // namespace fdlbm
