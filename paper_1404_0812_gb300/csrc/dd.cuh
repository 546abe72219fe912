// Double-double arithmetic: a value is the unevaluated sum hi + lo of two
// float64 numbers with |lo| <= ulp(hi) / 2, about 106 bits of significand
// (unit roundoff ~1.1e-32).  Built from the error-free transformations of
// Knuth (TwoSum: a + b = s + e exactly) and of Dekker with a fused
// multiply-add (TwoProduct: a * b = p + e exactly), in the arrangement of
// Hida, Li and Bailey's double-double library (accurate addition, one
// correction term in products, long division, one Newton step for the square
// root).  The exponential reduces by ln 2 and 2^10 and sums a Taylor series.
// The float64 operations use the _rn intrinsics so that the compiler never
// contracts them into fused multiply-adds, which would break the exactness of
// the transformations.
#pragma once

#include <cmath>

namespace rbffd {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_of(double a) { return dd{a, 0.0}; }

// s + e = a + b exactly
__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return dd{s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double e = __dsub_rn(b, __dsub_rn(s, a));
    return dd{s, e};
}

// p + e = a * b exactly (no overflow / underflow)
__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = __dmul_rn(a, b);
    double e = __fma_rn(a, b, -p);
    return dd{p, e};
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    dd r = fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
    return fast_two_sum(r.hi, __dadd_rn(r.lo, t.lo));
}

__device__ __forceinline__ dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    double c = __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi));
    return fast_two_sum(p.hi, __dadd_rn(p.lo, c));
}

__device__ __forceinline__ dd operator*(dd a, double b) {
    dd p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __dadd_rn(p.lo, __dmul_rn(a.lo, b)));
}

// a - b c, the update of every elimination and solve
__device__ __forceinline__ dd fms(dd a, dd b, dd c) { return a - b * c; }

// long division: three float64 quotient digits
__device__ __forceinline__ dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * q1;
    double q2 = r.hi / b.hi;
    r = r - b * q2;
    double q3 = r.hi / b.hi;
    return fast_two_sum(q1, q2) + dd_of(q3);
}

// one Newton step from the float64 square root: x + (a - x^2) / (2 x)
__device__ __forceinline__ dd dd_sqrt(dd a) {
    if (!(a.hi > 0.0)) return dd{a.hi == 0.0 ? 0.0 : NAN, 0.0};
    double x = sqrt(a.hi);
    dd r = a - two_prod(x, x);
    return fast_two_sum(x, r.hi / (2.0 * x));
}

// scale by 2^k exactly
__device__ __forceinline__ dd dd_ldexp(dd a, int k) { return dd{ldexp(a.hi, k), ldexp(a.lo, k)}; }

// exp(a): a = k ln 2 + r, |r| <= ln2 / 2; e^r = (e^{r / 1024})^1024 with
// e^{r/1024} - 1 summed as a Taylor series (|r / 1024| < 3.4e-4, nine terms
// leave < 1e-36) and squared ten times in the form e^{2y} - 1 = 2 s + s^2.
__device__ inline dd dd_exp(dd a) {
    if (a.hi < -745.0) return dd_of(0.0);
    const dd ln2 = {6.931471805599452862e-01, 2.319046813846299558e-17};
    const double k = rint(a.hi / ln2.hi);
    dd r = dd_ldexp(a - ln2 * k, -10);
    dd term = r, s = r;
    for (int j = 2; j <= 9; ++j) {
        term = term * r / dd_of((double)j);
        s = s + term;
    }
    for (int i = 0; i < 10; ++i) s = s * 2.0 + s * s;
    return dd_ldexp(s + dd_of(1.0), (int)k);
}

}  // namespace rbffd
