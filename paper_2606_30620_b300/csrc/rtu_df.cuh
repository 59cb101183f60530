// rtu_df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the
// error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the
// fused multiply-add product error, as in Dekker, "A floating-point technique
// for extending the available precision" (Numer. Math. 18, 1971); exp by
// argument reduction and a Taylor series, log by one Newton step on exp.
//
// On B300 a double-precision warp instruction occupies the FP64 pipe for 16
// cycles, so the FP64-class islands of the FP32 path (the centre rays that build
// the CDF) run in this type on the FP32 pipes instead.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rtu {

struct DF {
    float hi, lo;
    __device__ __forceinline__ DF() {}
    __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit DF(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __device__ __forceinline__ DF(float x) : hi(x), lo(0.0f) {}
    __device__ __forceinline__ DF(int x) : hi((float)x), lo(0.0f) {}
    __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ void df_quick(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// p + e = a b exactly
__device__ __forceinline__ void df_two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
    float s1, s2, t1, t2;
    df_two_sum(a.hi, b.hi, s1, s2);
    df_two_sum(a.lo, b.lo, t1, t2);
    s2 = __fadd_rn(s2, t1);
    df_quick(s1, s2, s1, s2);
    s2 = __fadd_rn(s2, t2);
    df_quick(s1, s2, s1, s2);
    return DF(s1, s2);
}
__device__ __forceinline__ DF operator-(const DF& a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(const DF& a, const DF& b) { return a + (-b); }
__device__ __forceinline__ DF operator*(const DF& a, const DF& b) {
    float p, e;
    df_two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df_quick(p, e, p, e);
    return DF(p, e);
}
__device__ __forceinline__ DF operator/(const DF& a, const DF& b) {
    // long division: three float quotient digits
    const float q1 = __fdiv_rn(a.hi, b.hi);
    DF r = a - b * DF(q1);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = r - b * DF(q2);
    const float q3 = __fdiv_rn(r.hi, b.hi);
    float s, e;
    df_quick(q1, q2, s, e);
    return DF(s, e) + DF(q3);
}
__device__ __forceinline__ DF& operator+=(DF& a, const DF& b) { a = a + b; return a; }
__device__ __forceinline__ DF& operator-=(DF& a, const DF& b) { a = a - b; return a; }
__device__ __forceinline__ DF& operator*=(DF& a, const DF& b) { a = a * b; return a; }
__device__ __forceinline__ bool operator<(const DF& a, const DF& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(const DF& a, const DF& b) { return b < a; }
__device__ __forceinline__ bool operator<=(const DF& a, const DF& b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(const DF& a, const DF& b) { return !(a < b); }
__device__ __forceinline__ bool operator==(const DF& a, const DF& b) { return a.hi == b.hi && a.lo == b.lo; }

__device__ __forceinline__ DF r_max(const DF& a, const DF& b) { return a < b ? b : a; }
__device__ __forceinline__ DF r_abs(const DF& a) { return a.hi < 0.0f ? -a : a; }

// sqrt: the float root refined by one Newton step y + (a - y^2) / (2 y)
__device__ __forceinline__ DF r_sqrt(const DF& a) {
    if (!(a.hi > 0.0f)) return DF(0.0f, 0.0f);
    const float y = sqrtf(a.hi);
    const DF y2 = DF(y) * DF(y);
    const float corr = __fdiv_rn((a - y2).hi, 2.0f * y);
    float s, e;
    df_quick(y, corr, s, e);
    return DF(s, e);
}
__device__ __forceinline__ void r_sqrt_inv(const DF& x, DF& R, DF& iR) {
    R = r_sqrt(x);
    iR = DF(1.0f) / R;
}

// exp: a = k ln2 + r, |r| <= ln2/2; exp(r) = (exp(r/16))^16 with the Taylor series of
// exp(r/16) to the 9th power of r/16 (|r/16| < 0.022: the next term is below 2^-56)
__device__ __forceinline__ DF r_exp(const DF& a) {
    if (a.hi > 88.0f) return DF(INFINITY, 0.0f);
    if (a.hi < -87.0f) return DF(0.0f, 0.0f);
    const DF ln2(0.6931471805599453);
    const float k = rintf(__fdiv_rn(a.hi, 0.6931472f));
    const DF r = (a - ln2 * DF(k)) * DF(0.0625f);
    DF term = r, sum = DF(1.0f) + r;
    for (int i = 2; i <= 9; ++i) {
        term = term * r * DF(1.0f / (float)i);
        sum = sum + term;
    }
    for (int i = 0; i < 4; ++i) sum = sum * sum;
    const int ki = (int)k;
    return DF(ldexpf(sum.hi, ki), ldexpf(sum.lo, ki));
}

// log: the float logarithm refined by one Newton step y + a exp(-y) - 1
__device__ __forceinline__ DF r_log(const DF& a) {
    const float y0 = logf(a.hi);
    const DF y(y0);
    return y + a * r_exp(-y) - DF(1.0f);
}

}  // namespace rtu
