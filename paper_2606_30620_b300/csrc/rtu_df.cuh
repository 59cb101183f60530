// rtu_df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits (the arithmetic below
// keeps relative errors of a few 2^-48 for values above 2^-100, where the low float
// is still normal; the tests bound exp, log, sqrt and the quotient against FP64 at
// 2^-46).  Built from the
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
// the EPL series' evaluation takes its float tail for this type (the primary
// template, false, is in rtu_math.cuh)
template <typename T> struct epl_pair_type;
template <> struct epl_pair_type<DF> { static constexpr bool value = true; };
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

// exp: a = k ln2 + r with ln2 split in three floats (the first of 15 significant bits,
// so k times it is exact for |k| < 2^9: the reduction adds no error of k ln2), then
// exp(r), |r| <= ln2/2, by Horner's rule over the Taylor coefficients 1/i!, i <= 12,
// each a double-float pair (the dropped terms are below 2^-52 of the sum), and the
// exact scaling by 2^k.  Measured against FP64 (tests): relative error below 2^-46.
__device__ __forceinline__ DF r_exp(const DF& a) {
    if (a.hi > 88.0f) return DF(INFINITY, 0.0f);
    if (a.hi < -87.0f) return DF(0.0f, 0.0f);
    const float k = rintf(__fmul_rn(a.hi, 1.44269504f));
    float p, e;
    DF r = a - DF(__fmul_rn(k, 0.693145751953125f), 0.0f);
    df_two_prod(k, 1.428606765330187e-06f, p, e);
    r = r - DF(p, e);
    r = r - DF(__fmul_rn(k, 5.497923148104107e-14f), 0.0f);
    // 1/i! as (hi, lo) float pairs, i = 0..12
    const float ch[13] = {1.0f, 1.0f, 0.5f, 0.1666666716337204f, 0.0416666679084301f, 0.008333333767950535f,
                          0.0013888889225199819f, 0.00019841270113829523f, 2.4801587642286904e-05f,
                          2.7557318844628753e-06f, 2.755731998149713e-07f, 2.5052107943679403e-08f,
                          2.0876755879584152e-09f};
    const float cl[13] = {0.0f, 0.0f, 0.0f, -4.967053879312289e-09f, -1.2417634698280722e-09f,
                          -4.34617203337595e-10f, -3.3631094437103215e-11f, -2.725596874933456e-12f,
                          -3.40699609366682e-13f, 3.793571224297229e-14f, -7.575112209051195e-15f,
                          4.4176230446483665e-16f, 1.1082839147459852e-16f};
    DF sum(ch[12], cl[12]);
#pragma unroll
    for (int i = 11; i >= 0; --i) sum = sum * r + DF(ch[i], cl[i]);
    const int ki = (int)k;
    return DF(ldexpf(sum.hi, ki), ldexpf(sum.lo, ki));
}

// log: the float logarithm y0 corrected by log(a exp(-y0)) = log(1 + u) = u - u^2/2 + ...
// with u = a exp(-y0) - 1 (|u| ~ |log a| 2^-24): the u^2/2 term, small, in float; the
// dropped u^3/3 is below 2^-60 for |log a| < 100
__device__ __forceinline__ DF r_log(const DF& a) {
    const float y0 = logf(a.hi);
    const DF u = a * r_exp(DF(-y0, 0.0f)) - DF(1.0f);
    return DF(y0, 0.0f) + u - DF(__fmul_rn(0.5f, __fmul_rn(u.hi, u.hi)), 0.0f);
}

}  // namespace rtu
