// rtu_math.cuh -- scalar and forward-mode dual arithmetic, and the lens
// deflections (App. A) written once over a generic scalar so the same code
// gives values (float / double) and parameter derivatives (Dual<T, N>).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace rtu {

// ---------------------------------------------------------------- scalars
__device__ __forceinline__ float  r_sqrt(float x)  { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float  r_exp(float x)   { return expf(x); }
__device__ __forceinline__ double r_exp(double x)  { return exp(x); }
__device__ __forceinline__ float  r_log(float x)   { return logf(x); }
__device__ __forceinline__ double r_log(double x)  { return log(x); }
__device__ __forceinline__ float  r_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double r_log1p(double x){ return log1p(x); }
__device__ __forceinline__ float  r_cos(float x)   { return cosf(x); }
__device__ __forceinline__ double r_cos(double x)  { return cos(x); }
__device__ __forceinline__ float  r_sin(float x)   { return sinf(x); }
__device__ __forceinline__ double r_sin(double x)  { return sin(x); }
__device__ __forceinline__ float  r_atan2(float y, float x)   { return atan2f(y, x); }
__device__ __forceinline__ double r_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float  r_atan(float x)  { return atanf(x); }
__device__ __forceinline__ double r_atan(double x) { return atan(x); }
__device__ __forceinline__ float  r_atanh(float x) { return atanhf(x); }
__device__ __forceinline__ double r_atanh(double x){ return atanh(x); }
__device__ __forceinline__ float  r_abs(float x)   { return fabsf(x); }
__device__ __forceinline__ double r_abs(double x)  { return fabs(x); }

// ------------------------------------------------------------ dual numbers
// v + sum_i d[i] eps_i, eps_i eps_j = 0: forward-mode derivatives w.r.t. N seeds.
template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T x) : v(x) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    __device__ __forceinline__ static Dual seed(T x, int k) {
        Dual r(x);
        r.d[k] = T(1);
        return r;
    }
};

template <typename T> struct base_of { typedef T type; };
template <typename T, int N> struct base_of<Dual<T, N>> { typedef T type; };

template <typename T> __device__ __forceinline__ T val(T x) { return x; }
template <typename T, int N> __device__ __forceinline__ T val(const Dual<T, N>& x) { return x.v; }

#define RTU_DUAL_LOOP _Pragma("unroll") for (int i = 0; i < N; ++i)

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v + b.v; RTU_DUAL_LOOP r.d[i] = a.d[i] + b.d[i]; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v - b.v; RTU_DUAL_LOOP r.d[i] = a.d[i] - b.d[i]; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a) {
    Dual<T, N> r; r.v = -a.v; RTU_DUAL_LOOP r.d[i] = -a.d[i]; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v * b.v; RTU_DUAL_LOOP r.d[i] = a.v * b.d[i] + a.d[i] * b.v; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v / b.v; T ib = T(1) / b.v;
    RTU_DUAL_LOOP r.d[i] = (a.d[i] - r.v * b.d[i]) * ib; return r;
}
// mixed with the base scalar
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v += b; return r; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(T b, const Dual<T, N>& a) { Dual<T, N> r = a; r.v += b; return r; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v -= b; return r; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(T b, const Dual<T, N>& a) {
    Dual<T, N> r; r.v = b - a.v; RTU_DUAL_LOOP r.d[i] = -a.d[i]; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, T b) {
    Dual<T, N> r; r.v = a.v * b; RTU_DUAL_LOOP r.d[i] = a.d[i] * b; return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(T b, const Dual<T, N>& a) { return a * b; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, T b) { return a * (T(1) / b); }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(T a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a / b.v; T s = -r.v / b.v; RTU_DUAL_LOOP r.d[i] = s * b.d[i]; return r;
}

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> chain(const Dual<T, N>& a, T fv, T dfdv) {
    Dual<T, N> r; r.v = fv; RTU_DUAL_LOOP r.d[i] = dfdv * a.d[i]; return r;
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_sqrt(const Dual<T, N>& a) {
    T s = r_sqrt(a.v); return chain(a, s, T(0.5) / s);
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_exp(const Dual<T, N>& a) {
    T e = r_exp(a.v); return chain(a, e, e);
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_log(const Dual<T, N>& a) {
    return chain(a, r_log(a.v), T(1) / a.v);
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_cos(const Dual<T, N>& a) {
    return chain(a, r_cos(a.v), -r_sin(a.v));
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_sin(const Dual<T, N>& a) {
    return chain(a, r_sin(a.v), r_cos(a.v));
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_atan(const Dual<T, N>& a) {
    return chain(a, r_atan(a.v), T(1) / (T(1) + a.v * a.v));
}
template <typename T, int N> __device__ __forceinline__ Dual<T, N> r_atanh(const Dual<T, N>& a) {
    return chain(a, r_atanh(a.v), T(1) / (T(1) - a.v * a.v));
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> r_atan2(const Dual<T, N>& y, const Dual<T, N>& x) {
    Dual<T, N> r; r.v = r_atan2(y.v, x.v);
    T den = x.v * x.v + y.v * y.v;
    T ax = (den > T(0)) ? x.v / den : T(0), ay = (den > T(0)) ? y.v / den : T(0);
    RTU_DUAL_LOOP r.d[i] = ax * y.d[i] - ay * x.d[i];
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> r_max(const Dual<T, N>& a, T lo) {
    return a.v >= lo ? a : Dual<T, N>(lo);
}
template <typename T> __device__ __forceinline__ T r_max(T a, T lo) { return a >= lo ? a : lo; }

// cast between base types (value and derivatives)
template <typename To, typename From> struct caster {
    __device__ __forceinline__ static To go(const From& x) { return To(x); }
};
template <typename To, typename From, int N> struct caster<Dual<To, N>, Dual<From, N>> {
    __device__ __forceinline__ static Dual<To, N> go(const Dual<From, N>& x) {
        Dual<To, N> r; r.v = To(x.v);
#pragma unroll
        for (int i = 0; i < N; ++i) r.d[i] = To(x.d[i]);
        return r;
    }
};
template <typename To, typename From> __device__ __forceinline__ To cast(const From& x) {
    return caster<To, From>::go(x);
}

// ----------------------------------------------------------- deflections
// EPL (Eq. A1): kappa = (3-gamma)/2 (theta_E/rho)^(gamma-1), rho^2 = q x'^2 + y'^2/q.
// Deflection by the Tessore & Metcalf (2015) series of
// 2F1(1, t/2; 2 - t/2; -f e^{2 i vphi}) with R^2 = q^2 x'^2 + y'^2, b = theta_E sqrt(q),
// t = gamma - 1, f = (1-q)/(1+q), e^{i vphi} = (q x' + i y')/R.  All rays of a
// system see the same term magnitudes |Omega_n| (|e^{2 i vphi}| = 1), so the
// stopping index is uniform across a warp.  `tol` is the absolute term size at
// which the sum stops.
template <typename S>
__device__ __forceinline__ void epl_deflect(const S& x, const S& y, const S& thE, const S& gam,
                                            const S& e1, const S& e2, const S& x0, const S& y0,
                                            S& ax, S& ay,
                                            typename base_of<S>::type tol, int max_terms) {
    typedef typename base_of<S>::type T;
    S cc = r_sqrt(r_max(e1 * e1 + e2 * e2, T(1e-30)));
    S q = (T(1) - cc) / (T(1) + cc);
    S phi = T(0.5) * r_atan2(e2, e1);
    S cp = r_cos(phi), sp = r_sin(phi);
    S dx = x - x0, dy = y - y0;
    S xr = cp * dx + sp * dy;
    S yr = sp * dx;
    yr = cp * dy - yr;
    S t = gam - T(1);
    S b = thE * r_sqrt(q);
    S R = r_sqrt(r_max(q * q * xr * xr + yr * yr, T(1e-20)));
    S iR = T(1) / R;
    S cre = q * xr * iR, cim = yr * iR;                 // e^{i vphi}
    S wre = cre * cre - cim * cim, wim = T(2) * cre * cim;  // e^{2 i vphi}
    S f = (T(1) - q) / (T(1) + q);
    S tre = cre, tim = cim;                             // Omega_0
    S sre = tre, sim = tim;
    S two_m_t = T(2) - t;
    for (int n = 1; n < max_terms; ++n) {
        S c = -f * (T(2 * n) - two_m_t) / (T(2 * n) + two_m_t);
        S nre = tre * wre - tim * wim;
        S nim = tre * wim + tim * wre;
        tre = c * nre;
        tim = c * nim;
        sre = sre + tre;
        sim = sim + tim;
        T mag = r_abs(val(tre)) + r_abs(val(tim));
        if (mag <= tol) break;
    }
    S pref = T(2) * b / (T(1) + q) * r_exp((t - T(1)) * r_log(b * iR));
    S axr = pref * sre, ayr = pref * sim;
    ax = cp * axr - sp * ayr;
    ay = sp * axr + cp * ayr;
}

// F(x) of Eq. A3 with the series sum_k w^k/(2k+1), w = 1 - x^2, near x = 1.
template <typename S>
__device__ __forceinline__ S nfw_F(const S& x) {
    typedef typename base_of<S>::type T;
    S w = T(1) - x * x;
    T wv = val(w);
    if (r_abs(wv) < T(1e-2)) {
        S s(T(0));
        S p(T(1));
#pragma unroll 1
        for (int k = 0; k < 14; ++k) {
            s = s + p * (T(1) / T(2 * k + 1));
            p = p * w;
        }
        return s;
    }
    if (wv > T(0)) {
        S sq = r_sqrt(w);
        return r_atanh(sq) / sq;
    }
    S sq = r_sqrt(T(0) - w);
    return r_atan(sq) / sq;
}

// Projected mass functions: alpha(r) = 4 kappa_s r_s g(x)/x, x = r/r_s.
// NFW: g = ln(x/2) + F(x).  Truncated NFW (Baltz, Marshall & Oguri 2009, density
// times tau^2/(tau^2 + x^2)).
template <typename S>
__device__ __forceinline__ S nfw_g(const S& x, const S& tau, int kind) {
    typedef typename base_of<S>::type T;
    S F = nfw_F(x);
    if (kind == 1) return r_log(x * T(0.5)) + F;
    S t2 = tau * tau;
    S sq = r_sqrt(t2 + x * x);
    S L = r_log(x / (sq + tau));
    S t21 = t2 + T(1);
    const T pi = T(3.14159265358979323846);
    S body = (t21 + T(2) * (x * x - T(1))) * F + tau * pi + (t2 - T(1)) * r_log(tau)
             + sq * (L * (t2 - T(1)) / tau - pi);
    return t2 / (t21 * t21) * body;
}

template <typename S>
__device__ __forceinline__ void nfw_deflect(const S& x, const S& y, const S& ks, const S& rs,
                                            const S& tau, const S& xs, const S& ys, int kind,
                                            S& ax, S& ay) {
    typedef typename base_of<S>::type T;
    S dx = x - xs, dy = y - ys;
    S r = r_sqrt(r_max(dx * dx + dy * dy, T(1e-20)));
    S xx = r / rs;
    S a = T(4) * ks * rs * nfw_g(xx, tau, kind) / xx / r;
    ax = a * dx;
    ay = a * dy;
}

}  // namespace rtu
