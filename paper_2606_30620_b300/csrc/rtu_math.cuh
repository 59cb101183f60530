// rtu_math.cuh -- scalar and forward-mode dual arithmetic, and the lens
// deflections (App. A) written once over a generic scalar so the same code
// gives values (float / double) and parameter derivatives (Dual<T, N>).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef RTU_HD
#define RTU_HD __host__ __device__ __forceinline__
#endif

namespace rtu {

// ---------------------------------------------------------------- scalars
RTU_HD float  r_sqrt(float x)  { return sqrtf(x); }
RTU_HD double r_sqrt(double x) { return sqrt(x); }
RTU_HD float  r_exp(float x)   { return expf(x); }
RTU_HD double r_exp(double x)  { return exp(x); }
RTU_HD float  r_log(float x)   { return logf(x); }
RTU_HD double r_log(double x)  { return log(x); }
RTU_HD float  r_log1p(float x) { return log1pf(x); }
RTU_HD double r_log1p(double x){ return log1p(x); }
RTU_HD float  r_cos(float x)   { return cosf(x); }
RTU_HD double r_cos(double x)  { return cos(x); }
RTU_HD float  r_sin(float x)   { return sinf(x); }
RTU_HD double r_sin(double x)  { return sin(x); }
RTU_HD float  r_atan2(float y, float x)   { return atan2f(y, x); }
RTU_HD double r_atan2(double y, double x) { return atan2(y, x); }
RTU_HD float  r_atan(float x)  { return atanf(x); }
RTU_HD double r_atan(double x) { return atan(x); }
RTU_HD float  r_atanh(float x) { return atanhf(x); }
RTU_HD double r_atanh(double x){ return atanh(x); }
// R = sqrt(x) and 1/R: one reciprocal square root in float, exact ops in double
RTU_HD void r_sqrt_inv(float x, float& R, float& iR) {
#ifdef __CUDA_ARCH__
    iR = rsqrtf(x);
#else
    iR = 1.0f / sqrtf(x);
#endif
    R = x * iR;
}
RTU_HD void r_sqrt_inv(double x, double& R, double& iR) {
    R = sqrt(x);
    iR = 1.0 / R;
}
RTU_HD float  r_abs(float x)   { return fabsf(x); }
RTU_HD double r_abs(double x)  { return fabs(x); }

// Unsigned division by a run-time invariant d (1 <= d < 2^32) as a multiply-high
// and two shifts, exact for every 32-bit numerator: the round-up method of
// Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), Sec. 4 / Fig. 4.1, with N = 32.
struct UDiv {
    uint32_t m, s1, s2;
};
RTU_HD UDiv udiv_make(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;                 // l = ceil(log2 d)
    const uint64_t mm = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    UDiv u;
    u.m = (uint32_t)mm;
    u.s1 = l < 1 ? l : 1;
    u.s2 = l > 1 ? l - 1 : 0;
    return u;
}
RTU_HD uint32_t udiv(uint32_t n, const UDiv& u) {
#ifdef __CUDA_ARCH__
    const uint32_t t1 = __umulhi(u.m, n);
#else
    const uint32_t t1 = (uint32_t)(((uint64_t)u.m * n) >> 32);
#endif
    return (t1 + ((n - t1) >> u.s1)) >> u.s2;
}

// ------------------------------------------------------------ dual numbers
// v + sum_i d[i] eps_i, eps_i eps_j = 0: forward-mode derivatives w.r.t. N seeds.
template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    RTU_HD Dual() {}
    RTU_HD Dual(T x) : v(x) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    RTU_HD static Dual seed(T x, int k) {
        Dual r(x);
        r.d[k] = T(1);
        return r;
    }
};

template <typename T> struct base_of { typedef T type; };
template <typename T, int N> struct base_of<Dual<T, N>> { typedef T type; };

template <typename T> RTU_HD T val(T x) { return x; }
template <typename T, int N> RTU_HD T val(const Dual<T, N>& x) { return x.v; }

#define RTU_DUAL_LOOP _Pragma("unroll") for (int i = 0; i < N; ++i)

template <typename T, int N>
RTU_HD Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v + b.v; RTU_DUAL_LOOP r.d[i] = a.d[i] + b.d[i]; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v - b.v; RTU_DUAL_LOOP r.d[i] = a.d[i] - b.d[i]; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator-(const Dual<T, N>& a) {
    Dual<T, N> r; r.v = -a.v; RTU_DUAL_LOOP r.d[i] = -a.d[i]; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v * b.v; RTU_DUAL_LOOP r.d[i] = a.v * b.d[i] + a.d[i] * b.v; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a.v / b.v; T ib = T(1) / b.v;
    RTU_DUAL_LOOP r.d[i] = (a.d[i] - r.v * b.d[i]) * ib; return r;
}
// mixed with the base scalar
template <typename T, int N>
RTU_HD Dual<T, N> operator+(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v += b; return r; }
template <typename T, int N>
RTU_HD Dual<T, N> operator+(T b, const Dual<T, N>& a) { Dual<T, N> r = a; r.v += b; return r; }
template <typename T, int N>
RTU_HD Dual<T, N> operator-(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v -= b; return r; }
template <typename T, int N>
RTU_HD Dual<T, N> operator-(T b, const Dual<T, N>& a) {
    Dual<T, N> r; r.v = b - a.v; RTU_DUAL_LOOP r.d[i] = -a.d[i]; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator*(const Dual<T, N>& a, T b) {
    Dual<T, N> r; r.v = a.v * b; RTU_DUAL_LOOP r.d[i] = a.d[i] * b; return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> operator*(T b, const Dual<T, N>& a) { return a * b; }
template <typename T, int N>
RTU_HD Dual<T, N> operator/(const Dual<T, N>& a, T b) { return a * (T(1) / b); }
template <typename T, int N>
RTU_HD Dual<T, N> operator/(T a, const Dual<T, N>& b) {
    Dual<T, N> r; r.v = a / b.v; T s = -r.v / b.v; RTU_DUAL_LOOP r.d[i] = s * b.d[i]; return r;
}

template <typename T, int N>
RTU_HD Dual<T, N> chain(const Dual<T, N>& a, T fv, T dfdv) {
    Dual<T, N> r; r.v = fv; RTU_DUAL_LOOP r.d[i] = dfdv * a.d[i]; return r;
}
template <typename T, int N> RTU_HD Dual<T, N> r_sqrt(const Dual<T, N>& a) {
    T s = r_sqrt(a.v); return chain(a, s, T(0.5) / s);
}
template <typename T, int N> RTU_HD Dual<T, N> r_exp(const Dual<T, N>& a) {
    T e = r_exp(a.v); return chain(a, e, e);
}
template <typename T, int N> RTU_HD Dual<T, N> r_log(const Dual<T, N>& a) {
    return chain(a, r_log(a.v), T(1) / a.v);
}
template <typename T, int N> RTU_HD Dual<T, N> r_cos(const Dual<T, N>& a) {
    return chain(a, r_cos(a.v), -r_sin(a.v));
}
template <typename T, int N> RTU_HD Dual<T, N> r_sin(const Dual<T, N>& a) {
    return chain(a, r_sin(a.v), r_cos(a.v));
}
template <typename T, int N> RTU_HD Dual<T, N> r_atan(const Dual<T, N>& a) {
    return chain(a, r_atan(a.v), T(1) / (T(1) + a.v * a.v));
}
template <typename T, int N> RTU_HD Dual<T, N> r_atanh(const Dual<T, N>& a) {
    return chain(a, r_atanh(a.v), T(1) / (T(1) - a.v * a.v));
}
template <typename T, int N>
RTU_HD Dual<T, N> r_atan2(const Dual<T, N>& y, const Dual<T, N>& x) {
    Dual<T, N> r; r.v = r_atan2(y.v, x.v);
    T den = x.v * x.v + y.v * y.v;
    T ax = (den > T(0)) ? x.v / den : T(0), ay = (den > T(0)) ? y.v / den : T(0);
    RTU_DUAL_LOOP r.d[i] = ax * y.d[i] - ay * x.d[i];
    return r;
}
template <typename T, int N>
RTU_HD Dual<T, N> r_max(const Dual<T, N>& a, T lo) {
    return a.v >= lo ? a : Dual<T, N>(lo);
}
template <typename T> RTU_HD T r_max(T a, T lo) { return a >= lo ? a : lo; }

// cast between base types (value and derivatives)
template <typename To, typename From> struct caster {
    RTU_HD static To go(const From& x) { return To(x); }
};
template <typename To, typename From, int N> struct caster<Dual<To, N>, Dual<From, N>> {
    RTU_HD static Dual<To, N> go(const Dual<From, N>& x) {
        Dual<To, N> r; r.v = To(x.v);
#pragma unroll
        for (int i = 0; i < N; ++i) r.d[i] = To(x.d[i]);
        return r;
    }
};
template <typename To, typename From> RTU_HD To cast(const From& x) {
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
RTU_HD void epl_deflect(const S& x, const S& y, const S& thE, const S& gam,
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
RTU_HD S nfw_F(const S& x) {
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
RTU_HD S nfw_g(const S& x, const S& tau, int kind) {
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
RTU_HD void nfw_deflect(const S& x, const S& y, const S& ks, const S& rs,
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

// ------------------------------------------------ EPL with per-system constants
// The Tessore & Metcalf series of the deflection of Eq. A1 split into what
// depends on the lens only (computed once per system in double) and the per-ray
// part, plus its analytic vector-Jacobian product with respect to
// (theta_E, gamma, e1, e2, x0, y0).
//
// Term n of the series is Omega_n = c_n w Omega_{n-1} with the lens-only factors
// c_n = -f (2n - 2 + t)/(2n + 2 - t) and w = e^{2 i vphi}, so Omega_n = A_n w^n Omega_0
// with A_n = c_1 ... c_n: every sum the deflection and its derivatives need is
// Omega_0 times a polynomial in w with lens-only real coefficients, evaluated per ray
// by Horner's rule (independent chains for the four sums of the adjoint).
constexpr int EPL_MAXT = 96;

// the coefficients of w^n, n = 0..nterm, of the series sums
//   S = sum Omega_n:              a_n = A_n
//   U = sum D_n Omega_n:          u_n = D_n A_n, D_n = sum_{k <= n} d log|c_k| / dt
// The two other sums of the derivatives follow from S and S' = dS/dw, since
// A_n = f g_n A_{n-1} (g_n = c_n / f):
//   H = sum (2n+1) Omega_n = S + 2 w S',   F = sum n g_n A_{n-1} w^n = w S' / f.
// one 8-byte (float) or 16-byte (double) shared-memory load per power
template <typename T>
struct __align__(2 * sizeof(T) >= 16 ? 16 : 2 * sizeof(T)) EplTerm {
    T a, u;
};

template <typename T>
struct EplC {
    T x0, y0, cp, sp, q, cc, e1, e2, thE, sq, b, t, pref0, lnb, opq;
    // lens-only factors of the vector-Jacobian product: dF/dq through f,
    // (t/b) db/dq, (t/b) db/dtheta_E, 1/(1+q), the (e1, e2) chain factors
    T f_q, tb_bq, tb_sq, iopq, qe1, qe2, pe1, pe2;
    T ftail;          // f / (1 - f): the series tail factor, f = (1 - q)/(1 + q)
    T ic;             // 1 / f
    int nterm;        // highest power of w
    EplTerm<T> term[EPL_MAXT + 1];
};

// whether T is the double-float pair type (specialised where that type is defined)
template <typename T> struct epl_pair_type { static constexpr bool value = false; };

// the lens-only scalars of the series (everything but the term tables), written with
// as few divisions and roots as the algebra allows (FP64 divides, roots and
// transcendentals are long serial chains on this part): with c = |(e1, e2)|,
// q = (1 - c)/(1 + c) gives f = (1 - q)/(1 + q) = c, 1 + q = 2/(1 + c), and the
// position angle's cos, sin follow from cos 2 phi = e1/c, sin 2 phi = e2/c by the
// half-angle formulas (phi = atan2(e2, e1)/2 in (-pi/2, pi/2], so cos phi >= 0 and
// sin phi takes the sign of e2).
// In three independent parts, so that three threads can take one chain each (the
// caller passes c = sqrt(max(e1^2 + e2^2, 1e-30))):
//   part 0  the frame (cos phi, sin phi), 1/f and the angle's chain factors
//   part 1  q, sqrt q, b = theta_E sqrt q, log b and the factors of 1 + q
//   part 2  dq/de1, dq/de2, the tail factor f/(1 - f) and (t/b) db/dtheta_E
constexpr int EPL_NSCAL = 25;      // the leading members of EplC, x0 .. ic, all of type T
template <typename T>
RTU_HD void epl_scalars_part(EplC<T>& C, const double* p, bool epl, double cc, int part) {
    const double e1 = p[2], e2 = p[3];
    const double t = (epl ? p[1] : 2.0) - 1.0;
    if (part == 0) {
        const double icc = 1.0 / cc;
        const double c2 = e1 * icc, s2 = e2 * icc;       // cos 2 phi, sin 2 phi
        double cp, sp;
        if (e1 == 0.0 && e2 == 0.0) {
            cp = 1.0;                                    // a round lens: phi = atan2(0, 0)/2 = 0
            sp = 0.0;
        } else if (c2 >= 0.0) {
            cp = sqrt(0.5 * (1.0 + c2));
            sp = 0.5 * s2 / cp;
        } else {
            sp = sqrt(0.5 * (1.0 - c2));
            if (s2 < 0.0) sp = -sp;
            cp = 0.5 * fabs(s2) / fabs(sp);
        }
        C.x0 = (T)p[4]; C.y0 = (T)p[5]; C.cp = (T)cp; C.sp = (T)sp; C.cc = (T)cc;
        C.e1 = (T)e1; C.e2 = (T)e2; C.thE = (T)p[0]; C.t = (T)t;
        C.pe1 = (T)(0.5 * c2 * icc);                    // dphi/de2 coefficient: e1/(2 c^2)
        C.pe2 = (T)(0.5 * s2 * icc);                    // -dphi/de1 coefficient: e2/(2 c^2)
        C.ic = (T)icc;                                  // 1/f
    } else if (part == 1) {
        const double i1pc = 1.0 / (1.0 + cc);
        const double q = (1.0 - cc) * i1pc;
        const double sq = sqrt(q);
        const double b = p[0] * sq;
        C.q = (T)q; C.sq = (T)sq; C.b = (T)b;
        C.pref0 = (T)(b * (1.0 + cc));                  // 2 b/(1 + q)
        C.lnb = (T)log(b); C.opq = (T)(2.0 * i1pc);     // 1 + q
        C.f_q = (T)(-0.5 * (1.0 + cc) * (1.0 + cc));    // df/dq = -2/(1 + q)^2
        C.tb_bq = (T)(0.5 * t / q);                     // (t/b) db/dq, b = theta_E sqrt(q)
        C.iopq = (T)(0.5 * (1.0 + cc));                 // 1/(1 + q)
    } else {
        const double icc = 1.0 / cc, i1pc = 1.0 / (1.0 + cc);
        const double c2 = e1 * icc, s2 = e2 * icc;
        const double q_c = -2.0 * i1pc * i1pc;          // dq/dc
        C.qe1 = (T)(q_c * c2);                          // dq/de1 = q_c e1/c
        C.qe2 = (T)(q_c * s2);                          // dq/de2 = q_c e2/c
        C.ftail = (T)(cc / (1.0 - cc));                 // f/(1 - f), f = c
        C.tb_sq = (T)(t / p[0]);                        // (t/b) db/dtheta_E
    }
}

template <typename T>
RTU_HD void epl_scalars(EplC<T>& C, const double* p, bool epl) {
    const double cc = sqrt(fmax(p[2] * p[2] + p[3] * p[3], 1e-30));
    for (int part = 0; part < 3; ++part) epl_scalars_part(C, p, epl, cc, part);
}

// coefficient n >= 1 of the two sums from A_{n-1} (running), c_n and D_n
template <typename T>
RTU_HD void epl_term(EplTerm<T>& tm, double A_prev, double c, double D) {
    const double A = A_prev * c;
    tm.a = (T)A;
    tm.u = (T)(D * A);
}
template <typename T>
RTU_HD void epl_term0(EplTerm<T>& tm) {
    tm.a = T(1); tm.u = T(0);
}

// p = theta_E, gamma, e1, e2, x0, y0 (gamma ignored unless epl); tol = size of the
// last summed term relative to the leading one
template <typename T>
RTU_HD void epl_setup(EplC<T>& C, const double* p, bool epl, double tol) {
    epl_scalars(C, p, epl);
    const double cc = sqrt(fmax(p[2] * p[2] + p[3] * p[3], 1e-30));
    const double q = (1.0 - cc) / (1.0 + cc);
    const double t = (epl ? p[1] : 2.0) - 1.0;
    const double f = (1.0 - q) / (1.0 + q);
    double A = 1.0, D = 0.0;
    epl_term0(C.term[0]);
    int n = 1;
    for (; n <= EPL_MAXT; ++n) {
        const double g = -(2.0 * n - 2.0 + t) / (2.0 * n + 2.0 - t);
        const double c = f * g;
        D += 1.0 / (2.0 * n - 2.0 + t) + 1.0 / (2.0 * n + 2.0 - t);
        epl_term(C.term[n], A, c, D);
        A *= c;
        if (fabs(A) <= tol) break;
    }
    C.nterm = n > EPL_MAXT ? EPL_MAXT : n;
}

// sum_{n=lo..hi} k_n w^n by Horner's rule (k_n = member `K` of term n)
#define RTU_EPL_HORNER(K, lo, hi, outr, outi)                                  \
    {                                                                          \
        outr = C.term[hi].K;                                                   \
        outi = T(0);                                                           \
        for (int n_ = (hi) - 1; n_ >= (lo); --n_) {                            \
            const T nr_ = outr * wre - outi * wim + C.term[n_].K;              \
            outi = outr * wim + outi * wre;                                    \
            outr = nr_;                                                        \
        }                                                                      \
    }

// The deflection in two parts: the first terms of the series (with the
// prefactor P), then all of it.  Between them, epl_tail_bound bounds what the
// remaining terms can add: |c_n| < f for 0 < t < 2 and |w| = 1, so the terms beyond
// power m add at most P |A_m| f / (1 - f).  finish evaluates the whole polynomial,
// exactly as epl_alpha does, so a ray that finishes gets the same bits.
template <typename T>
struct EplPart {
    T cre, cim, wre, wim, P, sre, sim;
    int m;
};

template <typename T>
RTU_HD void epl_alpha_begin(const EplC<T>& C, T x, T y, int m, EplPart<T>& s) {
    const T dx = x - C.x0, dy = y - C.y0;
    const T xr = C.cp * dx + C.sp * dy, yr = C.cp * dy - C.sp * dx;
    const T R2 = r_max(C.q * C.q * xr * xr + yr * yr, T(1e-20));
    T R, iR;
    r_sqrt_inv(R2, R, iR);
    const T cre = C.q * xr * iR, cim = yr * iR;
    const T wre = cre * cre - cim * cim, wim = T(2) * cre * cim;
    s.cre = cre; s.cim = cim; s.wre = wre; s.wim = wim;
    s.P = C.pref0 * r_exp((C.t - T(1)) * (C.lnb - r_log(R)));
    s.m = m < C.nterm ? m : C.nterm;
    T pr, pi;
    RTU_EPL_HORNER(a, 0, s.m, pr, pi);
    s.sre = cre * pr - cim * pi;
    s.sim = cre * pi + cim * pr;
}

// alpha from the terms summed so far
template <typename T>
RTU_HD void epl_alpha_of(const EplC<T>& C, const EplPart<T>& s, T& ax, T& ay) {
    const T axr = s.P * s.sre, ayr = s.P * s.sim;
    ax = C.cp * axr - C.sp * ayr;
    ay = C.sp * axr + C.cp * ayr;
}

template <typename T>
RTU_HD T epl_tail_bound(const EplC<T>& C, const EplPart<T>& s) {
    if (s.m >= C.nterm) return T(0);
    return s.P * r_abs(C.term[s.m].a) * C.ftail;
}

// nsplit: for the double-float type, the first power summed in float (|A_n| <= 1e-9)
template <typename T>
RTU_HD void epl_alpha_finish(const EplC<T>& C, EplPart<T>& s, T& ax, T& ay, int nsplit = 1 << 30) {
    const T wre = s.wre, wim = s.wim;
    T pr, pi;
    if (sizeof(T) == 4) {
        // float (the forward render): the loop unrolled by four (measured 1.3% faster)
        pr = C.term[C.nterm].a;
        pi = T(0);
#pragma unroll 4
        for (int n = C.nterm - 1; n >= 0; --n) {
            const T nr = pr * wre - pi * wim + C.term[n].a;
            pi = pr * wim + pi * wre;
            pr = nr;
        }
    } else if constexpr (epl_pair_type<T>::value) {
        // double-float: Horner's rule over the powers n >= nsplit in float (|A_n| <=
        // 1e-9, so the float rounding of that tail is below 1e-16 of the leading
        // term), continued in the pair type over the rest
        const int N = C.nterm, m = nsplit < N ? nsplit : N;
        float fr = C.term[N].a.hi, fi = 0.0f;
        const float wr = wre.hi, wi = wim.hi;
        for (int n = N - 1; n >= m; --n) {
            const float nr = fr * wr - fi * wi + C.term[n].a.hi;
            fi = fr * wi + fi * wr;
            fr = nr;
        }
        pr = T(fr);
        pi = T(fi);
        for (int n = m - 1; n >= 0; --n) {
            const T nr = pr * wre - pi * wim + C.term[n].a;
            pi = pr * wim + pi * wre;
            pr = nr;
        }
    } else {
        RTU_EPL_HORNER(a, 0, C.nterm, pr, pi);
    }
    s.sre = s.cre * pr - s.cim * pi;
    s.sim = s.cre * pi + s.cim * pr;
    s.m = C.nterm;
    epl_alpha_of(C, s, ax, ay);
}

template <typename T>
RTU_HD void epl_alpha(const EplC<T>& C, T x, T y, T& ax, T& ay, int nsplit = 1 << 30) {
    EplPart<T> s;
    epl_alpha_begin(C, x, y, 0, s);
    epl_alpha_finish(C, s, ax, ay, nsplit);
}

// Per-ray intermediates of the EPL deflection kept for the vector-Jacobian product.
template <typename T>
struct EplJ {
    T xr, yr, iR, P, lbR, are, aim, ax, ay, hre, him, ure, uim, fre, fim;
};

// deflection alpha = (ax, ay) plus the series sums needed for its derivatives
template <typename T>
RTU_HD void epl_eval(const EplC<T>& C, bool want_t, T x, T y, EplJ<T>& J) {
    const T dx = x - C.x0, dy = y - C.y0;
    const T xr = C.cp * dx + C.sp * dy, yr = C.cp * dy - C.sp * dx;
    const T q = C.q;
    const T R2 = r_max(q * q * xr * xr + yr * yr, T(1e-20));
    T R, iR;
    r_sqrt_inv(R2, R, iR);
    const T cre = q * xr * iR, cim = yr * iR;
    const T wre = cre * cre - cim * cim, wim = T(2) * cre * cim;
    // S, its derivative S' and U by Horner's rule, in one loop (independent chains;
    // the derivative's step takes S's running value before S's own step)
    const int N = C.nterm;
    T ar = C.term[N].a, ai = T(0), dr = T(0), di = T(0);
    T ur = C.term[N].u, ui = T(0);
    // one Horner step of the three chains at term n
    auto step3 = [&](int n) {
        const EplTerm<T> tm = C.term[n];
        const T dr2 = dr * wre - di * wim + ar;
        di = dr * wim + di * wre + ai;
        dr = dr2;
        const T ar2 = ar * wre - ai * wim + tm.a;
        ai = ar * wim + ai * wre;
        ar = ar2;
        if (want_t) {
            const T ur2 = ur * wre - ui * wim + tm.u;
            ui = ur * wim + ui * wre;
            ur = ur2;
        }
    };
#pragma unroll 1
    for (int n = N - 1; n >= 0; --n) step3(n);
    const T sre = cre * ar - cim * ai, sim = cre * ai + cim * ar;
    const T lbR = C.lnb - r_log(R);
    const T P = C.pref0 * r_exp((C.t - T(1)) * lbR);
    J.xr = xr; J.yr = yr; J.iR = iR; J.P = P; J.lbR = lbR;
    J.are = P * sre; J.aim = P * sim;
    J.ax = C.cp * J.are - C.sp * J.aim;
    J.ay = C.sp * J.are + C.cp * J.aim;
    // w S', then H = S + 2 w S' and F = w S' / f
    const T vr = wre * dr - wim * di, vi = wre * di + wim * dr;
    const T hr = ar + T(2) * vr, hi = ai + T(2) * vi;
    const T fr = vr * C.ic, fi = vi * C.ic;
    J.hre = cre * hr - cim * hi; J.him = cre * hi + cim * hr;
    if (want_t) { J.ure = cre * ur - cim * ui; J.uim = cre * ui + cim * ur; }
    else { J.ure = T(0); J.uim = T(0); }
    J.fre = cre * fr - cim * fi; J.fim = cre * fi + cim * fr;
}

// out[k] += Re(conj(G) d alpha / d p_k), G = (gx, gy) = dL/d alpha,
// p = (theta_E, gamma, e1, e2, x0, y0); gamma only when want_t
template <typename T>
RTU_HD void epl_vjp(const EplC<T>& C, const EplJ<T>& J, bool want_t, T gx, T gy, T* out) {
    const T q = C.q, t = C.t, xr = J.xr, yr = J.yr, iR = J.iR, P = J.P;
    const T sthr = -J.him, sthi = J.hre;                 // S_theta = i sum (2n+1) Omega_n
    const T iR2 = iR * iR;
    const T th_xr = -yr * q * iR2, th_yr = q * xr * iR2, th_q = -yr * xr * iR2;
    const T R_xr = q * q * xr * iR, R_yr = yr * iR, R_q = q * xr * xr * iR;
    const T tm1R = (t - T(1)) * iR;
    const T gxr = C.cp * gx + C.sp * gy, gyr = C.cp * gy - C.sp * gx;   // G in the lens frame
    const T Pd_th = P * (gxr * sthr + gyr * sthi);
    const T Pd_f = P * (gxr * J.fre + gyr * J.fim);
    const T ad = gxr * J.are + gyr * J.aim;
    const T d_xr = Pd_th * th_xr - ad * tm1R * R_xr;
    const T d_yr = Pd_th * th_yr - ad * tm1R * R_yr;
    const T d_q = Pd_th * th_q + Pd_f * C.f_q + ad * (C.tb_bq - tm1R * R_q - C.iopq);
    out[0] += ad * C.tb_sq;
    if (want_t) out[1] += P * (gxr * J.ure + gyr * J.uim) + ad * J.lbR;
    const T d_phi = d_xr * yr - d_yr * xr + (gy * J.ax - gx * J.ay);
    out[2] += d_q * C.qe1 - d_phi * C.pe2;
    out[3] += d_q * C.qe2 + d_phi * C.pe1;
    out[4] += -C.cp * d_xr + C.sp * d_yr;
    out[5] += -C.sp * d_xr - C.cp * d_yr;
}

template <typename T>
RTU_HD void epl_alpha_vjp(const EplC<T>& C, bool want_t, T x, T y, T gx, T gy, T& ax, T& ay, T* out) {
    EplJ<T> J;
    epl_eval(C, want_t, x, y, J);
    ax = J.ax;
    ay = J.ay;
    epl_vjp(C, J, want_t, gx, gy, out);
}

}  // namespace rtu
