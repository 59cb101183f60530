// k_gp.cuh -- the GP source on the uniform RTU grid (Sec. 2.1, Eq. 1-4) and
// its adjoint: mixed-radix (2, 3, 4) decimation-in-time line FFTs in shared
// memory, a few lines of one evaluation per CTA, over an n_src x n_src complex
// buffer that stays in L2 between the passes.
#pragma once
#include <cooperative_groups.h>
#include "rtu_internal.cuh"

namespace rtu {

constexpr int GP_NT = 512;
constexpr int GP_SMEM = 96 * 1024;   // bytes of dynamic shared memory for FFT chunks

template <typename T> struct Cx { T x, y; };
template <typename T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return Cx<T>{a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) { return Cx<T>{a.x - b.x, a.y - b.y}; }

// twiddle exp(-+2 pi i m / n) from the table (conjugate for the inverse)
template <typename T>
__device__ __forceinline__ Cx<T> twid(const Cx<T>* tw, int m, bool inv) {
    Cx<T> w = tw[m];
    if (inv) w.y = -w.y;
    return w;
}

// In-place DIT butterflies over `cnt` length-n sequences stored contiguously in
// shared memory, input already in digit-reversed order.
template <typename T>
__device__ void fft_seq_smem(Cx<T>* buf, int cnt, int n, const int* rad, int nrad, const Cx<T>* tw,
                             bool inv) {
    int L = 1;
    for (int s = 0; s < nrad; ++s) {
        const int r = rad[s];
        const int Ls = L * r;
        const int nb = n / r;
        const int step = n / Ls;
        for (int w = threadIdx.x; w < cnt * nb; w += blockDim.x) {
            const int row = w / nb, bi = w - row * nb;
            const int blk = bi / L, k = bi - blk * L;
            Cx<T>* p = buf + row * n + blk * Ls + k;
            if (r == 2) {
                Cx<T> y0 = p[0], y1 = cmul(p[L], twid(tw, k * step, inv));
                p[0] = cadd(y0, y1);
                p[L] = csub(y0, y1);
            } else if (r == 4) {
                Cx<T> y0 = p[0];
                Cx<T> y1 = cmul(p[L], twid(tw, k * step, inv));
                Cx<T> y2 = cmul(p[2 * L], twid(tw, 2 * k * step, inv));
                Cx<T> y3 = cmul(p[3 * L], twid(tw, 3 * k * step, inv));
                Cx<T> a0 = cadd(y0, y2), a1 = csub(y0, y2);
                Cx<T> b0 = cadd(y1, y3), b1 = csub(y1, y3);
                // -i (forward) / +i (inverse) times b1
                Cx<T> jb1 = inv ? Cx<T>{-b1.y, b1.x} : Cx<T>{b1.y, -b1.x};
                p[0] = cadd(a0, b0);
                p[L] = cadd(a1, jb1);
                p[2 * L] = csub(a0, b0);
                p[3 * L] = csub(a1, jb1);
            } else {  // r == 3
                Cx<T> y0 = p[0];
                Cx<T> y1 = cmul(p[L], twid(tw, k * step, inv));
                Cx<T> y2 = cmul(p[2 * L], twid(tw, 2 * k * step, inv));
                Cx<T> w3 = twid(tw, n / 3, inv);          // exp(-+2 pi i / 3)
                Cx<T> w32 = Cx<T>{w3.x, -w3.y};           // its square = its conjugate
                p[0] = cadd(y0, cadd(y1, y2));
                p[L] = cadd(y0, cadd(cmul(y1, w3), cmul(y2, w32)));
                p[2 * L] = cadd(y0, cadd(cmul(y1, w32), cmul(y2, w3)));
            }
        }
        __syncthreads();
        L = Ls;
    }
}

// 2-D FFT of a global n x n complex buffer in place (rows then columns), or
// one direction only (dir bit 1 = rows, bit 2 = columns).  `smem` holds a
// chunk; `tw` and `rev` are in shared memory.
template <typename T>
__device__ void fft2_pass(Cx<T>* g, int n, const int* rad, int nrad, const Cx<T>* tw, const int* rev,
                          Cx<T>* smem, int chunk, bool inv, bool cols) {
    for (int c0 = 0; c0 < n; c0 += chunk) {
        const int cnt = min(chunk, n - c0);
        // load with digit reversal: seq q position p <- element rev[p]
        for (int w = threadIdx.x; w < cnt * n; w += blockDim.x) {
            if (!cols) {
                const int q = w / n, p = w - q * n;
                smem[q * n + p] = g[(c0 + q) * n + rev[p]];
            } else {
                const int p = w / cnt, q = w - p * cnt;
                smem[q * n + p] = g[rev[p] * n + c0 + q];
            }
        }
        __syncthreads();
        fft_seq_smem<T>(smem, cnt, n, rad, nrad, tw, inv);
        for (int w = threadIdx.x; w < cnt * n; w += blockDim.x) {
            if (!cols) {
                const int q = w / n, p = w - q * n;
                g[(c0 + q) * n + p] = smem[q * n + p];
            } else {
                const int p = w / cnt, q = w - p * cnt;
                g[p * n + c0 + q] = smem[q * n + p];
            }
        }
        __syncthreads();
    }
}

template <typename T>
__device__ void fft2(Cx<T>* g, int n, const int* rad, int nrad, const Cx<T>* tw, const int* rev,
                     Cx<T>* smem, int chunk, bool inv) {
    fft2_pass<T>(g, n, rad, nrad, tw, rev, smem, chunk, inv, false);
    fft2_pass<T>(g, n, rad, nrad, tw, rev, smem, chunk, inv, true);
}

// numpy fftfreq(n)[i] in cycles per pixel, in the kernel's type (no FP64
// instruction in float mode)
template <typename T>
__device__ __forceinline__ T fftfreq(int i, int n) {
    return T(i < (n + 1) / 2 ? i : i - n) / T(n);
}

// sqrt(P(k)) and d sqrt(P)/d theta for the family (Eq. 4 and its stand-ins), in
// the type R (double in FP64 mode, float in FP32 mode)
template <typename R>
__device__ __forceinline__ R sqrtP_and_grad(int family, const R* ps, R k, R* g) {
    if (family == 0) {            // A k^-beta, zero mode removed
        if (k == R(0)) { g[0] = g[1] = R(0); return R(0); }
        const R A = ps[0], be = ps[1];
        const R lk = r_log(k);
        const R sp = r_sqrt(A) * r_exp(R(-0.5) * be * lk);
        g[0] = sp / (R(2) * A);
        g[1] = R(-0.5) * lk * sp;
        return sp;
    }
    if (family == 1) {            // A / (1 + (k/k0)^2)^2
        const R A = ps[0], k0 = ps[1];
        const R kk = k / k0;
        const R u = R(1) + kk * kk;
        const R sA = r_sqrt(A);
        const R sp = sA / u;
        g[0] = sp / (R(2) * A);
        g[1] = sA * R(2) * kk * kk / (k0 * u * u);
        return sp;
    }
    // Eq. 4: sigma^2 4 pi n (2n/zeta^2)^n (2n/zeta^2 + k^2)^-(n+1)
    const R sg = ps[0], nn = ps[1], ze = ps[2];
    const R a = R(2) * nn / (ze * ze);
    const R lak = r_log(a + k * k);
    const R logP = R(2) * r_log(sg) + r_log(R(4.0 * 3.14159265358979323846) * nn) + nn * r_log(a)
                   - (nn + R(1)) * lak;
    const R sp = r_exp(R(0.5) * logP);
    g[0] = sp / sg;
    g[1] = R(0.5) * sp * (R(1) / nn + r_log(a) + R(1) - lak - (nn + R(1)) * a / (nn * (a + k * k)));
    g[2] = R(0.5) * sp * (R(-2) * nn / ze + R(2) * (nn + R(1)) * a / (ze * (a + k * k)));
    return sp;
}

__device__ __forceinline__ int n_family(int family) { return family == 2 ? 3 : 2; }

// sqrt(P(k)) alone (the forward filter), with the parameter-only factors hoisted:
// c[0] = sqrt(A) (power law, Matern-like) or the log prefactor (Eq. 4)
template <typename R>
__device__ __forceinline__ R sqrtP_only(int family, const R* ps, const R* c, R k) {
    if (family == 0) return k == R(0) ? R(0) : c[0] * r_exp(R(-0.5) * ps[1] * r_log(k));
    if (family == 1) {
        const R kk = k / ps[1];
        return c[0] / (R(1) + kk * kk);
    }
    const R a = R(2) * ps[1] / (ps[2] * ps[2]);
    return r_exp(c[0] - R(0.5) * (ps[1] + R(1)) * r_log(a + k * k));
}

template <typename R>
__device__ __forceinline__ void sqrtP_consts(int family, const R* ps, R* c) {
    if (family == 0 || family == 1) {
        c[0] = r_sqrt(ps[0]);
    } else {
        const R sg = ps[0], nn = ps[1], ze = ps[2];
        const R a = R(2) * nn / (ze * ze);
        c[0] = R(0.5) * (R(2) * r_log(sg) + r_log(R(4.0 * 3.14159265358979323846) * nn) + nn * r_log(a));
    }
}

// ln(phi_sp(x) s0) without underflow, and sigma(x)/phi_sp(x)
template <typename T>
__device__ __forceinline__ T log_sp_s0(T x) {
    const T ls0 = T(-4.605170185988091);      // ln 0.01
    if (x < T(-30)) return x + ls0;
    T sp = (x > T(0) ? x : T(0)) + r_log1p(r_exp(-r_abs(x)));
    return r_log(sp) + ls0;
}
template <typename T>
__device__ __forceinline__ T sig_over_sp(T x) {
    if (x < T(-30)) return T(1);
    T e = r_exp(-r_abs(x));
    T sgm = x >= T(0) ? T(1) / (T(1) + e) : e / (T(1) + e);
    T sp = (x > T(0) ? x : T(0)) + r_log1p(e);
    return sgm / sp;
}

struct GPShared {
    int rad[MAX_RADIX];
};

template <typename T>
__device__ __forceinline__ void gp_setup(const EvalArgs& E, Cx<T>* tw_s, int* rev_s, int* rad_s) {
    const int n = E.n_src;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tw_s[i] = Cx<T>{(T)E.tw[2 * i], (T)E.tw[2 * i + 1]};
        rev_s[i] = E.digrev[i];
    }
    if (threadIdx.x < MAX_RADIX) rad_s[threadIdx.x] = E.rad[threadIdx.x];
    __syncthreads();
}

// S6 spread over many CTAs: the source's 2-D FFTs as passes of 1-D line FFTs
// (GP_LINES lines of one evaluation per CTA), computed in FP64-class arithmetic in
// both precisions (double-float for a float source).  Near f = 0 the softplus turns an absolute error of f into a relative
// error of s* amplified by 1/s0 = 100, and a float FFT's absolute error (~1e-7 of
// max |f|) reaches the gradients at their 1e-5 tolerance; one CTA per evaluation
// in double would leave the FP64 pipe of a single SM doing the whole transform.
//   pass 0: forward FFT of the rows of w (real) -> W
//   pass 1: forward FFT of the columns of W (kept, in the storage type, for the
//           adjoint's spectrum gradient), times sqrt(P(k)), inverse FFT of the columns
//   pass 2: inverse FFT of the rows; f = Re / N^2, s* = (phi_sp(f/s0) s0)^alpha
// W (complex double, row-major) stays in the workspace between the passes (L2).
constexpr int GP_LINES = 8;
constexpr int GP_LINE_NT = 256;
constexpr int GP_PASSES = 3;
constexpr int GP_CL = 8;              // CTAs of the GP adjoint's cluster kernel
// rows of per-CTA GP adjoint partials: one per line CTA, at least one per cluster CTA
// (rows a kernel does not write are zeroed by its first CTA)
__host__ __device__ inline int gp_part_rows(int n) { return max((n + GP_LINES - 1) / GP_LINES, GP_CL); }
constexpr int GP_PER_T = GP_LINES * 256 / GP_LINE_NT;   // line elements per thread, at most

// line q of the CTA's buffer from natural order into the digit-reversed order the
// DIT butterflies take (through registers: every thread reads, then writes)
// (called by all GP_LINE_NT threads of the CTA)
template <typename T>
__device__ __forceinline__ void lines_to_digit_reversed(Cx<T>* sm, int cnt, int n, const int* rev_s) {
    Cx<T> v[GP_PER_T];
#pragma unroll
    for (int k = 0; k < GP_PER_T; ++k) {
        const int i = threadIdx.x + k * GP_LINE_NT;
        if (i < cnt * n) {
            const int q = i / n, p = i - q * n;
            v[k] = sm[q * n + rev_s[p]];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GP_PER_T; ++k) {
        const int i = threadIdx.x + k * GP_LINE_NT;
        if (i < cnt * n) sm[i] = v[k];
    }
    __syncthreads();
}

// the arithmetic type of the source's transforms: double-float on the FP32 pipes for
// a float source (about 48 bits; the FP64 pipe is shared with the grid build's FP64
// set-up running beside it), double for a double source
template <typename TS> struct gp_src_type { typedef DF type; };
template <> struct gp_src_type<double> { typedef double type; };
__device__ __forceinline__ float gp_store(const DF& v, float) { return v.hi; }   // hi is the rounded value
__device__ __forceinline__ double gp_store(double v, double) { return v; }
__device__ __forceinline__ DF gp_sqrt(const DF& v) { return r_sqrt(v); }
__device__ __forceinline__ double gp_sqrt(double v) { return sqrt(v); }

template <typename TS>
__global__ void __launch_bounds__(GP_LINE_NT) k_gp_lines(const __grid_constant__ Batch B, int pass) {
    typedef typename gp_src_type<TS>::type T;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int n = E.n_src;
    __shared__ Cx<T> sm[GP_LINES * 256];
    __shared__ Cx<T> tw_s[256];
    __shared__ int rev_s[256];
    __shared__ int rad_s[MAX_RADIX];
    gp_setup<T>(E, tw_s, rev_s, rad_s);
    const bool cols = pass == 1;
    const int l0 = tile * GP_LINES, cnt = min(GP_LINES, n - l0);
    if (cnt <= 0) return;
    Cx<T>* W = reinterpret_cast<Cx<T>*>(E.cbufA);
    const TS* w = reinterpret_cast<const TS*>(E.latents);
    // load with digit reversal: line q position p <- element rev[p]
    for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
        if (!cols) {
            const int q = i / n, p = i - q * n;
            const int at = (l0 + q) * n + rev_s[p];
            sm[q * n + p] = pass == 0 ? Cx<T>{(T)w[at], T(0)} : W[at];
        } else {
            const int p = i / cnt, q = i - p * cnt;
            sm[q * n + p] = W[rev_s[p] * n + l0 + q];
        }
    }
    __syncthreads();
    fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, pass == 2);
    if (pass == 0) {
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int q = i / n, p = i - q * n;
            W[(l0 + q) * n + p] = sm[q * n + p];
        }
        return;
    }
    if (pass == 1) {
        // keep F(w) for the adjoint; times sqrt(P(k)) (Eq. 1): column l0 + q is kx,
        // row p is ky; then the inverse FFT of the same columns
        typedef typename real2_of<TS>::type C2;
        C2* Wk = reinterpret_cast<C2*>(E.cbufB);
        const int nf = n_family(E.family);
        T psv[4], pc[1];
        for (int q = 0; q < nf; ++q) psv[q] = T(E.ps[q]);
        sqrtP_consts<T>(E.family, psv, pc);
        const T kscale = T(2.0 * 3.14159265358979323846 / E.pitch);
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int p = i / cnt, q = i - p * cnt;
            const T fx = fftfreq<T>(l0 + q, n), fy = fftfreq<T>(p, n);
            const T k = kscale * gp_sqrt(fx * fx + fy * fy);
            const T sp = sqrtP_only<T>(E.family, psv, pc, k);
            const Cx<T> v = sm[q * n + p];
            C2 wv;
            wv.x = gp_store(v.x, TS(0));
            wv.y = gp_store(v.y, TS(0));
            Wk[p * n + l0 + q] = wv;
            sm[q * n + p] = Cx<T>{v.x * sp, v.y * sp};
        }
        __syncthreads();
        lines_to_digit_reversed<T>(sm, cnt, n, rev_s);
        fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, true);
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int p = i / cnt, q = i - p * cnt;
            W[p * n + l0 + q] = sm[q * n + p];
        }
        return;
    }
    // pass 2: the field and the source brightness (the map in the storage type: f is
    // already accurate, and the softplus of an accurately rounded argument is too)
    const int nf = n_family(E.family);
    const TS alpha = (TS)E.ps[nf];
    const T inv_n2 = T(1.0 / ((double)n * n));
    TS* fld = reinterpret_cast<TS*>(E.fld);
    TS* src = reinterpret_cast<TS*>(E.src);
    TS* so = reinterpret_cast<TS*>(E.source_out);
    for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
        const int q = i / n, p = i - q * n;
        const T f = sm[q * n + p].x * inv_n2;
        const TS fs = gp_store(f, TS(0));
        const TS sv = r_exp(alpha * log_sp_s0<TS>(gp_store(f * T(100.0), TS(0))));
        const int at = (l0 + q) * n + p;
        fld[at] = fs;
        src[at] = sv;
        if (so) so[at] = sv;
    }
}

// S9 (source part) as line passes over many CTAs, in the kernel's type: node
// gradients from the per-cell bilinear corner sums, back through the softplus /
// alpha map and the FFT filter (self-adjoint) to the latents;
// d log L / d sqrt(P_k) = Re(F(w)_k conj(G_k)) / N^2 to the spectrum parameters with
// F(w) kept by the forward; d s*/d alpha to alpha_src.  Per-CTA partial sums in
// gpart[tile][0..2] (spectrum) and [3] (alpha_src), summed by k_grad_final.
//   pass 0: G = g ds*/df row by row, forward FFT of the rows
//   pass 1: forward FFT of the columns, the spectrum sums, times sqrt(P(k)),
//           inverse FFT of the columns
//   pass 2: inverse FFT of the rows; d log L / d w = Re / N^2
template <typename T>
__global__ void __launch_bounds__(GP_LINE_NT) k_gp_adj_lines(const __grid_constant__ Batch B, int pass) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int n = E.n_src, nc = n - 1;
    __shared__ Cx<T> sm[GP_LINES * 256];
    __shared__ Cx<T> tw_s[256];
    __shared__ int rev_s[256];
    __shared__ int rad_s[MAX_RADIX];
    __shared__ double red[GP_LINE_NT / 32];
    gp_setup<T>(E, tw_s, rev_s, rad_s);
    const int l0 = tile * GP_LINES, cnt = min(GP_LINES, n - l0);
    if (cnt <= 0) return;
    Cx<T>* G = reinterpret_cast<Cx<T>*>(E.cbufA);
    const int nf = n_family(E.family);
    double* part = E.gpart + (size_t)tile * 4;
    if (pass == 0 && tile == 0) {
        const int ngl = (n + GP_LINES - 1) / GP_LINES;
        for (int i = ngl * 4 + threadIdx.x; i < gp_part_rows(n) * 4; i += blockDim.x) E.gpart[i] = 0.0;
    }
    if (pass == 0) {
        typedef typename real2_of<T>::type TP;
        const TP* cor = reinterpret_cast<const TP*>(E.corner);
        const T* fld = reinterpret_cast<const T*>(E.fld);
        const T* src = reinterpret_cast<const T*>(E.src);
        const T alpha = (T)E.ps[nf];
        T ga_t = T(0);
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int q = i / n, p = i - q * n;
            const int j = l0 + q, ii = rev_s[p];       // digit-reversed load of row j
            T g = T(0);
            if (ii < nc && j < nc) { const TP c = cor[(j * nc + ii) * 4 + 0]; g += c.x + c.y; }
            if (ii > 0 && j < nc) { const TP c = cor[(j * nc + ii - 1) * 4 + 1]; g += c.x + c.y; }
            if (ii < nc && j > 0) { const TP c = cor[((j - 1) * nc + ii) * 4 + 2]; g += c.x + c.y; }
            if (ii > 0 && j > 0) { const TP c = cor[((j - 1) * nc + ii - 1) * 4 + 3]; g += c.x + c.y; }
            const int at = j * n + ii;
            const T s = src[at];
            const T x = fld[at] / T(0.01);
            // d s / d f = alpha s (sigma(x)/phi_sp(x)) / s0
            const T dsdf = alpha * s * sig_over_sp<T>(x) / T(0.01);
            sm[q * n + p] = Cx<T>{g * dsdf, T(0)};
            if (s > T(0)) ga_t += g * s * log_sp_s0<T>(x);
        }
        const double ga = block_sum_t<GP_LINE_NT>(ga_t, red);
        if (threadIdx.x == 0) part[3] = ga;
        fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, false);
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int q = i / n, p = i - q * n;
            G[(l0 + q) * n + p] = sm[q * n + p];
        }
        return;
    }
    if (pass == 1) {
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int p = i / cnt, q = i - p * cnt;
            sm[q * n + p] = G[rev_s[p] * n + l0 + q];
        }
        __syncthreads();
        fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, false);
        typedef typename real2_of<T>::type C2;
        const C2* Wk = reinterpret_cast<const C2*>(E.cbufB);
        T psv[4];
        for (int q = 0; q < nf; ++q) psv[q] = (T)E.ps[q];
        const T kscale = (T)(2.0 * 3.14159265358979323846 / E.pitch);
        const T inv_n2s = T(1) / T(n * n);
        T gp[3] = {T(0), T(0), T(0)};
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int p = i / cnt, q = i - p * cnt;
            const T fx = fftfreq<T>(l0 + q, n), fy = fftfreq<T>(p, n);
            const T k = kscale * r_sqrt(fx * fx + fy * fy);
            T dsp[3] = {T(0), T(0), T(0)};
            const T sp = sqrtP_and_grad<T>(E.family, psv, k, dsp);
            const Cx<T> Gk = sm[q * n + p];
            const C2 W = Wk[p * n + l0 + q];
            const T d = (W.x * Gk.x + W.y * Gk.y) * inv_n2s;
            for (int c = 0; c < nf; ++c) gp[c] += d * dsp[c];
            sm[q * n + p] = Cx<T>{Gk.x * sp, Gk.y * sp};
        }
        for (int c = 0; c < 3; ++c) {
            const double v = block_sum_t<GP_LINE_NT>(gp[c], red);
            if (threadIdx.x == 0) part[c] = c < nf ? v : 0.0;
        }
        lines_to_digit_reversed<T>(sm, cnt, n, rev_s);
        fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, true);
        for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
            const int p = i / cnt, q = i - p * cnt;
            G[p * n + l0 + q] = sm[q * n + p];
        }
        return;
    }
    // pass 2
    for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
        const int q = i / n, p = i - q * n;
        sm[q * n + p] = G[(l0 + q) * n + rev_s[p]];
    }
    __syncthreads();
    fft_seq_smem<T>(sm, cnt, n, rad_s, E.nrad, tw_s, true);
    T* gl = reinterpret_cast<T*>(E.g_lat);
    const T inv_n2 = T(1) / T(n * n);
    for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
        const int q = i / n, p = i - q * n;
        gl[(l0 + q) * n + p] = sm[q * n + p].x * inv_n2;
    }
}

// S9 (source part) as one kernel per evaluation on a thread-block cluster of GP_CL
// CTAs: CTA r holds lines [r L, r L + L), L = n / GP_CL, and the transposes between
// the row and column passes read the other CTAs' shared memory (distributed shared
// memory) instead of a global buffer, with cluster barriers where the three line
// passes of k_gp_adj_lines had kernel boundaries.  The same arithmetic per line:
//   rows:    G = g ds*/df (node gradients from the corner sums), forward row FFTs  -> A
//   columns: forward column FFTs of A (remote), spectrum sums, times sqrt(P(k)),
//            digit-reversed into C, inverse column FFTs                            -> C
//   rows:    inverse row FFTs of C (remote); d log L / d w = Re / N^2
// Needs n % GP_CL == 0 and 3 L n complex values of shared memory (gp_cluster_ok).
constexpr int GP_CL_NT = 256;
constexpr size_t GP_CL_SMEM_MAX = 192 * 1024;
__host__ __device__ inline size_t gp_cluster_bytes(int n, int tb) { return (size_t)3 * (n / GP_CL) * n * 2 * tb; }
__host__ __device__ inline bool gp_cluster_ok(int n, int tb) {
    return n % GP_CL == 0 && n <= 256 && gp_cluster_bytes(n, tb) <= GP_CL_SMEM_MAX;
}
template <typename T>
__global__ void __cluster_dims__(GP_CL, 1, 1) __launch_bounds__(GP_CL_NT) k_gp_adj_cluster(const __grid_constant__ Batch B) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int rank = (int)cl.block_rank();
    const int n = E.n_src, nc = n - 1, L = n / GP_CL, l0 = rank * L;
    extern __shared__ __align__(16) unsigned char gp_smem[];
    Cx<T>* A = reinterpret_cast<Cx<T>*>(gp_smem);
    Cx<T>* Bf = A + (size_t)L * n;
    Cx<T>* C = Bf + (size_t)L * n;
    __shared__ Cx<T> tw_s[256];
    __shared__ int rev_s[256], inv_s[256];
    __shared__ int rad_s[MAX_RADIX];
    __shared__ double red[4][GP_CL_NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    gp_setup<T>(E, tw_s, rev_s, rad_s);
    for (int i = threadIdx.x; i < n; i += blockDim.x) inv_s[rev_s[i]] = i;
    const int nf = n_family(E.family);
    double* part = E.gpart + (size_t)rank * 4;
    if (rank == 0)
        for (int i = GP_CL * 4 + threadIdx.x; i < gp_part_rows(n) * 4; i += blockDim.x) E.gpart[i] = 0.0;
    // rows: node gradients (digit-reversed load of each row), then forward FFTs
    {
        typedef typename real2_of<T>::type TP;
        const TP* cor = reinterpret_cast<const TP*>(E.corner);
        const T* fld = reinterpret_cast<const T*>(E.fld);
        const T* src = reinterpret_cast<const T*>(E.src);
        const T alpha = (T)E.ps[nf];
        T ga_t = T(0);
        for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
            const int q = i / n, p = i - q * n;
            const int j = l0 + q, ii = rev_s[p];
            T g = T(0);
            if (ii < nc && j < nc) { const TP c = cor[(j * nc + ii) * 4 + 0]; g += c.x + c.y; }
            if (ii > 0 && j < nc) { const TP c = cor[(j * nc + ii - 1) * 4 + 1]; g += c.x + c.y; }
            if (ii < nc && j > 0) { const TP c = cor[((j - 1) * nc + ii) * 4 + 2]; g += c.x + c.y; }
            if (ii > 0 && j > 0) { const TP c = cor[((j - 1) * nc + ii - 1) * 4 + 3]; g += c.x + c.y; }
            const int at = j * n + ii;
            const T sv = src[at];
            const T x = fld[at] / T(0.01);
            // d s / d f = alpha s (sigma(x)/phi_sp(x)) / s0
            const T dsdf = alpha * sv * sig_over_sp<T>(x) / T(0.01);
            A[q * n + p] = Cx<T>{g * dsdf, T(0)};
            if (sv > T(0)) ga_t += g * sv * log_sp_s0<T>(x);
        }
        // the alpha_src partial: warp sums now, the CTA's sum with the spectrum's below
        const double w = warp_sum(ga_t);
        if (lane == 0) red[3][wid] = w;
        __syncthreads();                 // the rows are written before the butterflies read them
        fft_seq_smem<T>(A, L, n, rad_s, E.nrad, tw_s, false);
    }
    cl.sync();
    // columns: element (row r, column l0 + q) from the CTA holding row r
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int p = i / L, q = i - p * L;
        const int r = rev_s[p], owner = r / L;
        const Cx<T>* rA = cl.map_shared_rank(A, owner);
        Bf[q * n + p] = rA[(r - owner * L) * n + l0 + q];
    }
    __syncthreads();
    fft_seq_smem<T>(Bf, L, n, rad_s, E.nrad, tw_s, false);
    {
        typedef typename real2_of<T>::type C2;
        const C2* Wk = reinterpret_cast<const C2*>(E.cbufB);
        T psv[4];
        for (int q = 0; q < nf; ++q) psv[q] = (T)E.ps[q];
        const T kscale = (T)(2.0 * 3.14159265358979323846 / E.pitch);
        const T inv_n2s = T(1) / T(n * n);
        T gp[3] = {T(0), T(0), T(0)};
        for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
            const int p = i / L, q = i - p * L;
            const T fx = fftfreq<T>(l0 + q, n), fy = fftfreq<T>(p, n);
            const T k = kscale * r_sqrt(fx * fx + fy * fy);
            T dsp[3] = {T(0), T(0), T(0)};
            const T sp = sqrtP_and_grad<T>(E.family, psv, k, dsp);
            const Cx<T> Gk = Bf[q * n + p];
            const C2 W = Wk[p * n + l0 + q];
            const T d = (W.x * Gk.x + W.y * Gk.y) * inv_n2s;
            for (int c = 0; c < nf; ++c) gp[c] += d * dsp[c];
            C[q * n + inv_s[p]] = Cx<T>{Gk.x * sp, Gk.y * sp};    // digit-reversed for the inverse
        }
        for (int c = 0; c < 3; ++c) {
            const double w = warp_sum(gp[c]);
            if (lane == 0) red[c][wid] = w;
        }
    }
    __syncthreads();
    // the CTA's four partials: warps in order, one thread each
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < GP_CL_NT / 32; ++w) v += red[threadIdx.x][w];
        part[threadIdx.x] = threadIdx.x < 3 && threadIdx.x >= nf ? 0.0 : v;
    }
    fft_seq_smem<T>(C, L, n, rad_s, E.nrad, tw_s, true);
    cl.sync();
    // rows again: element (row l0 + q, column c) from the CTA holding column c
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int q = i / n, p = i - q * n;
        const int c = rev_s[p], owner = c / L;
        const Cx<T>* rC = cl.map_shared_rank(C, owner);
        A[q * n + p] = rC[(c - owner * L) * n + l0 + q];
    }
    // every CTA's remote reads are done before any CTA leaves or moves on
    cl.sync();
    fft_seq_smem<T>(A, L, n, rad_s, E.nrad, tw_s, true);
    T* gl = reinterpret_cast<T*>(E.g_lat);
    const T inv_n2 = T(1) / T(n * n);
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int q = i / n, p = i - q * n;
        gl[(l0 + q) * n + p] = A[q * n + p].x * inv_n2;
    }
}

}  // namespace rtu
