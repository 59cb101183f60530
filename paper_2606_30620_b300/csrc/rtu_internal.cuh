// rtu_internal.cuh -- per-evaluation launch descriptors and device helpers.
//
// Every kernel is launched once for a whole batch of evaluations.  The batch
// descriptor travels as a kernel parameter (no device allocation, graph
// capturable); blockIdx.x is mapped to (evaluation, tile) through a prefix
// array of per-evaluation tile counts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rtu_math.cuh"

namespace rtu {

constexpr int MAXB = 40;          // evaluations per launch (kernel-parameter budget)
constexpr int HB = 65536;         // level-1 histogram bins for order statistics
constexpr int SEL_CAP = 6144;     // candidate keys held in shared memory by the selector
constexpr int MAXM = 64;          // max Chebyshev nodes
constexpr int MAX_RADIX = 12;     // max FFT stages
constexpr int CTA_C = 256;        // centre-ray kernels: rays per CTA
constexpr int CTA_R = 128;        // render kernels: pixels per CTA (one thread each)
constexpr int PSF_T = 16;         // PSF kernels: 16 x 16 output tile per CTA
constexpr int NACC_FIX = 11;      // render-adjoint partials: 8 lens + mu_x, mu_y, sigma

// flag bits (mirror rtu.h)
constexpr int F_NONMONO = 1, F_SELECT = 2, F_TIMEOUT = 4;

struct EvalArgs {
    // static, from the system
    int n_img, s, n_src, psf_k;
    int profile, sub_kind, n_sub, family;
    int n_nodes, degree, n_mask, f64;
    int nrad, n_cta_c, n_cta_r, n_cta_p;
    int rad[MAX_RADIX];
    double pix, pitch, sigma, pad_;
    const void* data;
    const uint8_t* mask;
    const void* psf;
    const int* centre_idx;      // [n_mask] pixel index of each arc-mask pixel
    const double* tw;           // [2 n_src] exp(-2 pi i m / n_src)
    const int* digrev;          // [n_src] mixed-radix digit reversal
    // dynamic, from the rtu_eval binding
    const double* lens;
    const void* latents;
    const double* ps;
    const double* dlogL;
    double* stats;
    void* model_out;
    void* image_out;
    void* source_out;
    double* cdf_out;
    int* hist_out;
    void* g_lat;
    double* g_lens;
    double* g_ps;
    // workspace slot
    double* beta;      // [2][n_mask] traced centre rays (double)
    double* cpart;     // [n_cta_c][8] centre partial sums and ranges of beta
    double* cpart2;    // [n_cta_c][2] sum of squared deviations
    double* cadj;      // [n_cta_c][8 + 5 n_sub] centre-ray adjoint lens partials
    int* hist;         // [2][HB] level-1 histograms
    double* trd;       // transform, double (layout in tr_* helpers)
    float* trf;        // transform, float copy
    int* sel_idx;      // [2][2 MAXM] centre-ray index at each selected rank
    double* sel_val;   // [2][2 MAXM]
    double* tadj;      // transform adjoint block
    void* cbufA;       // complex real2 [n_src^2]
    void* cbufB;       // complex real2 [n_src^2]
    void* fld;         // real [n_src^2] GP field f
    void* src;         // real [n_src^2] source brightness s*
    void* img;         // real [n_img^2] unconvolved image
    void* resid;       // real [n_img^2] (d - m)/sigma^2
    void* gimg;        // real [n_img^2] d L / d image
    double* lpart;     // [n_cta_p][2]
    int* cell;         // [n_rays] RTU cell of every supersampled ray (-1 outside)
    int* ccount;       // [n_cells] ray counts, then [n_cells + 1] exclusive offsets
    int* cursor;       // [n_cells]
    void* rec;         // real4 [n_rays] counting-sorted (fx, fy, g, -) records
    double* corner;    // [n_cells][4] per-cell bilinear corner sums
    double* apart;     // [n_cta_r][nacc] render-adjoint partials
    int* flags;        // device flag word
};

struct Batch {
    int n;
    int tile0[MAXB + 1];
    EvalArgs e[MAXB];
};

// transform block layout (double and float copies share it):
//   [0] mu_x [1] mu_y [2] sigma [3] amin (0 = x, 1 = y) [4] n_knots
//   [8 ..)            knots x  (K = M+2)
//   [8+K ..)          knots y
//   [8+2K ..)         slopes x
//   [8+3K ..)         slopes y
//   [8+4K ..)         raw p'(u) x  (before the guard)  [8+5K ..) raw p' y
//   [8+6K ..)         raw knots x (before the guard)   [8+7K ..) raw knots y
//   [8+8K ..)         chebyshev coeffs x (D+1 <= MAXM) [8+8K+MAXM ..) y
//   [8+8K+2MAXM ..)   Q at nodes x, y (M each, MAXM stride)
constexpr int TR_HDR = 8;
__host__ __device__ constexpr int tr_size(int K) { return TR_HDR + 8 * K + 4 * MAXM; }

template <typename BatchT>
__device__ __forceinline__ int find_eval(const BatchT& B, int bid) {
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.tile0[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// deterministic block reduction of one double per thread (fixed tree order)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r += sh[i];
        sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

template <typename T> struct real2_of;
template <> struct real2_of<float> { typedef float2 type; };
template <> struct real2_of<double> { typedef double2 type; };
template <typename T> struct real4_of;
template <> struct real4_of<float> { typedef float4 type; };
template <> struct real4_of<double> { typedef double4_32a type; };

// ------------------------------------------------------------- lens trace
// Lens parameters as seen by a kernel: main lens and shear, then subhaloes.
struct LensP {
    double p[8];
    double sub[16][5];
};

template <typename T>
__device__ __forceinline__ T epl_tol() { return sizeof(T) == 4 ? T(1e-9) : T(1e-17); }

// Plain-value lens equation beta = theta - alpha(theta) (App. A).  In float
// mode, rays close to the EPL centre or to a subhalo's centre / scale radius
// are traced in double (the near-core FP64 island).
template <typename T>
__device__ __forceinline__ bool near_core(const LensP& L, int n_sub, int sub_kind, double x, double y) {
    double dx = x - L.p[4], dy = y - L.p[5];
    if (dx * dx + dy * dy < 0.0025 * L.p[0] * L.p[0] * 4.0) return true;  // |theta - c| < 0.1 theta_E
    if (sub_kind != 0) {
        for (int h = 0; h < n_sub; ++h) {
            double sx = x - L.sub[h][3], sy = y - L.sub[h][4];
            double r = sqrt(sx * sx + sy * sy) / L.sub[h][1];
            if (r < 1e-2 || fabs(r - 1.0) < 1e-2) return true;
        }
    }
    return false;
}

template <typename T>
__device__ __forceinline__ void trace_value_T(const LensP& L, int profile, int n_sub, int sub_kind,
                                              T x, T y, T& bx, T& by) {
    T gam = profile == 1 ? T(L.p[1]) : T(2);
    T ax, ay;
    epl_deflect<T>(x, y, T(L.p[0]), gam, T(L.p[2]), T(L.p[3]), T(L.p[4]), T(L.p[5]), ax, ay,
                   epl_tol<T>(), 200);
    ax += T(L.p[6]) * x + T(L.p[7]) * y;
    ay += T(L.p[7]) * x - T(L.p[6]) * y;
    for (int h = 0; h < n_sub; ++h) {
        T nx, ny;
        nfw_deflect<T>(x, y, T(L.sub[h][0]), T(L.sub[h][1]), T(L.sub[h][2]), T(L.sub[h][3]),
                       T(L.sub[h][4]), sub_kind, nx, ny);
        ax += nx;
        ay += ny;
    }
    bx = x - ax;
    by = y - ay;
}

template <typename T>
__device__ __forceinline__ void trace_value(const LensP& L, int profile, int n_sub, int sub_kind,
                                            double xd, double yd, T& bx, T& by) {
    if (sizeof(T) == 4 && near_core<T>(L, n_sub, sub_kind, xd, yd)) {
        double dbx, dby;
        trace_value_T<double>(L, profile, n_sub, sub_kind, xd, yd, dbx, dby);
        bx = T(dbx);
        by = T(dby);
    } else {
        trace_value_T<T>(L, profile, n_sub, sub_kind, T(xd), T(yd), bx, by);
    }
}

// Main lens with derivatives: returns beta and d beta / d(theta_E, gamma, e1, e2, x0, y0)
// (shear derivatives are analytic: d beta_x/d G1 = -x, d beta_x/d G2 = -y,
//  d beta_y/d G1 = +y, d beta_y/d G2 = -x).  Subhaloes contribute values only.
template <typename T>
__device__ __forceinline__ void trace_dual_T(const LensP& L, int profile, int n_sub, int sub_kind,
                                             T x, T y, Dual<T, 6>& bx, Dual<T, 6>& by) {
    typedef Dual<T, 6> D;
    D thE = D::seed(T(L.p[0]), 0);
    D gam = profile == 1 ? D::seed(T(L.p[1]), 1) : D(T(2));
    D e1 = D::seed(T(L.p[2]), 2), e2 = D::seed(T(L.p[3]), 3);
    D x0 = D::seed(T(L.p[4]), 4), y0 = D::seed(T(L.p[5]), 5);
    D ax, ay;
    epl_deflect<D>(D(x), D(y), thE, gam, e1, e2, x0, y0, ax, ay, epl_tol<T>(), 200);
    T sx = T(L.p[6]) * x + T(L.p[7]) * y;
    T sy = T(L.p[7]) * x - T(L.p[6]) * y;
    for (int h = 0; h < n_sub; ++h) {
        T nx, ny;
        nfw_deflect<T>(x, y, T(L.sub[h][0]), T(L.sub[h][1]), T(L.sub[h][2]), T(L.sub[h][3]),
                       T(L.sub[h][4]), sub_kind, nx, ny);
        sx += nx;
        sy += ny;
    }
    bx = T(0) - (ax + sx) + x;
    by = T(0) - (ay + sy) + y;
}

template <typename T>
__device__ __forceinline__ void trace_dual(const LensP& L, int profile, int n_sub, int sub_kind,
                                           double xd, double yd, Dual<T, 6>& bx, Dual<T, 6>& by) {
    if (sizeof(T) == 4 && near_core<T>(L, n_sub, sub_kind, xd, yd)) {
        Dual<double, 6> dbx, dby;
        trace_dual_T<double>(L, profile, n_sub, sub_kind, xd, yd, dbx, dby);
        bx = cast<Dual<T, 6>>(dbx);
        by = cast<Dual<T, 6>>(dby);
    } else {
        trace_dual_T<T>(L, profile, n_sub, sub_kind, T(xd), T(yd), bx, by);
    }
}

// Subhalo h with derivatives w.r.t. (kappa_s, r_s, tau, x_s, y_s): d alpha.
template <typename T>
__device__ __forceinline__ void sub_dual(const LensP& L, int h, int sub_kind, double xd, double yd,
                                         Dual<T, 5>& ax, Dual<T, 5>& ay) {
    typedef Dual<T, 5> D;
    D ks = D::seed(T(L.sub[h][0]), 0), rs = D::seed(T(L.sub[h][1]), 1);
    D tau = sub_kind == 2 ? D::seed(T(L.sub[h][2]), 2) : D(T(L.sub[h][2]));
    D xs = D::seed(T(L.sub[h][3]), 3), ys = D::seed(T(L.sub[h][4]), 4);
    nfw_deflect<D>(D(T(xd)), D(T(yd)), ks, rs, tau, xs, ys, sub_kind, ax, ay);
}

__device__ __forceinline__ void load_lens(LensP& L, const double* lens, int n_sub) {
    for (int i = 0; i < 8; ++i) L.p[i] = lens[i];
    for (int h = 0; h < n_sub; ++h)
        for (int k = 0; k < 5; ++k) L.sub[h][k] = lens[8 + 5 * h + k];
}

// pixel centre and sub-ray positions (Sec. 2.3)
__device__ __forceinline__ void ray_pos(int n_img, double pix, int s, int pixel, int sub,
                                        double& x, double& y) {
    int i = pixel % n_img, j = pixel / n_img;
    int a = sub % s, b = sub / s;
    double c = 0.5 * (n_img - 1);
    x = (i - c) * pix + ((a + 0.5) / s - 0.5) * pix;
    y = (j - c) * pix + ((b + 0.5) / s - 0.5) * pix;
}

}  // namespace rtu
