// rtu_internal.cuh -- per-evaluation launch descriptors and device helpers.
//
// Every kernel is launched once for a whole batch of evaluations.  The batch
// descriptor travels as a kernel parameter (no device allocation, graph
// capturable); blockIdx.x is mapped to (evaluation, tile) through a prefix
// array of per-evaluation tile counts.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rtu.h"
#include "rtu_math.cuh"
#include "rtu_df.cuh"

namespace rtu {

constexpr int MAXB = 40;          // evaluations per launch (kernel-parameter budget)
constexpr int HB = 65536;         // level-1 histogram bins for order statistics
constexpr int HROWS = HB / 32;    // rows of 32 level-1 bins (their counts are kept beside the bins)
constexpr int SEL_CAP = 6144;     // candidate keys held in shared memory by the selector
constexpr int MAXM = 64;          // max Chebyshev nodes
constexpr int MAX_RADIX = 12;     // max FFT stages
constexpr int CTA_C = 256;        // centre-ray kernels: rays per CTA
constexpr int CTA_R = 128;        // render kernels: pixels per CTA (one thread each)
constexpr int STG_SHIFT = 11;      // staged entry: low bits the ray within its render warp (< 32 * 64)
constexpr int STG_NEAR = 1 << 28;  // staged entry: a near-core ray (traced in FP64 by the float path)
constexpr int STG_DEFER = 1 << 29; // staged entry: a ray the near-edge pass decides (float path)
constexpr int NEAR_CTAS = 4;       // float render adjoint: CTAs per evaluation for the near-core rays (default)
constexpr int NEAR_CTAS_MAX = 16;  // the largest tuned value (the workspace holds its partial rows)
constexpr int ADJ_DIV = 4;         // render adjoint: CTAs per evaluation = rays / (ADJ_DIV CTA_R ADJ_RPT) (default)
constexpr int ADJ_RPT = 16;        // render adjoint: compacted rays per thread per chunk
constexpr int PSF_T = 32;         // PSF kernels: 32 x 32 output tile per CTA (4 outputs per thread)
constexpr int NACC_FIX = 11;      // render-adjoint partials: 8 lens + mu_x, mu_y, sigma

// flag bits (mirror rtu.h)
constexpr int F_NONMONO = 1, F_SELECT = 2, F_TIMEOUT = 4, F_RANGE = 8;

// Exact, order-independent accumulation of doubles as 128-bit fixed point: value
// v is v 2^80 rounded to an integer (a quantum of 2^-80), held as a low word (unsigned)
// and a high word (two's complement) at acc[0], acc[1].  Integer atomic additions are
// associative, so the sum has the same bits whatever the order of the additions; the
// low word's carry is detected from the value it returns.  |sum| must stay below 2^46:
// a term of |v| >= 2^40 raises F_RANGE instead of being added.
__device__ __forceinline__ void fix128_add(unsigned long long* acc, double v, int* flags) {
    if (v == 0.0) return;
    if (!(fabs(v) < 1099511627776.0)) {          // 2^40
        atomicOr(flags, F_RANGE);
        return;
    }
    const double s = v * 65536.0;                  // v 2^16: the high word's units
    const double h = floor(s);
    const long long hi = (long long)h;
    const unsigned long long lo = __double2ull_rn((s - h) * 18446744073709551616.0);   // (s - h) 2^64
    const unsigned long long old = atomicAdd(acc, lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    atomicAdd(acc + 1, (unsigned long long)hi + carry);
}
__device__ __forceinline__ double fix128_value(const unsigned long long* acc) {
    return (double)(long long)acc[1] * (1.0 / 65536.0) + (double)acc[0] * 0x1p-80;
}

struct EvalArgs {
    // static, from the system
    int n_img, s, n_src, psf_k;
    int profile, sub_kind, n_sub, family;
    int n_nodes, degree, n_mask, f64;
    int nrad, n_cta_c, n_cta_r, n_cta_p;
    int transform, n_light;
    int rad[MAX_RADIX];
    double pix, pitch, sigma, pad_;
    const void* data;
    const uint8_t* mask;
    const void* psf;
    const int* centre_idx;      // [n_mask] pixel index of each arc-mask pixel
    const double* psf_uv;       // [2 psf_k] psf[b][a] = u[b] v[a] (u then v) of a rank-1 PSF, or null
    const uint32_t* cwt;        // [n_mask] centre-ray weights (weighted grid) or null
    int wtot, pad3_;            // total centre-ray weight (n_mask when unweighted)
    const double* tw;           // [2 n_src] exp(-2 pi i m / n_src)
    const int* digrev;          // [n_src] mixed-radix digit reversal
    const double* cheb;         // Chebyshev tables (layout: cheb_* helpers)
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
    int* sel_hist_out;     // [2][HB] level-1 order-statistic histograms (nullable)
    double* centres_out;   // [2][n_mask] traced arc-mask centre positions (nullable)
    // workspace slot
    double* beta;      // [2][n_mask] traced centre rays (double)
    double* cpart;     // [n_cta_c][8] centre partial sums and ranges of beta
    double* cpart2;    // [n_cta_c][2] sum of squared deviations
    double* mom;       // [8] of the centre rays: mean x, y; min x, max x; min y, max y;
                       // sum of squared deviations x, y (each written once per call by the
                       // last CTA of k_trace_centres / k_centre_hist to finish)
    int* ccnt;         // [4] CTA-completion counters of those two kernels, of the
                       // likelihood kernel (whose last CTA finishes the forward) and of
                       // k_select_fit (whose last CTA tests the render tiles)
    int* cbin;         // [2][n_mask] level-1 histogram bin of each centre ray
    double* cadj;      // [n_cta_c + 2][8 + 5 n_sub] centre-ray adjoint lens partials; the last
                       // two rows the selected-rank terms of each axis
    double* jsel;      // [2][2 MAXM][8 + 5 n_sub] d beta_a / d lens of each selected-rank ray
    int* hist;         // [2][HB] level-1 histograms, then [2][HB/32] their sums over rows of 32 bins
    double* trd;       // transform, double (layout in tr_* helpers)
    float* trf;        // transform, float copy
    int* sel_idx;      // [2][2 MAXM] centre-ray index at each selected rank
    double* tadj;      // transform adjoint block
    void* cbufA;       // complex real2 [n_src^2]
    void* cbufB;       // complex real2 [n_src^2]: F(w), kept by the forward for the adjoint
    double* gpart;     // [GP line CTAs][4] spectrum (0..2) and alpha_src (3) gradient partials
    void* fld;         // real [n_src^2] GP field f
    void* src;         // real [n_src^2] source brightness s*
    void* img;         // real [n_img^2] unconvolved image
    void* resid;       // real [n_img^2] (d - m)/sigma^2
    void* gimg;        // real [n_img^2] d L / d image
    double* lpart;     // [n_cta_p][2]
    int* cell;         // staged in-grid rays: render warp u owns [u*32*s^2, (u+1)*32*s^2), entries
                       // (lane*s^2 + q) | (cell + 1) << STG_SHIFT in append order; cell + 1 = 0
                       // while a deferred ray is undecided, and after it ended outside;
                       // STG_NEAR set on the near-core rays of the float path
    int* ccount;       // [n_cells] ray counts, then [n_cells + 1] exclusive offsets
    int* cursor;       // [n_cells] the compaction's rank cursors (zeroed with the counts)
    int* elist;        // [n_rays] staging positions of the deferred rays (float mode)
    void* rec;         // real4 [n_rays] counting-sorted (fx, fy, g, -) records
    void* corner;      // real2 [n_cells][4] per-cell bilinear corner sums (float: hi + lo pairs)
    double* apart;     // [nacc][n_row_adj] render-adjoint partials (column-major)
    int* flags;        // device flag word
    unsigned long long* gmax;  // the largest |d L / d image| (bits of a non-negative float in the low
                               // word, or of a double): zeroed by k_zero and k_grad_final, raised
                               // by the PSF adjoint, read by the cell gather
    void* lensk;       // LensK<T> then LensK<double> of the evaluation
    int* ecount;       // number of deferred near-edge rays (float mode)
    unsigned long long* pdef;  // [n_img^2] bit q: sub-ray q deferred to the double pass (float mode)
    int* pcnt;         // [n_img^2] deferred sub-rays of the pixel still to finish (float mode)
    float* rval;       // [n_rays] values of deferred rays (float mode)
    int* cta_cnt;      // [n_cta_r] in-grid rays per render CTA (the N_IN_GRID statistic)
    unsigned char* tcull;  // [n_cta_r] 1: no ray of the render tile can reach the grid
    int* useg;         // [n_cta_r * CTA_R/32 + 1] staged rays per render warp; the total at the end
    int* kray;         // [n_rays] the adjoint's rays (staged rays in render-warp order): ray id, or -1
    int* kcell;        // [n_rays] their cells; -2 - cell for a near-core ray of the float path
    int* krank;        // [n_rays] their ranks inside their cells (the counting sort's slot = offset + rank)
    int* nseg;         // [n_cta_r * CTA_R/32 + 1] near-core staged rays per render warp; the total at the end
    int* nlist;        // [n_rays] adjoint positions of the near-core rays, in adjoint order
    void* gbuf;        // real2 [n_rays] d logL / d beta of each adjoint ray (subhalo pass)
    const double* light;   // [6 n_light] MGE lens light (A, sigma, q, phi, x_n, y_n)
    double* g_light;       // [6 n_light] adjoint out
    double* lpartl;        // [light CTAs][6 n_light] per-CTA lens-light moment sums
    int n_cta_adj;     // CTAs of the render adjoint (grid-stride over the compacted rays)
    int n_row_adj;     // rows of apart: n_cta_adj, plus n_near for the float path's near-core pass
    int n_near;        // CTAs per evaluation of the float path's near-core adjoint pass (tunable)
    int n_edge;        // CTAs per evaluation of the near-edge double pass (tunable)
    // the unsmoothed eCDF transform (App. C, first paragraph), per axis a at a * n_mask
    double* lkey;      // [2][n_mask] sorted centre-ray positions
    int* lidx;         // [2][n_mask] the centre ray at each rank
    int* lrank;        // [2][n_mask] the rank of each centre ray
    float* lkf;        // [2][n_mask] float2 (hi, lo) of lkey
    unsigned long long* gk;  // [2][n_mask] d logL / d (sorted position), adjoint: (low, high) words of
                             // a 128-bit fixed-point sum (fix128_add)
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
//   the unsmoothed eCDF transform keeps mu = 0, sigma = 1 and uses only the end
//   knots and end slopes, plus [8+6K + a] bin origin and [8+6K+2 + a] bin scale
//   of the level-1 histogram per axis a
constexpr int TR_HDR = 8;
__host__ __device__ constexpr int tr_size(int K) { return TR_HDR + 8 * K + 4 * MAXM; }

// Chebyshev tables of a system (M nodes, degree D, K = M + 2 knot points
// t = -1, t_1..t_M, +1), computed on the host at creation:
//   u[M]             the nodes u_j = (1 - cos((2j-1) pi / (2M))) / 2
//   V[K][D+1]        T_k(t) at the knot points
//   dV[K][D+1]       dp/du per coefficient: 2 T_k'(t)
//   C[D+1][M]        interpolating coefficients c = C Q  (2/M T_k(t_j), halved for k = 0)
__host__ __device__ constexpr int cheb_u(int, int) { return 0; }
__host__ __device__ constexpr int cheb_V(int M, int) { return M; }
__host__ __device__ constexpr int cheb_dV(int M, int D) { return M + (M + 2) * (D + 1); }
__host__ __device__ constexpr int cheb_C(int M, int D) { return M + 2 * (M + 2) * (D + 1); }
__host__ __device__ constexpr int cheb_size(int M, int D) { return M + 2 * (M + 2) * (D + 1) + (D + 1) * M; }

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

// Warp sum of one value per lane with a fixed shuffle tree, returned in lane 0
// as double.  Float lanes use compensated summation (TwoSum at each level,
// Knuth 1969), so the result carries about twice the float precision without
// FP64 arithmetic in the tree; double lanes add in double.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// compensated float pair (hi + lo) and its exact-error addition
struct F2 { float hi, lo; };
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    float s, e;
    two_sum_f(a.hi, b.hi, s, e);
    return F2{s, a.lo + b.lo + e};
}
__device__ __forceinline__ F2 f2_add(F2 a, float b) {
    float s, e;
    two_sum_f(a.hi, b, s, e);
    return F2{s, a.lo + e};
}
// the warp sum as a compensated pair (valid in lane 0); no FP64 arithmetic
__device__ __forceinline__ F2 warp_sum2(float v) {
    F2 a{v, 0.0f};
    for (int o = 16; o > 0; o >>= 1) {
        const F2 b{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
        a = f2_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double warp_sum(float v) {
    const F2 a = warp_sum2(v);
    return (double)a.hi + (double)a.lo;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// deterministic block reduction of one value per thread in its own type: a
// (compensated, for float) warp tree, then warps in order in double
template <int NT, typename T>
__device__ __forceinline__ double block_sum_t(T v, double* sh) {
    const double w = warp_sum(v);
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[wid] = w;
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

// One warp: the sum of a[t * stride] over t < rows, lanes striding over t, then a
// fixed shuffle tree; every lane gets lane 0's result (the same bits on every call).
__device__ __forceinline__ double warp_rows_sum(const double* a, int rows, size_t stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int t = lane; t < rows; t += 32) s += a[(size_t)t * stride];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return __shfl_sync(0xffffffffu, s, 0);
}

template <typename T> struct real2_of;
template <> struct real2_of<float> { typedef float2 type; };
template <> struct real2_of<double> { typedef double2 type; };

// running sums kept as (hi, lo) pairs of the kernel's type: compensated for
// float (no FP64 instruction), plain (lo = 0) for double
__device__ __forceinline__ void pair_add(float2& a, float b) {
    float s, e;
    two_sum_f(a.x, b, s, e);
    a.x = s;
    a.y += e;
}
__device__ __forceinline__ void pair_add(float2& a, float2 b) {
    float s, e;
    two_sum_f(a.x, b.x, s, e);
    a.x = s;
    a.y += b.y + e;
}
__device__ __forceinline__ void pair_add(double2& a, double b) { a.x += b; }
__device__ __forceinline__ void pair_add(double2& a, double2 b) { a.x += b.x + b.y; }
__device__ __forceinline__ float2 warp_pair_sum(float v) {
    const F2 a = warp_sum2(v);
    return make_float2(a.hi, a.lo);
}
__device__ __forceinline__ double2 warp_pair_sum(double v) { return make_double2(warp_sum(v), 0.0); }
// the warp sum (compensated pair for float) as a double, formed in lane 0 only (the
// other lanes get 0): the FP64 conversion is not repeated on every lane
template <typename T>
__device__ __forceinline__ double warp_sum_lane0(T v) {
    const auto p = warp_pair_sum(v);
    return (threadIdx.x & 31) == 0 ? (double)p.x + (double)p.y : 0.0;
}
template <typename T> struct real4_of;
template <> struct real4_of<float> { typedef float4 type; };
template <> struct real4_of<double> { typedef double4_32a type; };

// raise the evaluation's largest |d L / d image| (E.gmax) by this thread's value: a
// maximum, so the result does not depend on the order of the atomics (one per warp)
template <typename T>
__device__ __forceinline__ void note_gmax(const EvalArgs& E, T v) {
    v = v < T(0) ? -v : v;
    for (int o = 16; o > 0; o >>= 1) {
        const T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v > T(0)) {
        if (sizeof(T) == 4) atomicMax(reinterpret_cast<unsigned int*>(E.gmax), __float_as_uint((float)v));
        else atomicMax(E.gmax, (unsigned long long)__double_as_longlong((double)v));
    }
}

// ------------------------------------------------------------- lens trace
// Lens parameters as a kernel sees them: the EPL's per-system constants, the
// shear, the subhaloes, in the kernel's real type.  Built once per evaluation
// (k_zero) into the workspace and copied to shared memory by every CTA.
constexpr int MAX_SUB = 16;

template <typename T>
struct LensK {
    EplC<T> C;
    T g1, g2, rc2;           // shear; squared radius of the near-core FP64 island
    T sub[MAX_SUB][5];       // kappa_s, r_s, tau, x_s, y_s
    int nsub, kind, epl;
    int nsplit;              // double-float block: the first series power summed in float
};

template <typename T>
__device__ __forceinline__ T epl_tol() { return sizeof(T) == 4 ? T(2e-8) : T(1e-16); }

template <typename T>
__device__ inline void lens_rest(LensK<T>& K, const double* lens, int profile, int sub_kind, int n_sub) {
    K.g1 = (T)lens[6];
    K.g2 = (T)lens[7];
    K.rc2 = (T)(1e-4 * lens[0] * lens[0]);          // |theta - centre| < 0.01 theta_E
    K.nsub = sub_kind ? n_sub : 0;
    K.kind = sub_kind;
    K.epl = profile == 1;
    for (int h = 0; h < K.nsub; ++h)
        for (int k = 0; k < 5; ++k) K.sub[h][k] = (T)lens[8 + 5 * h + k];
}

// The three lens blocks of an evaluation (double, float and the double-float copy of
// the double one), built by one CTA of at least 160 threads.  On this part FP64
// divides, roots and logarithms are dependent chains of hundreds to thousands of
// cycles, so the work is spread so that no thread runs more than one such chain:
//   1. warps 0-2: the series coefficients, term n by thread n - 1 (the products
//      A_n = c_1 ... c_n and the sums D_n by warp scans, the warps synchronised by
//      a named barrier), written in all three types, and the stopping index of each
//      precision (1e-16 for double, 2e-8 for float: a third of the type's unit
//      roundoff or less, as |c_n| <= f <= 1/4) and the first power the double-float
//      evaluation sums in float (|A_n| <= 1e-9); meanwhile lane 0 of warps 3-5
//      computes one of the three independent parts of the lens-only scalars in
//      double (one chain per warp: lanes of one warp would run them one after the
//      other); every thread involved forms c = |(e1, e2)| (= f) itself;
//   2. one thread per scalar writes it in the three types (the float and
//      double-float values are the double one rounded, as a float build of the same
//      expressions gives), and three threads the shear, core radius and subhaloes.
__device__ inline void lens_setup_par(LensK<double>* Kd, LensK<float>* Kf, LensK<DF>* Kx, const double* lens,
                                      int profile, int sub_kind, int n_sub) {
    static_assert(offsetof(EplC<double>, ic) == (EPL_NSCAL - 1) * sizeof(double), "EplC scalars are contiguous");
    static_assert(offsetof(EplC<float>, ic) == (EPL_NSCAL - 1) * sizeof(float), "EplC scalars are contiguous");
    static_assert(offsetof(EplC<DF>, ic) == (EPL_NSCAL - 1) * sizeof(DF), "EplC scalars are contiguous");
    __shared__ double wA[3], wD[3];
    __shared__ EplC<double> sC;        // the double scalars (leading members only)
    __shared__ int nt_sh[3];
    const int tid = threadIdx.x;
    const bool epl = profile == 1;
    if (tid >= 96 && tid < 192 && (tid & 31) == 0) {
        const double p[6] = {lens[0], lens[1], lens[2], lens[3], lens[4], lens[5]};
        const double cc = sqrt(fmax(p[2] * p[2] + p[3] * p[3], 1e-30));
        epl_scalars_part(sC, p, epl, cc, (tid >> 5) - 3);
    } else if (tid < 96) {
        const int lane = tid & 31, w = tid >> 5, n = tid + 1;
        if (tid == 0) { nt_sh[0] = EPL_MAXT; nt_sh[1] = EPL_MAXT; nt_sh[2] = EPL_MAXT; }   // before the named barrier
        // f = (1 - q)/(1 + q) with q = (1 - c)/(1 + c) is c itself
        const double f = sqrt(fmax(lens[2] * lens[2] + lens[3] * lens[3], 1e-30));
        const double t = (epl ? lens[1] : 2.0) - 1.0;
        const double r1 = 1.0 / (2.0 * n - 2.0 + t), r2 = 1.0 / (2.0 * n + 2.0 - t);
        const double g = -(2.0 * n - 2.0 + t) * r2;
        const double c = f * g;
        const double dl = r1 + r2;
        // inclusive warp scans: A = product of c, D = sum of dl
        double A = c, D = dl;
        for (int o = 1; o < 32; o <<= 1) {
            const double a2 = __shfl_up_sync(0xffffffffu, A, o), d2 = __shfl_up_sync(0xffffffffu, D, o);
            if (lane >= o) { A *= a2; D += d2; }
        }
        if (lane == 31) { wA[w] = A; wD[w] = D; }
        asm volatile("bar.sync 1, 96;" ::: "memory");
        for (int v = 0; v < w; ++v) { A *= wA[v]; D += wD[v]; }
        double Ap = __shfl_up_sync(0xffffffffu, A, 1);          // A_{n-1}
        if (lane == 0) Ap = w == 0 ? 1.0 : wA[0] * (w == 2 ? wA[1] : 1.0);
        epl_term(Kd->C.term[n], Ap, c, D);
        epl_term(Kf->C.term[n], Ap, c, D);
        epl_term(Kx->C.term[n], Ap, c, D);
        if (tid == 0) { epl_term0(Kd->C.term[0]); epl_term0(Kf->C.term[0]); epl_term0(Kx->C.term[0]); }
        const double An = fabs(Ap * c);
        if (An <= 1e-16) atomicMin(&nt_sh[0], n);
        if (An <= 2e-8) atomicMin(&nt_sh[1], n);
        if (An <= 1e-9) atomicMin(&nt_sh[2], n);
    }
    __syncthreads();
    if (tid < EPL_NSCAL) {
        const double v = reinterpret_cast<const double*>(&sC)[tid];
        reinterpret_cast<double*>(&Kd->C)[tid] = v;
        reinterpret_cast<float*>(&Kf->C)[tid] = (float)v;
        reinterpret_cast<DF*>(&Kx->C)[tid] = DF(v);
    } else if (tid == 32) {
        Kd->C.nterm = nt_sh[0];
        Kx->C.nterm = nt_sh[0];            // the double-float copy sums as many terms as double,
        Kx->nsplit = nt_sh[2];             // those from |A_n| <= 1e-9 on in float
        Kf->C.nterm = nt_sh[1];
        Kd->nsplit = 1 << 30;              // (no float tail)
        Kf->nsplit = 1 << 30;
        lens_rest(*Kd, lens, profile, sub_kind, n_sub);
    } else if (tid == 64) {
        lens_rest(*Kf, lens, profile, sub_kind, n_sub);
    } else if (tid == 96) {
        // the double-float block serves the lens without subhaloes only
        Kx->g1 = DF(lens[6]);
        Kx->g2 = DF(lens[7]);
        Kx->rc2 = DF(1e-4 * lens[0] * lens[0]);
        Kx->nsub = 0; Kx->kind = sub_kind; Kx->epl = epl;
    }
}

// A bound on the subhaloes' total deflection, for every ray position: a subhalo deflects
// by 4 kappa_s r_s g(x)/x, x = r/r_s (App. A), with g the NFW projected-mass function
// h(x) = ln(x/2) + F(x), or the truncated one, which lies below h for every tau (the
// truncated density is the NFW one times tau^2/(tau^2 + x^2) <= 1, so it encloses less
// projected mass).  h is increasing and sup h(x)/x = 0.3105 (at x = 1.32; h(x)/x -> 0
// at both ends); with 0.32 taken, |alpha_h| <= 1.28 kappa_s r_s.
constexpr double SUB_ALPHA_PER_KR = 1.28;
template <typename T>
__device__ __forceinline__ T sub_alpha_bound(const LensK<T>& K) {
    T b = T(0);
    for (int h = 0; h < K.nsub; ++h) b += r_abs(K.sub[h][0]) * r_abs(K.sub[h][1]);
    return b * T(SUB_ALPHA_PER_KR) * T(1.001);
}

// rays near the EPL centre or a subhalo's centre / scale radius take the FP64 island
template <typename T>
__device__ __forceinline__ bool lens_near_core(const LensK<T>& K, T x, T y) {
    const T dx = x - K.C.x0, dy = y - K.C.y0;
    if (dx * dx + dy * dy < K.rc2) return true;
    for (int h = 0; h < K.nsub; ++h) {
        const T sx = x - K.sub[h][3], sy = y - K.sub[h][4];
        const T r = r_sqrt(sx * sx + sy * sy) / K.sub[h][1];
        if (r < T(1e-2) || r_abs(r - T(1)) < T(1e-2)) return true;
    }
    return false;
}

// lens equation beta = theta - alpha(theta) (App. A): EPL + shear + subhaloes
template <typename T>
__device__ __forceinline__ void lens_beta(const LensK<T>& K, T x, T y, T& bx, T& by) {
    T ax, ay;
    epl_alpha(K.C, x, y, ax, ay);
    ax += K.g1 * x + K.g2 * y;
    ay += K.g2 * x - K.g1 * y;
    for (int h = 0; h < K.nsub; ++h) {
        T nx, ny;
        nfw_deflect<T>(x, y, K.sub[h][0], K.sub[h][1], K.sub[h][2], K.sub[h][3], K.sub[h][4], K.kind, nx, ny);
        ax += nx;
        ay += ny;
    }
    bx = x - ax;
    by = y - ay;
}

// the lens equation without subhaloes (EPL + shear), for scalar types without
// the subhalo profiles' special functions
template <typename T>
__device__ __forceinline__ void lens_beta_smooth(const LensK<T>& K, T x, T y, T& bx, T& by) {
    T ax, ay;
    epl_alpha(K.C, x, y, ax, ay, K.nsplit);
    ax += K.g1 * x + K.g2 * y;
    ay += K.g2 * x - K.g1 * y;
    bx = x - ax;
    by = y - ay;
}

// the same, keeping the EPL intermediates for a later vector-Jacobian product
template <typename T>
__device__ __forceinline__ void lens_beta_eval(const LensK<T>& K, T x, T y, EplJ<T>& J, T& bx, T& by) {
    epl_eval(K.C, K.epl != 0, x, y, J);
    T ax = J.ax + K.g1 * x + K.g2 * y;
    T ay = J.ay + K.g2 * x - K.g1 * y;
    for (int h = 0; h < K.nsub; ++h) {
        T nx, ny;
        nfw_deflect<T>(x, y, K.sub[h][0], K.sub[h][1], K.sub[h][2], K.sub[h][3], K.sub[h][4], K.kind, nx, ny);
        ax += nx;
        ay += ny;
    }
    bx = x - ax;
    by = y - ay;
}

// the same without subhaloes (EPL + shear), for scalar types without the subhalo
// profiles' special functions
template <typename T>
__device__ __forceinline__ void lens_beta_eval_smooth(const LensK<T>& K, T x, T y, EplJ<T>& J, T& bx, T& by) {
    epl_eval(K.C, K.epl != 0, x, y, J);
    bx = x - (J.ax + K.g1 * x + K.g2 * y);
    by = y - (J.ay + K.g2 * x - K.g1 * y);
}

// out[0..7] += dL/d(theta_E, gamma, e1, e2, x0, y0, Gamma1, Gamma2) given dL/dbeta = (gbx, gby)
template <typename T>
__device__ __forceinline__ void lens_beta_vjp(const LensK<T>& K, const EplJ<T>& J, T x, T y, T gbx, T gby,
                                              T* out) {
    epl_vjp(K.C, J, K.epl != 0, -gbx, -gby, out);
    out[6] += -gbx * x + gby * y;      // d beta / d Gamma1 = (-x, +y)
    out[7] += -gbx * y - gby * x;      // d beta / d Gamma2 = (-y, -x)
}

// subhalo h: out[0..4] += dL/d(kappa_s, r_s, tau, x_s, y_s) given dL/dbeta.  The
// deflection is A (dx, dy) with A = 4 kappa_s r_s^2 g(u, tau) / r^2, u = r / r_s, so
// every partial follows from g and its two partials in (u, tau), taken with
// forward-mode duals: with P = G . (dx, dy), d/dkappa_s = (A / kappa_s) P,
// d/dr_s = 4 kappa_s (2 r_s g - r g_u) / r^2 P, d/dtau = 4 kappa_s r_s^2 g_tau / r^2 P,
// d/dx_s = -A_r (dx / r) P - A G_x (and y alike), A_r = 4 kappa_s (r_s r g_u - 2 r_s^2 g) / r^3
// (r^2 is clamped at 1e-20 as in the deflection, with no position derivative there).
template <typename T>
__device__ __forceinline__ void sub_vjp(const LensK<T>& K, int h, T x, T y, T gbx, T gby, T* out) {
    typedef Dual<T, 2> D;
    const T ks = K.sub[h][0], rs = K.sub[h][1];
    const T dx = x - K.sub[h][3], dy = y - K.sub[h][4];
    const T d2 = dx * dx + dy * dy;
    const bool clamped = d2 < T(1e-20);
    const T r = r_sqrt(clamped ? T(1e-20) : d2);
    const D g = nfw_g<D>(D::seed(r / rs, 0), K.kind == 2 ? D::seed(K.sub[h][2], 1) : D(K.sub[h][2]), K.kind);
    const T ir2 = T(1) / (r * r);
    const T f = T(4) * ks * ir2;                    // 4 kappa_s / r^2
    const T A = f * rs * rs * g.v;
    const T P = gbx * dx + gby * dy;
    out[0] -= T(4) * rs * rs * g.v * ir2 * P;
    out[1] -= f * (T(2) * rs * g.v - r * g.d[0]) * P;
    out[2] -= f * rs * rs * g.d[1] * P;
    const T Ar = clamped ? T(0) : f * (rs * r * g.d[0] - T(2) * rs * rs * g.v) / r;
    out[3] -= -Ar * (dx / r) * P - A * gbx;
    out[4] -= -Ar * (dy / r) * P - A * gby;
}

// the evaluation's lens blocks: LensK<double> first, then LensK<float>, then the
// double-float copy of the double block (written once per call by the lens set-up)
constexpr size_t LENSK_D_BYTES = (sizeof(LensK<double>) + 255) / 256 * 256;
constexpr size_t LENSK_DF_AT = LENSK_D_BYTES + (sizeof(LensK<float>) + 255) / 256 * 256;
constexpr size_t LENSK_BYTES = LENSK_DF_AT + (sizeof(LensK<DF>) + 255) / 256 * 256;
__host__ __device__ inline const void* lensk_df_src(const void* base) {
    return static_cast<const char*>(base) + LENSK_DF_AT;
}

// copy a lens block from global memory into shared memory (all threads)
template <typename T>
__device__ __forceinline__ void load_lensk(LensK<T>& dst, const void* src) {
    const int n = (int)(sizeof(LensK<T>) / 4);
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

template <typename T>
__device__ __forceinline__ const void* lensk_src(const void* base) {
    return sizeof(T) == 8 ? base : static_cast<const char*>(base) + LENSK_D_BYTES;
}

// ------------------------------------------------------------ MGE lens light
// Per component: A/(2 pi), 1/(2 sigma^2), q, 1/q, cos phi, sin phi, x_n, y_n, 1/A,
// 1/sigma in the kernel's type (App. A.3; rho^2 = q x'^2 + y'^2/q about (x_n, y_n),
// rotated by phi).
constexpr int MAX_LIGHT = RTU_MAX_LIGHT;
template <typename T>
struct LightK {
    // per component: amplitude A/(2 pi), centre, and the exponent
    // E = (q x'^2 + y'^2/q)/(2 sigma^2) as a quadratic form a dx^2 + b dx dy + c dy^2 in
    // the offsets (dx, dy) from the centre -- natural (e) and times log2(e) (e2)
    T amp[MAX_LIGHT], xn[MAX_LIGHT], yn[MAX_LIGHT];
    T ea[MAX_LIGHT], eb[MAX_LIGHT], ec[MAX_LIGHT];
    T e2a[MAX_LIGHT], e2b[MAX_LIGHT], e2c[MAX_LIGHT];
    int n;
};

template <typename T>
__device__ __forceinline__ void light_setup(LightK<T>& L, const double* light, int n) {
    if (threadIdx.x == 0) L.n = light ? n : 0;
    if (light && (int)threadIdx.x < n) {
        const int k = threadIdx.x;
        const double* p = light + 6 * k;
        const double c1 = 0.5 / (p[1] * p[1]), q = p[2], cs = cos(p[3]), sn = sin(p[3]);
        // x' = cs dx + sn dy, y' = cs dy - sn dx
        const double a = c1 * (q * cs * cs + sn * sn / q);
        const double b = c1 * 2.0 * cs * sn * (q - 1.0 / q);
        const double c = c1 * (q * sn * sn + cs * cs / q);
        const double l2e = 1.4426950408889634;      // log2(e): exp(-E) = 2^(-E log2 e)
        L.amp[k] = (T)(p[0] / (2.0 * 3.14159265358979323846));
        L.xn[k] = (T)p[4];
        L.yn[k] = (T)p[5];
        L.ea[k] = (T)a; L.eb[k] = (T)b; L.ec[k] = (T)c;
        L.e2a[k] = (T)(a * l2e); L.e2b[k] = (T)(b * l2e); L.e2c[k] = (T)(c * l2e);
    }
}

// the lens-light adjoint: pixels per thread and CTAs per evaluation
constexpr int LIGHT_PPT = 8;
__host__ __device__ inline int light_ctas(int n_img) {
    return (n_img * n_img + CTA_R * LIGHT_PPT - 1) / (CTA_R * LIGHT_PPT);
}

// 2^x: the float path takes the hardware approximation (PTX ex2.approx, relative error
// about 2^-22; subnormal results flushed to zero), the double path exp2
__device__ __forceinline__ float r_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double r_exp2(double x) { return exp2(x); }


// ------------------------------------------------------------ render tiles
// A render CTA covers an 8 x 16 pixel tile of four 8 x 4 warp blocks stacked in y; lane
// l of warp w takes pixel (l mod 8, 4 w + l / 8) of it.  A compact warp block straddles
// the edge of the arc's preimage less often than two 16-pixel rows (measured: the step
// 1.6% faster, the render adjoint 4%), so fewer warp steps carry both rays that leave
// the grid early and rays that do not, and the compacted ray list (warp by warp) keeps
// neighbouring rays together.  Tiles run row-major over the image.
constexpr int RT_X = 8, RT_Y = CTA_R / RT_X;
constexpr int RW_X = 8, RW_Y = 4;
static_assert(RW_X * RW_Y == 32 && (RT_X / RW_X) * (RT_Y / RW_Y) == CTA_R / 32, "warp blocks must tile a render tile");
__host__ __device__ inline int render_tiles_x(int n_img) { return (n_img + RT_X - 1) / RT_X; }
__host__ __device__ inline int render_tiles(int n_img) {
    return render_tiles_x(n_img) * ((n_img + RT_Y - 1) / RT_Y);
}
__device__ __forceinline__ int render_pixel(int n_img, int tile, int t, bool& valid) {
    const int tx_n = render_tiles_x(n_img);
    const int ty = tile / tx_n, tx = tile - ty * tx_n;
    const int w = t >> 5, l = t & 31;
    const int i = tx * RT_X + (w % (RT_X / RW_X)) * RW_X + (l % RW_X);
    const int j = ty * RT_Y + (w / (RT_X / RW_X)) * RW_Y + (l / RW_X);
    valid = i < n_img && j < n_img;
    return valid ? j * n_img + i : 0;
}
// Near-edge margin of the FP32 render: a ray whose grid coordinate lies within this
// many cells of a cell edge or of the grid boundary is decided in double.
constexpr float EDGE_DELTA = 2e-3f;

// The RTU grid's reach in beta per axis, [reach[2a], reach[2a+1]]: the z range whose
// image under the CDF comes within the near-edge margin of [0, 1] (the CDF is linear
// beyond its end knots), with slack, mapped back through the standardisation.  From the
// float transform; cg: read it through L2 (written by another CTA of the same kernel).
__device__ inline void grid_reach(const EvalArgs& E, bool cg, float* reach) {
    const int K = E.n_nodes + 2;
    const float* tr = E.trf;
    auto ld = [&](int i) { return cg ? __ldcg(tr + i) : tr[i]; };
    const float m = 4.0f * EDGE_DELTA / (E.n_src - 1);
    for (int a = 0; a < 2; ++a) {
        const int X = TR_HDR + a * K, d = TR_HDR + (2 + a) * K;
        float zlo = ld(X) - m / ld(d), zhi = ld(X + K - 1) + m / ld(d + K - 1);
        zlo -= 1e-3f * (1.0f + fabsf(zlo));
        zhi += 1e-3f * (1.0f + fabsf(zhi));
        const float lo = ld(a) + zlo * ld(2), hi = ld(a) + zhi * ld(2);
        reach[2 * a] = lo - 1e-5f * (1.0f + fabsf(lo));
        reach[2 * a + 1] = hi + 1e-5f * (1.0f + fabsf(hi));
    }
}

// True when no sub-ray of render tile `tile` can reach the RTU grid (beta beyond the
// reach on an axis), so that every ray would take the "far outside" exit: the tile's
// ray positions lie in a box; there the EPL deflection is at most
// P_max (1 + f/(1 - f)) (|c_n| < f, |w| = 1) with P = pref0 (b/R)^(t-1) taken at the
// box's smallest (t > 1) or largest (t < 1) elliptical radius R -- R >= q |theta - c|,
// and R is convex so its maximum sits at a corner -- and the shear deflection is
// linear (extremes at the corners).  Evaluated in float from the float lens block, with
// slack far above float rounding.  Subhaloes widen the deflection bound by
// sub_alpha_bound, whatever their positions.
__device__ inline bool tile_out_of_reach(const EvalArgs& E, int tile, const float* reach) {
    const LensK<float>& Kf = *reinterpret_cast<const LensK<float>*>(lensk_src<float>(E.lensk));
    const int n = E.n_img, tx_n = render_tiles_x(n);
    const int ty = tile / tx_n, tx = tile - ty * tx_n;
    const int i0 = tx * RT_X, i1 = min(i0 + RT_X - 1, n - 1);
    const int j0 = ty * RT_Y, j1 = min(j0 + RT_Y - 1, n - 1);
    const float c = 0.5f * (n - 1), pix = (float)E.pix;
    const float omin = (0.5f / E.s - 0.5f) * pix, omax = ((E.s - 0.5f) / E.s - 0.5f) * pix;
    const float xl = (i0 - c) * pix + omin, xh = (i1 - c) * pix + omax;
    const float yl = (j0 - c) * pix + omin, yh = (j1 - c) * pix + omax;
    const EplC<float>& C = Kf.C;
    // elliptical radius bounds over the box
    const float cx = fminf(fmaxf(C.x0, xl), xh), cy = fminf(fmaxf(C.y0, yl), yh);
    const float dmin = sqrtf((cx - C.x0) * (cx - C.x0) + (cy - C.y0) * (cy - C.y0));
    float rmax = 0.0f, shx_lo = 1e30f, shx_hi = -1e30f, shy_lo = 1e30f, shy_hi = -1e30f;
    for (int k = 0; k < 4; ++k) {
        const float x = (k & 1) ? xh : xl, y = (k & 2) ? yh : yl;
        const float dx = x - C.x0, dy = y - C.y0;
        const float xr = C.cp * dx + C.sp * dy, yr = C.cp * dy - C.sp * dx;
        rmax = fmaxf(rmax, sqrtf(C.q * C.q * xr * xr + yr * yr));
        const float sx = Kf.g1 * x + Kf.g2 * y, sy = Kf.g2 * x - Kf.g1 * y;
        shx_lo = fminf(shx_lo, sx); shx_hi = fmaxf(shx_hi, sx);
        shy_lo = fminf(shy_lo, sy); shy_hi = fmaxf(shy_hi, sy);
    }
    const float rmin = C.q * dmin * 0.999f;
    const float e = C.t - 1.0f;
    float pmax;
    if (e > 1e-6f) {
        if (rmin < 1e-4f) return false;
        pmax = C.pref0 * powf(C.b / rmin, e);
    } else if (e < -1e-6f) {
        pmax = C.pref0 * powf(C.b / fmaxf(rmax * 1.001f, 1e-6f), e);
    } else {
        pmax = C.pref0 * powf(fmaxf(C.b / fmaxf(rmin, 1e-4f), fmaxf(rmax, 1e-4f) / C.b), fabsf(e));
    }
    const float amax = pmax * (1.0f + C.ftail) * 1.001f + 1e-4f + sub_alpha_bound(Kf);
    const float sh_slack = 1e-5f * (fabsf(xl) + fabsf(xh) + fabsf(yl) + fabsf(yh) + 1.0f);
    // beta = theta - alpha_EPL - alpha_shear ranges per axis
    const float bxl = xl - shx_hi - amax - sh_slack, bxh = xh - shx_lo + amax + sh_slack;
    const float byl = yl - shy_hi - amax - sh_slack, byh = yh - shy_lo + amax + sh_slack;
    return bxh < reach[0] || bxl > reach[1] || byh < reach[2] || byl > reach[3];
}

// the ray id of staged entry `local` (lane s^2 + q) of render warp u
__device__ __forceinline__ int staged_ray_id(int n_img, int s2, int u, int local) {
    const int lane = local / s2, q = local - lane * s2;
    bool valid;
    const int pixel = render_pixel(n_img, u / (CTA_R / 32), (u % (CTA_R / 32)) * 32 + lane, valid);
    return pixel * s2 + q;
}

// Sub-ray positions in the kernel's type (Sec. 2.3): the offset from the image
// centre in pixel units, (i - (n-1)/2) + ((a + 1/2)/s - 1/2), is exact in float
// (a multiple of 1/(2s) for s a power of two), and it is scaled by the pixel size
// held as a (hi, lo) pair, so the position is rounded once instead of suffering a
// rounded image-centre offset shared by every ray.
template <typename T>
struct PixGeom {
    T hi, lo, ci;
    T offp[8];
};

template <typename T>
__device__ __forceinline__ void pixgeom_setup(PixGeom<T>& g, double pix, int n_img, int s) {
    if (threadIdx.x == 0) {
        g.hi = (T)pix;
        g.lo = (T)(pix - (double)g.hi);
        g.ci = (T)(0.5 * (n_img - 1));
    }
    if ((int)threadIdx.x < s) g.offp[threadIdx.x] = (T)((threadIdx.x + 0.5) / s - 0.5);
}

template <typename T>
__device__ __forceinline__ T ray_coord(const PixGeom<T>& g, int i, int a) {
    const T e = (T(i) - g.ci) + g.offp[a];
    return fma(e, g.hi, e * g.lo);
}

// pixel centre and sub-ray positions (Sec. 2.3) in double
__device__ __forceinline__ void ray_pos(int n_img, double pix, int s, int pixel, int sub,
                                        double& x, double& y) {
    int i = pixel % n_img, j = pixel / n_img;
    int a = sub % s, b = sub / s;
    double c = 0.5 * (n_img - 1);
    x = (i - c) * pix + ((a + 0.5) / s - 0.5) * pix;
    y = (j - c) * pix + ((b + 0.5) / s - 0.5) * pix;
}

}  // namespace rtu
