// k_render.cuh -- S7 (supersampled ray trace through the RTU map, bilinear
// source interpolation, supersample average), S11 (integer rays-per-cell
// histogram) and the atomic-free adjoint of the interpolation.
//
// The source grid of the evaluation is staged into shared memory with one TMA
// bulk copy (cp.async.bulk completing on an mbarrier); every ray then gathers
// its four bilinear corners from shared memory.
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

// ------------------------------------------------------------ TMA staging
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Stage `bytes` from global to shared in two parts, so that the copy runs while the
// CTA does other set-up: stage_begin (thread 0 initialises the barrier and issues the
// bulk copy; no CTA barrier) and stage_end (every thread; the wait).  Bulk path:
// bytes % 16 == 0 and both addresses 16-byte aligned; otherwise stage_end copies with
// plain loads.  No thread may leave between the two parts (a copy would be in flight).
// The wait is bounded: on give-up the flag word gets F_TIMEOUT and stage_end returns
// false after a second bounded wait for the copy; the caller then skips its work.
__device__ __forceinline__ bool stage_is_bulk(const void* dst, const void* src, uint32_t bytes) {
    return (bytes % 16u == 0u) && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u) &&
           ((smem_u32(dst) & 15u) == 0u) && bytes > 0u;
}
__device__ __forceinline__ void stage_begin(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    if (!stage_is_bulk(dst, src, bytes) || threadIdx.x != 0) return;
    const uint32_t mb = smem_u32(mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(mb)
        : "memory");
}
__device__ __forceinline__ bool stage_end(void* dst, const void* src, uint32_t bytes, uint64_t* mbar, int* flags) {
    if (!stage_is_bulk(dst, src, bytes)) {
        const unsigned char* s = static_cast<const unsigned char*>(src);
        unsigned char* d = static_cast<unsigned char*>(dst);
        for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) d[i] = s[i];
        __syncthreads();
        return true;
    }
    const uint32_t mb = smem_u32(mbar);
    __syncthreads();         // the barrier's initialisation is visible to every thread
    // bounded wait on phase 0
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mb), "r"(0u)
            : "memory");
    }
    int ok = __syncthreads_and(done ? 1 : 0);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(flags, F_TIMEOUT);
        // second bounded wait for the copy still in flight before the CTA may exit
        for (int it = 0; it < (1 << 24) && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(mb), "r"(0u)
                : "memory");
        }
        __syncthreads();
        return false;
    }
    return true;
}

// ------------------------------------------------------ Hermite CDF (App. C iv)
// knots X[0..K-1], values U, slopes d.  Interval code: -1 left of X[0], K-1 at or
// right of X[K-1], else j with X[j] <= z < X[j+1].
template <typename T>
__device__ __forceinline__ int cdf_interval(const T* X, int K, T z) {
    if (z < X[0]) return -1;
    if (z >= X[K - 1]) return K - 1;
    int lo = 0, hi = K - 1;     // X[lo] <= z < X[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (X[mid] <= z) lo = mid; else hi = mid;
    }
    return lo;
}

// the same from a table of the interval at IV_BINS equal bins over [X_0, X_{K-1}]
// (iv[b] = the interval holding the bin's left edge, origin o, scale sc = IV_BINS /
// (X_{K-1} - X_0)): the table's guess is moved up or down to the interval holding z,
// so the result is the binary search's; the knots inside one bin bound the steps
constexpr int IV_BINS = 64;
template <typename T>
__device__ __forceinline__ int cdf_interval_lut(const T* X, int K, T z, const unsigned char* iv, T o, T sc) {
    if (z < X[0]) return -1;
    if (z >= X[K - 1]) return K - 1;
    int b = (int)((z - o) * sc);
    b = b < 0 ? 0 : (b > IV_BINS - 1 ? IV_BINS - 1 : b);
    int j = iv[b];
    while (j < K - 2 && X[j + 1] <= z) ++j;
    while (j > 0 && X[j] > z) --j;
    return j;
}

template <typename T>
__device__ __forceinline__ T cdf_value(const T* X, const T* U, const T* d, int K, int j, T z) {
    if (j < 0) return U[0] + d[0] * (z - X[0]);
    if (j >= K - 1) return U[K - 1] + d[K - 1] * (z - X[K - 1]);
    T h = X[j + 1] - X[j];
    T t = (z - X[j]) / h;
    T t2 = t * t, t3 = t2 * t;
    T h00 = T(2) * t3 - T(3) * t2 + T(1);
    T h10 = t3 - T(2) * t2 + t;
    T h01 = T(-2) * t3 + T(3) * t2;
    T h11 = t3 - t2;
    return h00 * U[j] + h10 * h * d[j] + h01 * U[j + 1] + h11 * h * d[j + 1];
}

// the same with the interval's 1/h from a table (no division per ray)
template <typename T>
__device__ __forceinline__ T cdf_value_r(const T* X, const T* U, const T* d, const T* IH, int K, int j, T z) {
    if (j < 0) return U[0] + d[0] * (z - X[0]);
    if (j >= K - 1) return U[K - 1] + d[K - 1] * (z - X[K - 1]);
    T h = X[j + 1] - X[j];
    T t = (z - X[j]) * IH[j];
    T t2 = t * t, t3 = t2 * t;
    T h00 = T(2) * t3 - T(3) * t2 + T(1);
    T h10 = t3 - T(2) * t2 + t;
    T h01 = T(-2) * t3 + T(3) * t2;
    T h11 = t3 - t2;
    return h00 * U[j] + h10 * h * d[j] + h01 * U[j + 1] + h11 * h * d[j + 1];
}

// value, dC/dz and the partials w.r.t. (X_j, X_{j+1}, d_j, d_{j+1}) of the
// touched knots (for the extrapolation branches only one knot is touched: the
// left branch reports it in slot "j+1" = knot 0, the right in slot "j" = K-1).
// IH holds 1/(X_{j+1} - X_j) per interval.
template <typename T>
__device__ __forceinline__ T cdf_grad(const T* X, const T* U, const T* d, const T* IH, int K, int j, T z, T& dz,
                                      T& pX0, T& pX1, T& pd0, T& pd1) {
    if (j < 0) {
        dz = d[0]; pX0 = T(0); pd0 = T(0); pX1 = -d[0]; pd1 = z - X[0];
        return U[0] + d[0] * (z - X[0]);
    }
    if (j >= K - 1) {
        dz = d[K - 1]; pX1 = T(0); pd1 = T(0); pX0 = -d[K - 1]; pd0 = z - X[K - 1];
        return U[K - 1] + d[K - 1] * (z - X[K - 1]);
    }
    T h = X[j + 1] - X[j], ih = IH[j];
    T t = (z - X[j]) * ih;
    T t2 = t * t, t3 = t2 * t;
    T h00 = T(2) * t3 - T(3) * t2 + T(1), h10 = t3 - T(2) * t2 + t;
    T h01 = T(-2) * t3 + T(3) * t2, h11 = t3 - t2;
    T h00p = T(6) * t2 - T(6) * t, h10p = T(3) * t2 - T(4) * t + T(1);
    T h01p = T(-6) * t2 + T(6) * t, h11p = T(3) * t2 - T(2) * t;
    T Dz = (h00p * U[j] + h01p * U[j + 1]) * ih + h10p * d[j] + h11p * d[j + 1];
    T Hd = h10 * d[j] + h11 * d[j + 1];
    dz = Dz;
    pX0 = Dz * (t - T(1)) - Hd;
    pX1 = -Dz * t + Hd;
    pd0 = h * h10;
    pd1 = h * h11;
    return h00 * U[j] + h10 * h * d[j] + h01 * U[j + 1] + h11 * h * d[j + 1];
}

// ------------------------------------------- the unsmoothed eCDF (App. C)
// Observation i of axis a is at most b: double positions, or float (hi, lo) pairs
// compared exactly against a float b.
__device__ __forceinline__ bool lin_le(const EvalArgs& E, int a, int i, double b) {
    return E.lkey[(size_t)a * E.n_mask + i] <= b;
}
__device__ __forceinline__ bool lin_le(const EvalArgs& E, int a, int i, float b) {
    const float2 k = reinterpret_cast<const float2*>(E.lkf)[(size_t)a * E.n_mask + i];
    return k.x < b || (k.x == b && k.y <= 0.0f);
}
// position difference b - x_i and segment width x_{i+1} - x_i in the kernel's type
__device__ __forceinline__ void lin_seg(const EvalArgs& E, int a, int i, double b, double& d0, double& h) {
    const double* k = E.lkey + (size_t)a * E.n_mask + i;
    d0 = b - k[0];
    h = k[1] - k[0];
}
__device__ __forceinline__ void lin_seg(const EvalArgs& E, int a, int i, float b, float& d0, float& h) {
    const float2* k = reinterpret_cast<const float2*>(E.lkf) + (size_t)a * E.n_mask + i;
    const float2 k0 = k[0], k1 = k[1];
    d0 = (b - k0.x) - k0.y;
    h = (k1.x - k0.x) + (k1.y - k0.y);
}

// #{observations of axis a <= b}.  The histogram bin of b (bin origin bo, scale bs;
// in float it can be off by one) narrows the search to the bins next to it; the
// window is checked at both ends, else the search runs over all observations.
// After k_lin_sort, hist[b] is the end of bin b.
template <typename T>
__device__ __forceinline__ int lin_count(const EvalArgs& E, int a, T b, T bo, T bs) {
    const int N = E.n_mask;
    const int* h = E.hist + a * HB;
    const T t = (b - bo) * bs;
    const int bin = t > T(0) ? (t < T(HB - 1) ? (int)t : HB - 1) : 0;
    int lo = bin > 1 ? min(h[bin - 2], N) : 0;
    int hi = bin < HB - 1 ? min(h[bin + 1], N) : N;
    if (!((lo == 0 || lin_le(E, a, lo - 1, b)) && (hi == N || !lin_le(E, a, hi, b)))) {
        lo = 0;
        hi = N;
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lin_le(E, a, mid, b)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// u = (k + t)/(N - 1) on segment k = clamp(count - 1, 0, N - 2), t = (b - x_k)/(x_{k+1} - x_k);
// beyond the end observations the end segment continues; a zero-width segment
// gives t = 0.  With grad: du/db and the partials w.r.t. x_k and x_{k+1}.
template <typename T>
__device__ __forceinline__ T lin_value(const EvalArgs& E, int a, T b, T bo, T bs, T inv_nm1, int& k, T* dub = nullptr,
                                       T* p0 = nullptr, T* p1 = nullptr) {
    const int N = E.n_mask;
    k = min(max(lin_count<T>(E, a, b, bo, bs) - 1, 0), N - 2);
    T d0, h;
    lin_seg(E, a, k, b, d0, h);
    const bool ok = h > T(0);
    const T ih = ok ? T(1) / h : T(0);
    const T t = d0 * ih;
    if (dub) {
        const T s = inv_nm1 * ih;
        *dub = s;
        *p0 = (t - T(1)) * s;
        *p1 = -t * s;
    }
    return ((T)k + t) * inv_nm1;
}

// bin origin and scale of axis a from the transform block
template <typename T>
__device__ __forceinline__ void lin_bins(const EvalArgs& E, int a, T& bo, T& bs) {
    const int K = E.n_nodes + 2;
    const int at = TR_HDR + 6 * K;
    if (sizeof(T) == 4) { bo = (T)E.trf[at + a]; bs = (T)E.trf[at + 2 + a]; }
    else { bo = (T)E.trd[at + a]; bs = (T)E.trd[at + 2 + a]; }
}

// transform (mu, sigma, knots, slopes) and node values into shared memory
template <typename T>
__device__ __forceinline__ void load_transform(const EvalArgs& E, T* trs, T* U) {
    const int K = E.n_nodes + 2;
    const int nt = TR_HDR + 4 * K;
    for (int i = threadIdx.x; i < nt; i += blockDim.x)
        trs[i] = sizeof(T) == 4 ? (T)E.trf[i] : (T)E.trd[i];
    for (int j = threadIdx.x; j < K; j += blockDim.x)
        U[j] = (T)(j == 0 ? 0.0 : (j == K - 1 ? 1.0 : E.cheb[cheb_u(E.n_nodes, E.degree) + j - 1]));
}

// S7 + S11: one thread per image pixel, s^2 sub-rays each.
// Near-edge FP64 island (float mode): a ray whose grid coordinate lies within
// EDGE_DELTA cells of a cell edge or of the grid boundary is not decided in
// float.  The render kernel appends it to a per-evaluation list; k_render_edge
// traces the listed rays in double (no warp divergence in the float kernel), and
// the thread finishing a pixel's last deferred ray completes the pixel in a fixed
// order.  So the integer
// cell of every ray -- the rays-per-cell histogram and the kink of the bilinear
// slope the adjoint differentiates -- is the double-precision decision.

__device__ __forceinline__ bool near_edge(float gx, float gy, int n) {
    const float lo = -EDGE_DELTA, hi = (float)(n - 1) + EDGE_DELTA;
    if (gx < lo || gx > hi || gy < lo || gy > hi) return false;     // clearly outside
    const float fx = gx - floorf(gx), fy = gy - floorf(gy);
    return fx < EDGE_DELTA || fx > 1.0f - EDGE_DELTA || fy < EDGE_DELTA || fy > 1.0f - EDGE_DELTA;
}

// the same with extra margins mx, my (cells) per axis
__device__ __forceinline__ bool near_edge_m(float gx, float gy, int n, float mx, float my) {
    const float dx = EDGE_DELTA + mx, dy = EDGE_DELTA + my;
    if (gx < -dx || gx > (float)(n - 1) + dx || gy < -dy || gy > (float)(n - 1) + dy) return false;
    const float fx = gx - floorf(gx), fy = gy - floorf(gy);
    return fx < dx || fx > 1.0f - dx || fy < dy || fy > 1.0f - dy;
}

// bilinear value at grid coordinate (gx, gy) with the cell decided by the caller
template <typename T, typename G>
__device__ __forceinline__ T bilinear_at(const G* grid, int n, int i0, int j0, T fx, T fy) {
    const G* r0 = grid + j0 * n + i0;
    return (T(1) - fx) * (T(1) - fy) * (T)r0[0] + fx * (T(1) - fy) * (T)r0[1] + (T(1) - fx) * fy * (T)r0[n] +
           fx * fy * (T)r0[n + 1];
}

// cell of a grid coordinate inside [0, n-1]^2 (else -1), and the offsets in it
template <typename T>
__device__ __forceinline__ int cell_of(T yx, T yy, int n, T& fx, T& fy, int& i0, int& j0) {
    if (!(yx >= T(0) && yx <= T(1) && yy >= T(0) && yy <= T(1))) return -1;
    const T gx = yx * T(n - 1), gy = yy * T(n - 1);
    i0 = (int)gx;
    j0 = (int)gy;
    i0 = i0 > n - 2 ? n - 2 : i0;
    j0 = j0 > n - 2 ? n - 2 : j0;
    fx = gx - T(i0);
    fy = gy - T(j0);
    return j0 * (n - 1) + i0;
}

// double-precision grid coordinates of a source-plane position (the Hermite CDF
// from the shared transform block, or the unsmoothed eCDF)
__device__ __forceinline__ void rtu_coords_from_beta(const EvalArgs& E, const double* trd, const double* U, int K,
                                                     double bx, double by, double& yx, double& yy) {
    if (E.transform == RTU_TRANSFORM_LINEAR) {
        const double inv = 1.0 / (E.n_mask - 1);
        double bo, bs;
        int k;
        lin_bins<double>(E, 0, bo, bs);
        yx = lin_value<double>(E, 0, bx, bo, bs, inv, k);
        lin_bins<double>(E, 1, bo, bs);
        yy = lin_value<double>(E, 1, by, bo, bs, inv, k);
        return;
    }
    const double* X = trd + TR_HDR;
    const double zx = (bx - trd[0]) / trd[2], zy = (by - trd[1]) / trd[2];
    yx = cdf_value<double>(X, U, X + 2 * K, K, cdf_interval<double>(X, K, zx), zx);
    yy = cdf_value<double>(X + K, U, X + 3 * K, K, cdf_interval<double>(X + K, K, zy), zy);
}

// double-precision grid coordinates of a ray from the double lens block
__device__ __forceinline__ void rtu_coords_d(const EvalArgs& E, const LensK<double>& Kd, const double* trd,
                                             const double* U, int K, double x, double y, double& yx, double& yy) {
    double bx, by;
    lens_beta(Kd, x, y, bx, by);
    rtu_coords_from_beta(E, trd, U, K, bx, by, yx, yy);
}

template <typename T>
struct RenderShared {
    LensK<T> K;
    T trs[TR_HDR + 4 * (MAXM + 2)];
    T U[MAXM + 2];
    PixGeom<T> G;              // sub-ray positions
    T ih[2 * (MAXM + 2)];      // 1/(X_{j+1} - X_j) per knot interval, axis-major
    UDiv dv_s2, dv_n, dv_s, dv_nc;   // dividers by s^2, n_img, s, n_src - 1
    unsigned char iv[2][IV_BINS];    // per axis: the knot interval at each table bin's left edge
    T ivo[2], ivs[2];                // per axis: the table's origin X_0 and scale IV_BINS/(X_{K-1} - X_0)
};

// Source grids up to GRID_STAGE_MAX bytes are staged in shared memory; larger ones
// (float n_src = 256, double n_src >= 144) are read through L1/L2 from global memory.
constexpr uint32_t GRID_STAGE_MAX = 160u * 1024u;
__host__ __device__ inline bool grid_staged(int n_src, int bytes_per_value) {
    return (uint32_t)n_src * (uint32_t)n_src * (uint32_t)bytes_per_value <= GRID_STAGE_MAX;
}
// bytes of dynamic shared memory the staged grid takes (0 when read from global)
__host__ __device__ inline size_t grid_smem_bytes(int n_src, int bytes_per_value) {
    return grid_staged(n_src, bytes_per_value) ? ((size_t)n_src * n_src * bytes_per_value + 127) & ~(size_t)127 : 0;
}

template <typename T>
__device__ __forceinline__ void render_setup(const EvalArgs& E, RenderShared<T>& sh) {
    load_lensk(sh.K, lensk_src<T>(E.lensk));
    load_transform<T>(E, sh.trs, sh.U);
    {
        const int K = E.n_nodes + 2;
        for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) {
            const int a = i / K, j = i - a * K;
            if (j < K - 1) {
                const int at = TR_HDR + a * K + j;
                const T x0 = sizeof(T) == 4 ? (T)E.trf[at] : (T)E.trd[at];
                const T x1 = sizeof(T) == 4 ? (T)E.trf[at + 1] : (T)E.trd[at + 1];
                sh.ih[i] = T(1) / (x1 - x0);
            }
        }
    }
    // the interval table: one thread per (axis, bin), a scan of the axis's knots
    {
        const int K = E.n_nodes + 2;
        for (int i = threadIdx.x; i < 2 * IV_BINS; i += blockDim.x) {
            const int a = i / IV_BINS, b = i - a * IV_BINS;
            auto X = [&](int j) {
                const int at = TR_HDR + a * K + j;
                return sizeof(T) == 4 ? (T)E.trf[at] : (T)E.trd[at];
            };
            const T o = X(0), sc = T(IV_BINS) / (X(K - 1) - o);
            const T edge = o + T(b) / sc;
            int j = 0;
            while (j < K - 2 && X(j + 1) <= edge) ++j;
            sh.iv[a][b] = (unsigned char)j;
            if (b == 0) { sh.ivo[a] = o; sh.ivs[a] = sc; }
        }
    }
    pixgeom_setup<T>(sh.G, E.pix, E.n_img, E.s);
    if (threadIdx.x == 0) {
        sh.dv_s2 = udiv_make((uint32_t)(E.s * E.s));
        sh.dv_n = udiv_make((uint32_t)E.n_img);
        sh.dv_s = udiv_make((uint32_t)E.s);
        sh.dv_nc = udiv_make((uint32_t)(E.n_src - 1));
    }
}

// the tile test for every render tile of an evaluation, one thread per tile (the
// unsmoothed map's systems; the smoothed grid's last k_select_fit CTA does it for its
// own), after the transform is built: k_render reads the byte
constexpr int CULL_NT = 256;
__global__ void __launch_bounds__(CULL_NT) k_cull_tiles(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    __shared__ float reach[4];
    if (threadIdx.x == 0) grid_reach(E, false, reach);
    __syncthreads();
    const int tile = (blockIdx.x - B.tile0[ev]) * CULL_NT + threadIdx.x;
    if (tile < E.n_cta_r) E.tcull[tile] = tile_out_of_reach(E, tile, reach) ? 1 : 0;
}

// S7 + S11: one thread per image pixel, s^2 sub-rays each.  LIN: the unsmoothed
// eCDF map (its own instantiation, so the smoothed map's code is not burdened).
template <typename T, bool LIN>
__global__ void __launch_bounds__(CTA_R, sizeof(T) == 4 && !LIN ? 8 : 6) k_render(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sgrid = reinterpret_cast<T*>(smem_raw);
    __shared__ RenderShared<T> sh;
    __shared__ __align__(8) uint64_t mbar;
    const int n = E.n_src, K = E.n_nodes + 2;
    __shared__ int cnt_sh, cull_sh;
    bool valid;
    const int pixel = render_pixel(E.n_img, tile, threadIdx.x, valid);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s = E.s, s2 = E.s * E.s;
    if (threadIdx.x == 0) {
        cnt_sh = 0;
        cull_sh = E.tcull[tile];
    }
    __syncthreads();
    if (cull_sh) {
        // no ray of this tile reaches the grid: a zero source image, nothing staged
        if (threadIdx.x < CTA_R / 32) E.useg[tile * (CTA_R / 32) + threadIdx.x] = 0;
        if (threadIdx.x < CTA_R / 32) E.nseg[tile * (CTA_R / 32) + threadIdx.x] = 0;
        if (threadIdx.x == 0) E.cta_cnt[tile] = 0;
        if (!valid) return;
        if (sizeof(T) == 4) E.pdef[pixel] = 0ull;
        reinterpret_cast<T*>(E.img)[pixel] = T(0);
        if (E.image_out) reinterpret_cast<T*>(E.image_out)[pixel] = T(0);
        return;
    }
    // the source grid's copy runs beside the set-up (or the grid is read from global)
    const bool gstaged = grid_staged(n, sizeof(T));
    const T* grid = gstaged ? sgrid : reinterpret_cast<const T*>(E.src);
    if (gstaged) stage_begin(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar);
    render_setup<T>(E, sh);
    if (!gstaged) __syncthreads();
    if (gstaged && !stage_end(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar, E.flags)) {
        // the copy timed out (flagged): this tile stages nothing
        if (threadIdx.x < CTA_R / 32) E.useg[tile * (CTA_R / 32) + threadIdx.x] = 0;
        if (threadIdx.x < CTA_R / 32) E.nseg[tile * (CTA_R / 32) + threadIdx.x] = 0;
        if (threadIdx.x == 0) E.cta_cnt[tile] = 0;
        return;
    }
    int nin = 0;                 // in-grid (or deferred) sub-rays of this pixel
    const T mux = sh.trs[0], muy = sh.trs[1], isg = T(1) / sh.trs[2];
    const T* Xx = sh.trs + TR_HDR;
    const T* Xy = Xx + K;
    const T* dx_ = Xx + 2 * K;
    const T* dy_ = Xx + 3 * K;
    // z range whose image under the CDF reaches within the near-edge margin of
    // [0, 1] (the CDF is linear beyond its end knots with slopes d_0, d_{K-1})
    T zlo[2], zhi[2];
    for (int a = 0; a < 2; ++a) {
        const T* X = Xx + a * K;
        const T* d = dx_ + a * K;
        const T m = T(4) * T(EDGE_DELTA) / T(n - 1);
        zlo[a] = X[0] - m / d[0];
        zhi[a] = X[K - 1] + m / d[K - 1];
    }
    const int pj = (int)udiv((uint32_t)pixel, sh.dv_n), pi = pixel - pj * E.n_img;
    // the unsmoothed eCDF: bin lookup constants (z is the raw position there)
    constexpr bool lin = LIN;
    T lbo[2] = {T(0), T(0)}, lbs[2] = {T(0), T(0)};
    const T linv = lin ? T(1) / T(E.n_mask - 1) : T(0);
    if (lin) {
        lin_bins<T>(E, 0, lbo[0], lbs[0]);
        lin_bins<T>(E, 1, lbo[1], lbs[1]);
    }

    T acc = T(0);
    unsigned long long deferred = 0ull;      // bit q: sub-ray q went to the double pass
    // this warp's staging segment: in-grid and deferred rays appended in (q, lane) order
    const size_t ubase = ((size_t)tile * (CTA_R / 32) + wid) * 32 * s2;
    int* stg = E.cell + ubase;
    int wpos = 0;
    // code of a sub-ray: -1 no cell, 0 deferred to the double pass, c + 1 in cell c
    unsigned long long nearm = 0ull;         // bit q: sub-ray q is near a lens core
    auto trace = [&](int q) -> int {
        const int qb = (int)udiv((uint32_t)q, sh.dv_s), qa = q - qb * s;
        const T x = ray_coord(sh.G, pi, qa), y = ray_coord(sh.G, pj, qb);
        T yx, yy;
        if (sizeof(T) == 4 && lens_near_core(sh.K, x, y)) {
            // near a lens core: traced and decided by the double pass, and
            // differentiated by the adjoint's near-core pass
            nearm |= 1ull << q;
            deferred |= 1ull << q;
            ++nin;
            return 0;
        } else {
            T bx, by;
            if (sh.K.nsub == 0) {
                // two series terms first: a ray whose partial z lies beyond the
                // margin by more than the tail bound (and a rounding allowance)
                // is outside the grid whatever the other terms add
                EplPart<T> ps;
                epl_alpha_begin(sh.K.C, x, y, 2, ps);
                T ax, ay;
                epl_alpha_of(sh.K.C, ps, ax, ay);
                const T shx = sh.K.g1 * x + sh.K.g2 * y, shy = sh.K.g2 * x - sh.K.g1 * y;
                const T px = (x - (ax + shx) - mux) * isg, py = (y - (ay + shy) - muy) * isg;
                const T tail = (T(1.25) * epl_tail_bound(sh.K.C, ps) +
                                T(1e-6) * (T(1) + r_abs(ax) + r_abs(ay) + r_abs(x) + r_abs(y))) * isg;
                if (px < zlo[0] - tail || px > zhi[0] + tail || py < zlo[1] - tail || py > zhi[1] + tail)
                    return -1;
                epl_alpha_finish(sh.K.C, ps, ax, ay);
                bx = x - (ax + shx);
                by = y - (ay + shy);
            } else {
                // with subhaloes: the same two-term test, the tail widened by the bound on
                // the subhaloes' deflection; a ray that may reach the grid takes the full
                // lens equation (the same bits as without the test)
                EplPart<T> ps;
                epl_alpha_begin(sh.K.C, x, y, 2, ps);
                T ax, ay;
                epl_alpha_of(sh.K.C, ps, ax, ay);
                const T shx = sh.K.g1 * x + sh.K.g2 * y, shy = sh.K.g2 * x - sh.K.g1 * y;
                const T px = (x - (ax + shx) - mux) * isg, py = (y - (ay + shy) - muy) * isg;
                const T tail = (T(1.25) * epl_tail_bound(sh.K.C, ps) + sub_alpha_bound(sh.K) +
                                T(1e-6) * (T(1) + r_abs(ax) + r_abs(ay) + r_abs(x) + r_abs(y))) * isg;
                if (px < zlo[0] - tail || px > zhi[0] + tail || py < zlo[1] - tail || py > zhi[1] + tail)
                    return -1;
                lens_beta(sh.K, x, y, bx, by);
            }
            const T zx = (bx - mux) * isg, zy = (by - muy) * isg;
            // far outside the grid (beyond the near-edge margin): no cell, zero source
            if (zx < zlo[0] || zx > zhi[0] || zy < zlo[1] || zy > zhi[1]) return -1;
            float mx = 0.0f, my = 0.0f;     // extra near-edge margin (cells)
            if constexpr (lin) {
                int kk;
                T sx, sy, pu;
                yx = lin_value<T>(E, 0, zx, lbo[0], lbs[0], linv, kk, &sx, &pu, &pu);
                yy = lin_value<T>(E, 1, zy, lbo[1], lbs[1], linv, kk, &sy, &pu, &pu);
                if (sizeof(T) == 4) {
                    // the float position's error (a few 1e-7 of the positions involved)
                    // times the map's slope there, in cells: narrow segments make it large
                    mx = (float)(T(n - 1) * sx * T(1e-6) * (T(1) + r_abs(zx) + r_abs(x)));
                    my = (float)(T(n - 1) * sy * T(1e-6) * (T(1) + r_abs(zy) + r_abs(y)));
                }
            } else {
                const int jx = cdf_interval_lut<T>(Xx, K, zx, sh.iv[0], sh.ivo[0], sh.ivs[0]);
                const int jy = cdf_interval_lut<T>(Xy, K, zy, sh.iv[1], sh.ivo[1], sh.ivs[1]);
                yx = cdf_value_r<T>(Xx, sh.U, dx_, sh.ih, K, jx, zx);
                yy = cdf_value_r<T>(Xy, sh.U, dy_, sh.ih + K, K, jy, zy);
            }
            if (sizeof(T) == 4 && (lin ? near_edge_m((float)(yx * T(n - 1)), (float)(yy * T(n - 1)), n, mx, my)
                                       : near_edge((float)(yx * T(n - 1)), (float)(yy * T(n - 1)), n))) {
                deferred |= 1ull << q;
                ++nin;               // may turn out outside: k_render_edge takes it back
                return 0;
            }
        }
        T fx, fy;
        int i0, j0;
        const int cell = cell_of<T>(yx, yy, n, fx, fy, i0, j0);
        if (cell < 0) return -1;
        acc += bilinear_at<T, T>(grid, n, i0, j0, fx, fy);
        atomicAdd(E.ccount + cell, 1);
        ++nin;
        return cell + 1;
    };
    // codes of this thread's sub-rays in shared memory (16 bits: cell + 1 < 2^16 - 1
    // for n_src <= 256, 0xffff for no cell), then the warp's staged rays in ray
    // order (lane-major, i.e. pixel by pixel): consecutive adjoint rays then come
    // from the same or neighbouring pixels (layout [q][thread]: conflict-free banks)
    unsigned short* codes = reinterpret_cast<unsigned short*>(smem_raw + grid_smem_bytes(n, sizeof(T))) + threadIdx.x;
    int mine = 0;
    for (int q = 0; q < s2; ++q) {
        const int code = valid ? trace(q) : -1;
        codes[q * CTA_R] = (unsigned short)(code < 0 ? 0xffff : code);
        mine += code >= 0;
    }
    int excl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, excl, o);
        if (lane >= o) excl += y;
    }
    wpos = __shfl_sync(0xffffffffu, excl, 31);
    excl -= mine;
    const int mnear = __popcll(nearm);      // near-core rays of this thread (all staged)
    for (int q = 0, pos = excl; q < s2; ++q) {
        const int c16 = codes[q * CTA_R];
        if (c16 == 0xffff) continue;
        const int code = c16;
        stg[pos] = (lane * s2 + q) | (code << STG_SHIFT) | ((nearm >> q & 1ull) ? STG_NEAR : 0) |
                   (code == 0 ? STG_DEFER : 0);
        if (code == 0) {
            // the double pass finds the ray through its staging position
            const int at = atomicAdd(E.ecount, 1);
            E.elist[at] = (int)(ubase + pos);
        }
        ++pos;
    }
    const int wnear = __reduce_add_sync(0xffffffffu, mnear);
    if (lane == 0) {
        E.useg[tile * (CTA_R / 32) + wid] = wpos;
        E.nseg[tile * (CTA_R / 32) + wid] = wnear;
    }
    // in-grid rays of the CTA (deferred rays counted; k_render_edge takes back the
    // ones that end outside): the N_IN_GRID statistic
    atomicAdd(&cnt_sh, nin);
    __syncthreads();
    if (threadIdx.x == 0) E.cta_cnt[tile] = cnt_sh;
    if (!valid) return;
    if (sizeof(T) == 4) {
        E.pdef[pixel] = deferred;
        if (deferred) E.pcnt[pixel] = __popcll(deferred);
    }
    // pixels with deferred rays keep the partial sum; k_render_edge completes them
    const T val = deferred ? acc : acc / T(s2);
    reinterpret_cast<T*>(E.img)[pixel] = val;
    if (E.image_out && !deferred) reinterpret_cast<T*>(E.image_out)[pixel] = val;
}

// Distance of a double-float grid coordinate from the nearest integer (a cell edge
// or the grid boundary), in cells
__device__ __forceinline__ float df_edge_dist(const DF& g) {
    const float r = rintf(g.hi);
    return fabsf((g.hi - r) + g.lo);      // g.hi - r is exact
}
// floor of a double-float value (hi may have rounded up onto the integer above it)
__device__ __forceinline__ int df_floor(const DF& g) {
    int i = (int)floorf(g.hi);
    if ((float)i == g.hi && g.lo < 0.0f) --i;
    return i;
}

// the deferred near-edge rays of the float path, traced and decided in double
constexpr int EDGE_NT = 128;
constexpr int EDGE_CTAS = 16;      // CTAs per evaluation (default; E.n_edge when tuned)
__global__ void __launch_bounds__(EDGE_NT) k_render_edge(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LensK<double> Kd;
    __shared__ LensK<DF> Kdf;
    __shared__ double trd[TR_HDR + 4 * (MAXM + 2)];
    __shared__ double Ud[MAXM + 2];
    __shared__ DF trx[TR_HDR + 4 * (MAXM + 2)];
    __shared__ DF Ux[MAXM + 2];
    load_lensk(Kd, E.lensk);
    load_transform<double>(E, trd, Ud);
    __syncthreads();
    // the lens in double-float (about 48 bits) unless subhaloes are present; the
    // Hermite map in double-float too, with the cell decided from it where the grid
    // coordinate is farther from every cell edge than the map's double-float error
    // bound, else (rarely) by the map in double from the same position
    const bool use_df = Kd.nsub == 0;
    const int n = E.n_src, K = E.n_nodes + 2, s2 = E.s * E.s;
    const bool map_df = use_df && E.transform != RTU_TRANSFORM_LINEAR;
    if (use_df) {
        load_lensk(Kdf, lensk_df_src(E.lensk));
        if (map_df) {
            for (int i = threadIdx.x; i < TR_HDR + 4 * K; i += EDGE_NT) trx[i] = DF(trd[i]);
            for (int j = threadIdx.x; j < K; j += EDGE_NT) Ux[j] = DF(Ud[j]);
        }
        __syncthreads();
    }
    const int cnt = min(*E.ecount, E.n_img * E.n_img * s2);
    const float* grid = reinterpret_cast<const float*>(E.src);
    float* img = reinterpret_cast<float*>(E.img);
    const int cap = 32 * s2;                 // staged entries per render warp
    for (int k = tile * EDGE_NT + threadIdx.x; k < cnt; k += E.n_edge * EDGE_NT) {
        const int at = E.elist[k];     // staging position
        const int e0 = E.cell[at];
        const int local = e0 & ((1 << STG_SHIFT) - 1);
        const int u = at / cap;
        const int ray = staged_ray_id(E.n_img, s2, u, local);
        const int pixel = ray / s2, q = ray - pixel * s2;
        double xd, yd, yx, yy;
        ray_pos(E.n_img, E.pix, E.s, pixel, q, xd, yd);
        int cell = -1, i0 = 0, j0 = 0;
        float fxf = 0.0f, fyf = 0.0f;
        bool decided = false;
        if (use_df) {
            DF bxf, byf;
            lens_beta_smooth<DF>(Kdf, DF(xd), DF(yd), bxf, byf);
            if (map_df) {
                // the Hermite map (App. C iv) in double-float: z, its interval, the value
                const DF isg = DF(1.0f) / trx[2];
                const DF zx = (bxf - trx[0]) * isg, zy = (byf - trx[1]) * isg;
                const DF* X = trx + TR_HDR;
                const int jx = cdf_interval<DF>(X, K, zx), jy = cdf_interval<DF>(X + K, K, zy);
                const DF gx = cdf_value<DF>(X, Ux, X + 2 * K, K, jx, zx) * DF((float)(n - 1));
                const DF gy = cdf_value<DF>(X + K, Ux, X + 3 * K, K, jy, zy) * DF((float)(n - 1));
                // error bound of the double-float map, in cells: 2^-36 (over 2^10 times
                // the pair type's tested 2^-46 per operation) of the terms, scaled by
                // |z| and a bound on the map's slope in the interval -- the knots'
                // slopes and three times the secant (a narrow interval amplifies the
                // error of z - X_j by 1/h); an interval too narrow to measure in float
                // leaves the ray to the double map
                auto slope_bound = [&](const DF* Xa, const DF* da, int j) -> float {
                    const int k0 = j < 0 ? 0 : j;
                    float sb = fmaxf(da[k0].hi, da[min(k0 + 1, K - 1)].hi);
                    if (j >= 0 && j < K - 1) {
                        const float h = (Xa[j + 1].hi - Xa[j].hi) + (Xa[j + 1].lo - Xa[j].lo);
                        sb = h > 0.0f ? fmaxf(sb, 3.0f * (Ux[j + 1].hi - Ux[j].hi) / h) : INFINITY;
                    }
                    return sb;
                };
                const float sx = slope_bound(X, X + 2 * K, jx), sy = slope_bound(X + K, X + 3 * K, jy);
                const float tol_x = (float)(n - 1) * 1.4551915e-11f * (1.0f + fabsf(zx.hi)) * (1.0f + sx) + 1e-12f;
                const float tol_y = (float)(n - 1) * 1.4551915e-11f * (1.0f + fabsf(zy.hi)) * (1.0f + sy) + 1e-12f;
                if (df_edge_dist(gx) > tol_x && df_edge_dist(gy) > tol_y) {
                    decided = true;
                    const DF zero(0.0f, 0.0f), top((float)(n - 1), 0.0f);
                    if (zero < gx && gx < top && zero < gy && gy < top) {
                        i0 = df_floor(gx);
                        j0 = df_floor(gy);
                        fxf = (gx.hi - (float)i0) + gx.lo;
                        fyf = (gy.hi - (float)j0) + gy.lo;
                        cell = j0 * (n - 1) + i0;
                    }
                }
            }
            if (!decided) rtu_coords_from_beta(E, trd, Ud, K, bxf.to_double(), byf.to_double(), yx, yy);
        } else {
            rtu_coords_d(E, Kd, trd, Ud, K, xd, yd, yx, yy);
        }
        if (!decided) {
            double fx, fy;
            cell = cell_of<double>(yx, yy, n, fx, fy, i0, j0);
            fxf = (float)fx;
            fyf = (float)fy;
        }
        float v = 0.0f;
        if (cell >= 0) {
            v = bilinear_at<float, float>(grid, n, i0, j0, fxf, fyf);
            atomicAdd(E.ccount + cell, 1);
            E.cell[at] = (e0 & (STG_NEAR | STG_DEFER)) | local | ((cell + 1) << STG_SHIFT);
        } else {
            atomicSub(E.cta_cnt + u / (CTA_R / 32), 1);
        }
        E.rval[ray] = v;
        // the thread that finishes a pixel's last deferred ray completes the pixel:
        // the render's partial sum plus the deferred values in sub-ray order, / s^2
        __threadfence();
        if (atomicSub(E.pcnt + pixel, 1) == 1) {
            const unsigned long long mask = E.pdef[pixel];
            float val = img[pixel];
            // the deferred values' loads issued 16 at a time, then added in order
            const float* rv = E.rval + (size_t)pixel * s2;
            for (int q0 = 0; q0 < s2; q0 += 16) {
                float r[16];
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    r[u] = (q0 + u < s2 && (mask >> (q0 + u) & 1ull)) ? __ldcg(rv + q0 + u) : 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (q0 + u < s2 && (mask >> (q0 + u) & 1ull)) val += r[u];
            }
            val = val / (float)s2;
            img[pixel] = val;
            if (E.image_out) reinterpret_cast<float*>(E.image_out)[pixel] = val;
        }
    }
}

// in-place exclusive scans of a[0..n) and b[0..n) by one CTA of SCAN_NT threads
// (both in one pass), totals in a[n] and b[n]; wtot holds 2 x SCAN_NT/32 ints
constexpr int SCAN_NT = 256;
__device__ __forceinline__ void block_exclusive_scan2(int* a, int* b, int n, int* wtot) {
    const int tid = threadIdx.x;
    const int per = (n + SCAN_NT - 1) / SCAN_NT;
    int own_a = 0, own_b = 0;
    for (int i = 0; i < per; ++i) {
        const int c = tid * per + i;
        if (c < n) { own_a += a[c]; own_b += b[c]; }
    }
    int inc_a = own_a, inc_b = own_b;
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(0xffffffffu, inc_a, o);
        const int yb = __shfl_up_sync(0xffffffffu, inc_b, o);
        if ((tid & 31) >= o) { inc_a += ya; inc_b += yb; }
    }
    if ((tid & 31) == 31) { wtot[tid >> 5] = inc_a; wtot[SCAN_NT / 32 + (tid >> 5)] = inc_b; }
    __syncthreads();
    if (tid < 64) {
        // exclusive scans of the warp totals: warp 0 for a, warp 1 for b
        int* w = wtot + (tid >> 5) * (SCAN_NT / 32);
        const int l = tid & 31;
        const int t = l < SCAN_NT / 32 ? w[l] : 0;
        int x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
        }
        if (l < SCAN_NT / 32) w[l] = x - t;
    }
    __syncthreads();
    int base_a = wtot[tid >> 5] + inc_a - own_a, base_b = wtot[SCAN_NT / 32 + (tid >> 5)] + inc_b - own_b;
    for (int i = 0; i < per; ++i) {
        const int c = tid * per + i;
        if (c < n) {
            const int va = a[c], vb = b[c];
            a[c] = base_a; b[c] = base_b;
            base_a += va; base_b += vb;
        }
    }
    if (tid == SCAN_NT - 1) { a[n] = base_a; b[n] = base_b; }
}

// The render warps' list offsets, one small CTA per evaluation right after the
// render (it fits beside the near-edge pass): the per-render-warp staged and
// near-core counts scanned in place into offsets, totals at the end (the near-edge
// pass changes neither count)
__global__ void __launch_bounds__(SCAN_NT) k_scan_warps(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    __shared__ int wtot[2 * (SCAN_NT / 32)];
    block_exclusive_scan2(E.useg, E.nseg, E.n_cta_r * (CTA_R / 32), wtot);
}

// S11's cell offsets: the exclusive scan of the per-cell ray counts by one CTA of
// SCAN_NT threads, after the near-edge pass (the last counts)
__device__ __forceinline__ void cell_offsets(const EvalArgs& E) {
    __shared__ int wtot[SCAN_NT / 32];
    const int nc = (E.n_src - 1) * (E.n_src - 1);
    const int per = (nc + SCAN_NT - 1) / SCAN_NT;
    const int tid = threadIdx.x;
    int own = 0;
    for (int i = 0; i < per; ++i) {
        int c = tid * per + i;
        if (c < nc) own += E.ccount[c];
    }
    int incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((tid & 31) >= o) incl += y;
    }
    if ((tid & 31) == 31) wtot[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        const int t = tid < SCAN_NT / 32 ? wtot[tid] : 0;
        int x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += y;
        }
        if (tid < SCAN_NT / 32) wtot[tid] = x - t;
    }
    __syncthreads();
    int base = wtot[tid >> 5] + incl - own;
    int* off = E.ccount + nc;              // counts [0, ncell), offsets [ncell, 2 ncell + 1)
    for (int i = 0; i < per; ++i) {
        int c = tid * per + i;
        if (c < nc) { off[c] = base; base += E.ccount[c]; }
    }
    if (tid == SCAN_NT - 1) off[nc] = base;
}

// The adjoint's rays: the staged rays of all render warps in warp order (ray k
// of warp u at useg[u] + its position), i.e. in ray order, gathered into flat
// arrays (ray id; cell, or -2 - cell for a near-core ray of the float path; the ray's
// rank inside its cell, from an atomic on the cell's cursor, zeroed with the counts:
// the counting sort's slot is the cell's offset plus the rank), coalesced.  It runs
// right after the render, beside the near-edge pass: the rays that pass defers
// (STG_DEFER: their cells are decided there) are left to k_compact_deferred.  The
// near-core rays' adjoint positions go to nlist in the same order (warp u's at
// nseg[u] on), for the adjoint's separate double-precision pass; near-core rays are
// always deferred, so their cells come from k_compact_deferred too.
// Up to CMP_CTAS CTAs per evaluation (one wave at c2; one per 64 render warps below
// that, so small systems launch few); each warp takes an equal share of
// consecutive list positions (the rays cluster in the few render tiles the grid's
// reach leaves unculled, so shares by render warp would be uneven) and walks the
// render warps it overlaps: it finds the first with a 32-wide probe of the offsets,
// and the near-core entries before its share in that warp with one strided count;
// the next ones from a window of 32 consecutive offsets held one per lane (a ballot,
// no memory round trip, until the window is used up).  It loads up to CMP_G groups
// of 32 entries before it stores any and keeps their slot atomics in flight together.
constexpr int CMP_NT = 256;
constexpr int CMP_CTAS = 20;
constexpr int CMP_G = 4;
// the largest u in [from, nu) with useg[u] <= pos (useg non-decreasing, useg[from] <= pos),
// by a 32-ary search: the warp's lanes probe 32 evenly spaced offsets of the range
// and keep the segment below the first one past pos (about log_32(nu) rounds)
__device__ __forceinline__ int cmp_find_warp(const int* useg, int nu, int from, int pos) {
    const int lane = threadIdx.x & 31;
    int lo = from, n = nu - from;            // answer in [lo, lo + n)
    while (n > 1) {
        const int step = (n + 31) / 32;
        const int v = lo + lane * step;
        const bool past = lane > 0 && (v >= lo + n || useg[v] > pos);
        const unsigned pm = __ballot_sync(0xffffffffu, past);
        const int k = pm ? __ffs(pm) - 1 : 32;  // probes 0..k-1 are not past pos
        lo += (k - 1) * step;
        n = min(step, n - (k - 1) * step);
    }
    return lo;
}
__global__ void __launch_bounds__(CMP_NT) k_compact(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int ncta = B.tile0[ev + 1] - B.tile0[ev];          // this evaluation's CTAs
    const int lane = threadIdx.x & 31;
    constexpr int NWC = CMP_NT / 32;
    const int nu = E.n_cta_r * (CTA_R / 32);
    if (E.transform == RTU_TRANSFORM_LINEAR) {
        // the unsmoothed eCDF's position gradients, accumulated by k_render_adj
        for (int i = tile * CMP_NT + threadIdx.x; i < 4 * E.n_mask; i += ncta * CMP_NT) E.gk[i] = 0ull;
    }
    const int cap = 32 * E.s * E.s;
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    const int ncell = (E.n_src - 1) * (E.n_src - 1);
    const int s2 = E.s * E.s;
    const float inv_s2 = 1.0f / (float)s2;
    const int total = max(0, min(E.useg[nu], n_rays));
    const int nw = ncta * NWC, w = tile * NWC + (threadIdx.x >> 5);
    const int share = (total + nw - 1) / nw;
    const int lo = min(total, w * share), hi = min(total, lo + share);
    if (lo >= hi) return;
    int u = cmp_find_warp(E.useg, nu, 0, lo);
    // near-core entries of warp u before position lo (lanes count strided entries)
    int nat;
    {
        const int* stg = E.cell + (size_t)u * cap;
        const int i0 = min(lo - E.useg[u], cap);
        int c = 0;
        for (int i0k = 0; i0k < i0; i0k += 32 * 8) {
            int e8[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0k + 32 * k + lane;
                e8[k] = i < i0 ? stg[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) c += (e8[k] & STG_NEAR) ? 1 : 0;
        }
        nat = E.nseg[u] + (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
    }
    // the pixel of each lane of render warp u: a staged entry's ray is the pixel of its
    // lane (one shuffle) times s^2 plus its sub-ray
    auto lane_pixel = [&](int uu) {
        bool valid;
        return render_pixel(E.n_img, uu / (CTA_R / 32), (uu % (CTA_R / 32)) * 32 + lane, valid);
    };
    int pix = lane_pixel(u);
    // the offsets window: lane l holds useg[wb + l] (useg[nu] = the total past the end)
    // and nseg[wb + l]
    int wb, wv, wn;
    auto window_at = [&](int base) {
        wb = base;
        const int idx = min(base + lane, nu);
        wv = E.useg[idx];
        wn = E.nseg[idx];
    };
    window_at(u);
    int pos = lo;
    while (pos < hi) {
        if (u + 1 - wb >= 32) window_at(u);
        if (u + 1 < nu && __shfl_sync(0xffffffffu, wv, u + 1 - wb) <= pos) {
            // the last render warp from u + 1 on whose offset is at most pos
            const int from = u + 1;
            for (;;) {
                const unsigned past = __ballot_sync(0xffffffffu, wb + lane >= from && (wb + lane >= nu || wv > pos));
                if (past) {
                    u = wb + __ffs(past) - 2;
                    break;
                }
                window_at(wb + 32);
            }
            if (u < wb || u + 1 - wb >= 32) window_at(u);   // (the answer may precede a slid window)
            nat = __shfl_sync(0xffffffffu, wn, u - wb);
            pix = lane_pixel(u);
        }
        const int o = __shfl_sync(0xffffffffu, wv, u - wb);
        const int end = min(hi, min(u + 1 < nu ? __shfl_sync(0xffffffffu, wv, u + 1 - wb) : total, o + cap));
        if (end <= pos) break;          // inconsistent offsets: leave the rest unwritten
        const int* stg = E.cell + (size_t)u * cap;
        for (int g0 = pos - o; g0 < end - o; g0 += 32 * CMP_G) {
            const int gend = end - o;
            int ent[CMP_G], cell[CMP_G], slot[CMP_G];
            bool nr[CMP_G];
            unsigned grp[CMP_G];
#pragma unroll
            for (int j = 0; j < CMP_G; ++j) {
                const int i = g0 + 32 * j + lane;
                ent[j] = i < gend ? stg[i] : 0;
            }
            // decode the groups, then their slot atomics (one per group of lanes
            // sharing the cell, slots by lane order inside the group; the order of the
            // records inside a cell is free: the cell sums are exact integer sums), all
            // in flight before any result is used
#pragma unroll
            for (int j = 0; j < CMP_G; ++j) {
                const int i = g0 + 32 * j + lane;
                cell[j] = -1;
                nr[j] = false;
                if (i < gend) {
                    const int e = ent[j];
                    int c = ((e & (STG_NEAR - 1)) >> STG_SHIFT) - 1;
                    cell[j] = c >= ncell || (e & STG_DEFER) ? -1 : c;
                    nr[j] = (e & STG_NEAR) != 0;
                }
                const unsigned act = __ballot_sync(0xffffffffu, cell[j] >= 0);
                grp[j] = cell[j] >= 0 ? __match_any_sync(act, cell[j]) : 0u;
                slot[j] = 0;
                if (cell[j] >= 0 && lane == __ffs(grp[j]) - 1) slot[j] = atomicAdd(E.cursor + cell[j], __popc(grp[j]));
            }
#pragma unroll
            for (int j = 0; j < CMP_G; ++j) {
                const int i = g0 + 32 * j + lane;
                if (g0 + 32 * j >= gend) break;
                const int leader = cell[j] >= 0 ? __ffs(grp[j]) - 1 : lane;
                const int b = __shfl_sync(0xffffffffu, slot[j], leader);
                // the entry's render lane (local / s^2, exact in float: local < 32 s^2)
                const int local = ent[j] & ((1 << STG_SHIFT) - 1);
                const int le = min(31, (int)(((float)local + 0.5f) * inv_s2));
                const int ppix = __shfl_sync(0xffffffffu, pix, le);
                if (i < gend && !(ent[j] & STG_DEFER)) {
                    const int c = cell[j];
                    E.kray[o + i] = c >= 0 ? ppix * s2 + (local - le * s2) : -1;
                    E.kcell[o + i] = c;
                    if (c >= 0) E.krank[o + i] = b + __popc(grp[j] & ((1u << lane) - 1u));
                }
                // every flagged entry keeps its list slot (counted by the render); one
                // that the double pass found outside the grid lists -1
                const unsigned bn = __ballot_sync(0xffffffffu, nr[j]);
                const int at = nat + __popc(bn & ((1u << lane) - 1u));
                if (nr[j] && at >= 0 && at < n_rays) E.nlist[at] = o + i;
                nat += __popc(bn);
            }
        }
        pos = end;
    }
}

// The rays the near-edge pass decided (STG_DEFER), after it: their flat-array
// entries at list position useg[u] + i of staging position u cap + i, from the decided
// entry (ray id, or -1 for a ray that ended outside the grid; cell, or -2 - cell for a
// near-core ray; the rank from the cell's cursor), one thread per deferred ray over
// n_edge CTAs per evaluation; one more CTA computes S11's cell offsets meanwhile.
constexpr int CMPD_NT = SCAN_NT;
__global__ void __launch_bounds__(CMPD_NT) k_compact_deferred(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    if (tile == E.n_edge) {
        cell_offsets(E);
        return;
    }
    const int s2 = E.s * E.s, cap = 32 * s2;
    const int n_rays = E.n_img * E.n_img * s2;
    const int ncell = (E.n_src - 1) * (E.n_src - 1);
    const int nu = E.n_cta_r * (CTA_R / 32);
    const int cnt = min(*E.ecount, n_rays);
    for (int j = tile * CMPD_NT + threadIdx.x; j < cnt; j += E.n_edge * CMPD_NT) {
        const int at = E.elist[j];
        const int u = at / cap, i = at - u * cap;
        if (u < 0 || u >= nu) continue;
        const int e = E.cell[at];
        const int k = E.useg[u] + i;
        if (k < 0 || k >= n_rays) continue;
        int c = ((e & (STG_NEAR - 1)) >> STG_SHIFT) - 1;
        if (c >= ncell) c = -1;
        const bool nr = (e & STG_NEAR) != 0;
        E.kray[k] = c >= 0 ? staged_ray_id(E.n_img, s2, u, e & ((1 << STG_SHIFT) - 1)) : -1;
        E.kcell[k] = nr && c >= 0 ? -2 - c : c;
        if (c >= 0) E.krank[k] = atomicAdd(E.cursor + c, 1);
    }
}

// S9 (image -> source/transform/lens part) over the adjoint's rays (render-warp
// order): every CTA takes one equal chunk of CTA_R x per consecutive rays (per set
// from the device-side ray count), thread t taking rays t, t + CTA_R, ... of it.  Each ray is recomputed (value + the EPL
// series sums) and differentiated analytically; its cell comes from the forward
// pass.  Writes one counting-sorted record per ray and fixed-order per-CTA
// partial sums of the lens, standardisation and spline-knot gradients (for the
// unsmoothed eCDF: exact 128-bit fixed-point sums into the gradients of the sorted
// positions).
// The float path splits the rays in two launches that may run concurrently: the
// main one (NEAR false) in float, leaving out the near-core rays the forward traced
// in double, and a small one (NEAR true, NEAR_CTAS CTAs per evaluation) over those
// rays' list, lens and lens adjoint in double, writing partial rows of its own
// after the main pass's (the double code kept out of the main pass's registers).
template <typename T, bool LIN, bool NEAR>
__global__ void __launch_bounds__(CTA_R, NEAR ? 1 : (sizeof(T) == 4 && !LIN ? 6 : 4)) k_render_adj(const __grid_constant__ Batch B) {
    typedef typename real4_of<T>::type R4;
    typedef typename real2_of<T>::type R2;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int n = E.n_src, K = E.n_nodes + 2, nc = n - 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sgrid = reinterpret_cast<T*>(smem_raw);
    const bool gstaged = grid_staged(n, sizeof(T));
    const T* grid = gstaged ? sgrid : reinterpret_cast<const T*>(E.src);
    const size_t gbytes = grid_smem_bytes(n, sizeof(T));
    // per-warp spline-knot tables [NW][2 axes][2][K]: (hi, lo) pairs of T
    typedef typename real2_of<T>::type TP;
    TP* tab = reinterpret_cast<TP*>(smem_raw + gbytes);
    constexpr int NW = CTA_R / 32;
    __shared__ RenderShared<T> sh;
    __shared__ TP wacc[NW][NACC_FIX];
    __shared__ __align__(8) uint64_t mbar;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if constexpr (NEAR) {
        // a CTA of the near-core pass with no share of the list (the list is short)
        // writes its zero row and leaves before any set-up
        const int nu_ = E.n_cta_r * (CTA_R / 32);
        const int tot_ = max(0, min(E.useg[nu_], E.n_img * E.n_img * E.s * E.s));
        const int cnt_ = max(0, min(E.nseg[nu_], tot_));
        const int per_ = max(1, (cnt_ + E.n_near * CTA_R - 1) / (E.n_near * CTA_R));
        if (tile * CTA_R * per_ >= cnt_) {
            double* o0 = E.apart + E.n_cta_adj + tile;
            const int nc0 = NACC_FIX + 4 * K + 5 * (E.sub_kind ? E.n_sub : 0);
            for (int i = threadIdx.x; i < nc0; i += blockDim.x) o0[(size_t)i * E.n_row_adj] = 0.0;
            return;
        }
    }
    // the source grid's copy runs beside the set-up (or the grid is read from global)
    if (gstaged) stage_begin(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar);
    render_setup<T>(E, sh);
    // the lens in double for the float path's FP64 islands (the near-core pass; the
    // unsmoothed map's positions), loaded by the instantiations that use it
    const LensK<double>* Kdp = nullptr;
    if constexpr (sizeof(T) == 4 && (LIN || NEAR)) {
        __shared__ LensK<double> kd_s;
        load_lensk(kd_s, E.lensk);
        Kdp = &kd_s;
    }
    for (int i = threadIdx.x; i < NW * 4 * K; i += blockDim.x) { tab[i].x = T(0); tab[i].y = T(0); }
    bool staged = true;
    if (gstaged) staged = stage_end(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar, E.flags);
    else __syncthreads();
    // column-major partials: column i of this CTA's row at apart[i * n_row_adj + row];
    // the near-core pass also owns the subhalo columns of its rows (zero: k_sub_adj
    // takes every ray in its own rows)
    double* out = E.apart + (NEAR ? E.n_cta_adj + tile : tile);
    const size_t ostr = (size_t)E.n_row_adj;
    const int ncol = NACC_FIX + 4 * K + (NEAR ? 5 * (E.sub_kind ? E.n_sub : 0) : 0);
    if (!staged) {
        for (int i = threadIdx.x; i < ncol; i += blockDim.x) out[i * ostr] = 0.0;
        return;
    }
    const int s = E.s, s2 = s * s;
    const int nsub = sh.K.nsub;
    const int nu = E.n_cta_r * (CTA_R / 32);
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    const int total = max(0, min(E.useg[nu], n_rays));
    // rays of this pass: all adjoint positions, or the near-core list
    const int count = NEAR ? max(0, min(E.nseg[nu], total)) : total;
    const int nstride = NEAR ? E.n_near : E.n_cta_adj;
    const int ncell = nc * nc;
    const T mux = sh.trs[0], muy = sh.trs[1], isg = T(1) / sh.trs[2];
    const T* Xa[2] = {sh.trs + TR_HDR, sh.trs + TR_HDR + K};
    const T* Da[2] = {sh.trs + TR_HDR + 2 * K, sh.trs + TR_HDR + 3 * K};
    const T nm1 = T(n - 1);
    constexpr bool lin = LIN;
    T lbo[2] = {T(0), T(0)}, lbs[2] = {T(0), T(0)};
    double lbo_d[2] = {0.0, 0.0}, lbs_d[2] = {0.0, 0.0};
    const T linv = lin ? T(1) / T(E.n_mask - 1) : T(0);
    const double linv_d = lin ? 1.0 / (E.n_mask - 1) : 0.0;
    LensK<DF>* kdf = nullptr;
    if constexpr (lin) {
        lin_bins<T>(E, 0, lbo[0], lbs[0]);
        lin_bins<T>(E, 1, lbo[1], lbs[1]);
        lin_bins<double>(E, 0, lbo_d[0], lbs_d[0]);
        lin_bins<double>(E, 1, lbo_d[1], lbs_d[1]);
    }
    if constexpr (sizeof(T) == 4 && (LIN || NEAR)) {
        // the double-float lens (no subhaloes): the unsmoothed map's positions, and
        // the near-core pass's lens and lens adjoint (about 48 bits on the FP32 pipes)
        __shared__ LensK<DF> kdf_s;
        kdf = &kdf_s;
        __syncthreads();
        if (Kdp->nsub == 0) load_lensk(kdf_s, lensk_df_src(E.lensk));
        __syncthreads();
    }
    // the near-core pass in double-float when there are no subhaloes
    const bool near_df = NEAR && kdf != nullptr && Kdp->nsub == 0;
    const int* off = E.ccount + nc * nc;
    R4* rec = reinterpret_cast<R4*>(E.rec);
    R2* gbuf = reinterpret_cast<R2*>(E.gbuf);
    const T* gimg = reinterpret_cast<const T*>(E.gimg);
    // pixel centre x = i pix - c, c = (n_img - 1)/2 pix, in the kernel's type
    const T inv_s2 = T(1) / T(s2);

    T acc[NACC_FIX];
#pragma unroll
    for (int i = 0; i < NACC_FIX; ++i) acc[i] = T(0);
    int cj[2] = {-2, -2};
    T ca[2][4] = {{T(0), T(0), T(0), T(0)}, {T(0), T(0), T(0), T(0)}};
    TP* mytab = tab + wid * 4 * K;

    // merge the running knot partials of the lanes that leave their interval:
    // one fixed-order warp sum per distinct interval among those lanes
    auto flush = [&](int a, bool need) {
        unsigned m = __ballot_sync(0xffffffffu, need);
        while (m) {
            const int key = __shfl_sync(0xffffffffu, cj[a], __ffs(m) - 1);
            const bool in = need && cj[a] == key;
            m &= ~__ballot_sync(0xffffffffu, in);
            const T v0 = in ? ca[a][0] : T(0), v1 = in ? ca[a][1] : T(0);
            const T v2 = in ? ca[a][2] : T(0), v3 = in ? ca[a][3] : T(0);
            // the four warp sums by a transposing butterfly: at xor 16 the lower half
            // keeps (v0, v1) and the upper (v2, v3), at xor 8 each quarter keeps one,
            // then three levels on it -- 6 shuffles instead of 20; lanes 0, 8, 16, 24
            // end with the sums of v0 (X, key), v1 (X, key+1), v2 (d, key), v3 (d, key+1)
            const bool up = lane & 16, h8 = lane & 8;
            T k0 = up ? v2 : v0, k1 = up ? v3 : v1;
            k0 += __shfl_xor_sync(0xffffffffu, up ? v0 : v2, 16);
            k1 += __shfl_xor_sync(0xffffffffu, up ? v1 : v3, 16);
            T kk = h8 ? k1 : k0;
            kk += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
            if ((lane & 7) == 0) {
                const int c = lane >> 3;
                const int at = key + (c & 1);
                if (at >= 0 && at <= K - 1) pair_add(mytab[(c >= 2 ? 2 * K : 0) + a * K + at], kk);
            }
        }
        __syncwarp();
        if (need) { ca[a][0] = ca[a][1] = ca[a][2] = ca[a][3] = T(0); }
    };

    // an equal share of the pass's rays per CTA: per rays per thread, CTA_R apart
    const int per = max(1, (count + nstride * CTA_R - 1) / (nstride * CTA_R));
    const int chunk = CTA_R * per;
    for (int base = tile * chunk; base < count; base += nstride * chunk) {
        for (int r = 0; r < per; ++r) {
            // coalesced: the CTA's threads take consecutive rays; a thread's rays
            // are CTA_R apart, i.e. from nearby pixels (mostly the same intervals)
            const int idx = base + r * CTA_R + threadIdx.x;
            int k = idx;
            if constexpr (NEAR) k = idx < count ? E.nlist[idx] : total;
            int jn[2] = {cj[0], cj[1]};
            T pn[2][4];
            bool have = false;
            int cell = -1, ray = 0, slot = -1;
            bool other = false;      // a near-core ray in the main pass: the near pass takes it
            if (k >= 0 && k < total) {
                ray = E.kray[k];
                const int kc = E.kcell[k];
                if constexpr (NEAR) {
                    cell = kc <= -2 ? -2 - kc : -1;
                } else {
                    cell = kc;
                    other = kc <= -2;
                }
                if (cell >= ncell || ray < 0 || ray >= n_rays) cell = -1;
            }
            // the ray's record slot in the counting sort by cell (rank from the compaction)
            if (cell >= 0) slot = off[cell] + E.krank[k];
            T gb0 = T(0), gb1 = T(0);
            if (cell >= 0) {
                const int pixel = (int)udiv((uint32_t)ray, sh.dv_s2), q = ray - pixel * s2;
                const int pj = (int)udiv((uint32_t)pixel, sh.dv_n), pi = pixel - pj * E.n_img;
                const int qb = (int)udiv((uint32_t)q, sh.dv_s), qa = q - qb * s;
                const T x = ray_coord(sh.G, pi, qa);
                const T y = ray_coord(sh.G, pj, qb);
                const T gpix = gimg[pixel] * inv_s2;
                constexpr bool near = NEAR;
                EplJ<T> J;
                EplJ<double> Jd;
                EplJ<DF> Jf;
                double xd = 0.0, yd = 0.0;
                T bx, by;
                double bxd = 0.0, byd = 0.0;
                if (near) {
                    ray_pos(E.n_img, E.pix, s, pixel, q, xd, yd);
                    if (near_df) {
                        DF bxf, byf;
                        lens_beta_eval_smooth(*kdf, DF(xd), DF(yd), Jf, bxf, byf);
                        bxd = bxf.to_double();
                        byd = byf.to_double();
                    } else {
                        lens_beta_eval(*Kdp, xd, yd, Jd, bxd, byd);
                    }
                    bx = (T)bxd;
                    by = (T)byd;
                } else {
                    lens_beta_eval(sh.K, x, y, J, bx, by);
                }
                const T z[2] = {(bx - mux) * isg, (by - muy) * isg};
                T yv[2], dz[2];
                int ks[2] = {0, 0};
                double pk[2][2] = {{0.0, 0.0}, {0.0, 0.0}};     // unsmoothed eCDF: segment partials
                if constexpr (lin && sizeof(T) == 4) {
                    // The split of the ray's gradient between the two observations of its
                    // segment, t = (beta - x_k)/(x_{k+1} - x_k), needs beta far below the
                    // narrowest segment widths (1e-9 arcsec occur): the position in
                    // double-float (double with subhaloes), the segment in double.
                    if (!near) {
                        ray_pos(E.n_img, E.pix, s, pixel, q, xd, yd);
                        if (nsub) {
                            lens_beta(*Kdp, xd, yd, bxd, byd);
                        } else {
                            DF bxf, byf;
                            lens_beta_smooth<DF>(*kdf, DF(xd), DF(yd), bxf, byf);
                            bxd = bxf.to_double();
                            byd = byf.to_double();
                        }
                    }
                    const double bd[2] = {bxd, byd};
                    for (int a = 0; a < 2; ++a) {
                        double dub;
                        yv[a] = (T)lin_value<double>(E, a, bd[a], lbo_d[a], lbs_d[a], linv_d, ks[a], &dub, &pk[a][0],
                                                     &pk[a][1]);
                        dz[a] = (T)dub;
                        pn[a][0] = pn[a][1] = pn[a][2] = pn[a][3] = T(0);
                    }
                } else if constexpr (lin) {
                    for (int a = 0; a < 2; ++a) {
                        yv[a] = lin_value<T>(E, a, z[a], lbo[a], lbs[a], linv, ks[a], &dz[a], &pn[a][0], &pn[a][1]);
                        pk[a][0] = (double)pn[a][0];
                        pk[a][1] = (double)pn[a][1];
                        pn[a][2] = pn[a][3] = T(0);
                    }
                } else {
                    for (int a = 0; a < 2; ++a) {
                        jn[a] = cdf_interval_lut<T>(Xa[a], K, z[a], sh.iv[a], sh.ivo[a], sh.ivs[a]);
                        yv[a] = cdf_grad<T>(Xa[a], sh.U, Da[a], sh.ih + a * K, K, jn[a], z[a], dz[a], pn[a][0], pn[a][1],
                                            pn[a][2], pn[a][3]);
                    }
                }
                const int j0 = (int)udiv((uint32_t)cell, sh.dv_nc), i0 = cell - j0 * nc;
                const T fx = yv[0] * nm1 - T(i0), fy = yv[1] * nm1 - T(j0);
                const T* r0 = grid + j0 * n + i0;
                const T dsdx = nm1 * ((T(1) - fy) * (r0[1] - r0[0]) + fy * (r0[n + 1] - r0[n]));
                const T dsdy = nm1 * ((T(1) - fx) * (r0[n] - r0[0]) + fx * (r0[n + 1] - r0[1]));
                const T gy[2] = {gpix * dsdx, gpix * dsdy};
                const T gz0 = gy[0] * dz[0], gz1 = gy[1] * dz[1];
                gb0 = gz0 * isg;
                gb1 = gz1 * isg;
                acc[8] -= gb0;
                acc[9] -= gb1;
                acc[10] -= (gz0 * z[0] + gz1 * z[1]) * isg;
                if (near) {
                    double o8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (near_df) {
                        const DF zero(0.0f, 0.0f);
                        DF o8f[8] = {zero, zero, zero, zero, zero, zero, zero, zero};
                        lens_beta_vjp(*kdf, Jf, DF(xd), DF(yd), DF((double)gb0), DF((double)gb1), o8f);
#pragma unroll
                        for (int p = 0; p < 8; ++p) o8[p] = o8f[p].to_double();
                    } else {
                        lens_beta_vjp(*Kdp, Jd, xd, yd, (double)gb0, (double)gb1, o8);
                    }
#pragma unroll
                    for (int p = 0; p < 8; ++p) acc[p] += (T)o8[p];
                } else {
                    lens_beta_vjp(sh.K, J, x, y, gb0, gb1, acc);
                }
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 4; ++c) pn[a][c] *= gy[a];
                if constexpr (lin) {
                    // the two observations of the ray's segment, per axis: exact
                    // fixed-point sums into d logL / d (sorted position), the same bits
                    // whatever the order of the rays
                    for (int a = 0; a < 2; ++a) {
                        const double ga = (double)gy[a];
                        if (ga == 0.0 || (pk[a][0] == 0.0 && pk[a][1] == 0.0)) continue;
                        unsigned long long* g = E.gk + 2 * ((size_t)a * E.n_mask + ks[a]);
                        fix128_add(g, ga * pk[a][0], E.flags);
                        fix128_add(g + 2, ga * pk[a][1], E.flags);
                    }
                }
                have = !lin;
                if (slot >= off[cell] && slot < off[cell + 1]) {
                    R4 rr;
                    rr.x = fx; rr.y = fy; rr.z = gpix; rr.w = T(0);
                    rec[slot] = rr;
                }
            }
            if (nsub && k >= 0 && k < total && !other) {
                R2 g;
                g.x = gb0; g.y = gb1;
                gbuf[k] = g;
            }
            for (int a = 0; a < 2; ++a) {
                const bool need = have && jn[a] != cj[a] && cj[a] != -2;
                flush(a, need);
                if (have) {
                    cj[a] = jn[a];
                    for (int c = 0; c < 4; ++c) ca[a][c] += pn[a][c];
                }
            }
        }
    }
    for (int a = 0; a < 2; ++a) flush(a, cj[a] != -2);
    // fixed-order reductions: warp tree -> per-warp slots -> warps in order
#pragma unroll
    for (int i = 0; i < NACC_FIX; ++i) {
        const TP v = warp_pair_sum(acc[i]);
        if (lane == 0) wacc[wid][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
        TP r;
        r.x = T(0); r.y = T(0);
        if (i < NACC_FIX) {
            for (int w = 0; w < NW; ++w) pair_add(r, wacc[w][i]);
        } else if (i < NACC_FIX + 4 * K) {
            const int kk = i - NACC_FIX;    // [0, 2K) knots X (axis-major), [2K, 4K) slopes d
            for (int w = 0; w < NW; ++w) pair_add(r, tab[w * 4 * K + kk]);
        }
        out[i * ostr] = (double)r.x + (double)r.y;
    }
}

constexpr int SUB_GROUP = 2;
// subhalo parameters: d logL / d(kappa_s, r_s, tau, x_s, y_s) over the compacted rays
// with the stored d logL / d beta, same CTA tiling (and partial rows) as k_render_adj
template <typename T>
__global__ void __launch_bounds__(CTA_R) k_sub_adj(const __grid_constant__ Batch B) {
    typedef typename real2_of<T>::type R2;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LensK<T> K;
    __shared__ PixGeom<T> G;
    __shared__ double wsub[CTA_R / 32][5];
    load_lensk(K, lensk_src<T>(E.lensk));
    pixgeom_setup<T>(G, E.pix, E.n_img, E.s);
    __syncthreads();
    const int Kn = E.n_nodes + 2;
    double* out = E.apart + tile;           // column-major, as k_render_adj
    const size_t ostr = (size_t)E.n_row_adj;
    const int nu = E.n_cta_r * (CTA_R / 32);
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    const int total = max(0, min(E.useg[nu], n_rays));
    const int s = E.s, s2 = s * s;
    const R2* gbuf = reinterpret_cast<const R2*>(E.gbuf);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int chunk = CTA_R * ADJ_RPT;
    // SUB_GROUP subhaloes per pass over the ray list: each ray is read and placed once per
    // group; every subhalo's sums still take the thread's rays in list order (the same
    // bits as one pass per subhalo)
    for (int h0 = 0; h0 < K.nsub; h0 += SUB_GROUP) {
        const int hn = min(SUB_GROUP, K.nsub - h0);
        T a5[SUB_GROUP][5];
#pragma unroll
        for (int j = 0; j < SUB_GROUP; ++j)
#pragma unroll
            for (int c = 0; c < 5; ++c) a5[j][c] = T(0);
        for (int base = tile * chunk; base < total; base += E.n_cta_adj * chunk) {
            for (int r = 0; r < ADJ_RPT; ++r) {
                const int k = base + r * CTA_R + threadIdx.x;
                if (k >= total) continue;
                const R2 g = gbuf[k];
                if (g.x == T(0) && g.y == T(0)) continue;
                const int ray = E.kray[k];
                if (ray < 0 || ray >= n_rays) continue;
                const int pixel = ray / s2, q = ray - pixel * s2;
                const int pj = pixel / E.n_img, pi = pixel - pj * E.n_img;
                const T x = ray_coord(G, pi, q % s);
                const T y = ray_coord(G, pj, q / s);
#pragma unroll
                for (int j = 0; j < SUB_GROUP; ++j)
                    if (j < hn) sub_vjp<T>(K, h0 + j, x, y, g.x, g.y, a5[j]);
            }
        }
        for (int j = 0; j < hn; ++j) {
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const double v = warp_sum_lane0(a5[j][c]);
                if (lane == 0) wsub[wid][c] = v;
            }
            __syncthreads();
            if (threadIdx.x < 5) {
                double r = 0.0;
                for (int w = 0; w < CTA_R / 32; ++w) r += wsub[w][threadIdx.x];
                out[(NACC_FIX + 4 * Kn + 5 * (h0 + j) + threadIdx.x) * ostr] = r;
            }
            __syncthreads();
        }
    }
}

// Per-cell bilinear corner sums over the counting-sorted records: one half-warp per
// cell (two cells' loads in flight per warp).  The records of a cell arrive in an
// order that depends on atomic timing, so the sums are formed order-independently:
// every term is rounded to an integer multiple of a quantum fixed per evaluation
// (from the largest |g| of its records, bounded by the largest |d L / d image|, a
// maximum the PSF adjoint takes with integer atomics) and the integers are added
// exactly in 64 bits.  Float path: the
// quantum is 2^-22 of that largest |g| -- the product's own rounding is 2^-24 of the
// term -- and a term is rounded by one fused multiply-add into the integer-valued range
// of a float (1.5 2^23 + v, |v| < 2^22); double path: 2^-(62 - bits(ray count)) of it,
// by a conversion to 64-bit integer.  The result is the same bits from run to run and
// alone or in a batch.
constexpr int GATHER_NT = 256;
__device__ __forceinline__ float pow2_of(int S, float) { return __int_as_float((min(max(S, -126), 127) + 127) << 23); }
__device__ __forceinline__ double pow2_of(int S, double) {
    return __longlong_as_double((long long)(min(max(S, -1022), 1023) + 1023) << 52);
}
// the evaluation's quantum exponent S (terms times 2^S are integers after rounding),
// from the largest |d L / d image| that the PSF adjoint noted, times 1/s^2 as the
// render adjoint forms its records' g (the same rounded product: no record exceeds it)
__device__ __forceinline__ int gather_scale(const EvalArgs& E, float) {
    const float gm = __uint_as_float(*reinterpret_cast<const unsigned int*>(E.gmax)) * (1.0f / (float)(E.s * E.s));
    const int e = max(((__float_as_int(gm) >> 23) & 0xff) - 126, -100);   // every |g| < 2^e
    return 22 - e;
}
__device__ __forceinline__ int gather_scale(const EvalArgs& E, double) {
    const double gm = __longlong_as_double((long long)*E.gmax) * (1.0 / (double)(E.s * E.s));
    const int e = max((int)((__double_as_longlong(gm) >> 52) & 0x7ff) - 1022, -1000);
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    return 62 - e - (32 - __clz(n_rays));
}
// w g 2^S rounded to the nearest integer (g already scaled by 2^S)
__device__ __forceinline__ long long fix_term(float w, float gs) {
    return (long long)(__float_as_int(__fmaf_rn(w, gs, 12582912.0f)) - 0x4B400000);
}
// (the 32-bit accumulation below casts this back to int: exact, |value| < 2^22)
__device__ __forceinline__ long long fix_term(double w, double gs) { return __double2ll_rn(w * gs); }
// The float path's integer sum as a (hi, lo) float pair on the FP32 pipe: its terms
// are below 2^22 and a cell holds fewer than 2^26 rays, so |k| < 2^48 and
// k = a 2^24 + b with a, b exact in float; an exact two-sum of a 2^24 and b gives
// hi = k rounded to float and lo = the rest, both scaled by the power of two 2^-S.
// (A conversion through double would cost an FP64 instruction per step, and the
// SM's FP64 pipe takes one warp instruction at a time whatever the active lanes.)
__device__ __forceinline__ float2 fix_to_pair(long long k, int S, float) {
    const float fa = (float)(int)(k >> 24) * 16777216.0f;      // exact
    const float fb = (float)(int)(k & 0xffffff);              // exact
    float hi, lo;
    df_two_sum(fa, fb, hi, lo);
    const float p = pow2_of(-S, 0.0f);
    return make_float2(hi * p, lo * p);
}
__device__ __forceinline__ double2 fix_to_pair(long long k, int S, double) {
    return make_double2((double)k * pow2_of(-S, 0.0), 0.0);
}
template <typename T>
__global__ void __launch_bounds__(GATHER_NT) k_cell_gather(const __grid_constant__ Batch B) {
    typedef typename real4_of<T>::type R4;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int nc = E.n_src - 1, ncell = nc * nc;
    const int cell = tile * (GATHER_NT / 16) + (threadIdx.x >> 4);
    const int hl = threadIdx.x & 15;
    const bool valid = cell < ncell;
    const int* off = E.ccount + ncell;
    const R4* rec = reinterpret_cast<const R4*>(E.rec);
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    const int lo = valid ? max(0, off[cell]) : 0, hi = valid ? min(off[cell + 1], n_rays) : 0;
    const int S = gather_scale(E, T(0));
    const T sc = pow2_of(S, T(0));
    long long l0 = 0, l1 = 0, l2 = 0, l3 = 0;
    auto terms = [&](const R4& r, long long& t0, long long& t1, long long& t2, long long& t3) {
        const T fx = r.x, fy = r.y, gs = r.z * sc;      // exact: a power of two
        const T w0 = (T(1) - fx) * (T(1) - fy), w1 = fx * (T(1) - fy);
        const T w2 = (T(1) - fx) * fy, w3 = fx * fy;
        t0 = fix_term(w0, gs);
        t1 = fix_term(w1, gs);
        t2 = fix_term(w2, gs);
        t3 = fix_term(w3, gs);
    };
    if (sizeof(T) == 4 && hi - lo <= 16 * 511) {
        // float terms are below 2^22: a lane's at most 511 of them sum exactly in 32 bits
        int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int i = lo + hl; i < hi; i += 16) {
            long long t0, t1, t2, t3;
            terms(rec[i], t0, t1, t2, t3);
            a0 += (int)t0; a1 += (int)t1; a2 += (int)t2; a3 += (int)t3;
        }
        l0 = a0; l1 = a1; l2 = a2; l3 = a3;
    } else {
        for (int i = lo + hl; i < hi; i += 16) {
            long long t0, t1, t2, t3;
            terms(rec[i], t0, t1, t2, t3);
            l0 += t0; l1 += t1; l2 += t2; l3 += t3;
        }
    }
    // the half-warp's four sums by a transposing butterfly: at xor 8 the lower eight
    // lanes keep corners 0, 1 and the upper eight 2, 3, at xor 4 each quarter keeps one
    // corner, then two levels on it; lanes 0, 4, 8, 12 of the half hold corners 0..3
    const bool up = hl & 8;
    long long k0 = up ? l2 : l0, k1 = up ? l3 : l1;
    k0 += __shfl_xor_sync(0xffffffffu, up ? l0 : l2, 8);
    k1 += __shfl_xor_sync(0xffffffffu, up ? l1 : l3, 8);
    const bool hi4 = hl & 4;
    long long k = hi4 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, hi4 ? k0 : k1, 4);
    for (int o = 2; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    typedef typename real2_of<T>::type TP;
    if (valid && (hl & 3) == 0) reinterpret_cast<TP*>(E.corner)[(size_t)cell * 4 + (hl >> 2)] = fix_to_pair(k, S, T(0));
}

}  // namespace rtu
