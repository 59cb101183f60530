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

// Stage `bytes` from global to shared.  Bulk path: bytes % 16 == 0 and both
// addresses 16-byte aligned; otherwise plain loads.  The wait is bounded: on
// give-up the flag word gets F_TIMEOUT and the caller skips its work.
// Returns false on timeout.  Must be called by all threads of the CTA.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* mbar,
                                              int* flags) {
    const bool bulk = (bytes % 16u == 0u) && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u) &&
                      ((smem_u32(dst) & 15u) == 0u) && bytes > 0u;
    if (!bulk) {
        const unsigned char* s = static_cast<const unsigned char*>(src);
        unsigned char* d = static_cast<unsigned char*>(dst);
        for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) d[i] = s[i];
        __syncthreads();
        return true;
    }
    const uint32_t mb = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(mb)
            : "memory");
    }
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

// value, dC/dz and the partials w.r.t. (X_j, X_{j+1}, d_j, d_{j+1}) of the
// touched knots (for the extrapolation branches only one knot is touched: the
// left branch reports it in slot "j+1" = knot 0, the right in slot "j" = K-1).
template <typename T>
__device__ __forceinline__ T cdf_grad(const T* X, const T* U, const T* d, int K, int j, T z, T& dz,
                                      T& pX0, T& pX1, T& pd0, T& pd1) {
    if (j < 0) {
        dz = d[0]; pX0 = T(0); pd0 = T(0); pX1 = -d[0]; pd1 = z - X[0];
        return U[0] + d[0] * (z - X[0]);
    }
    if (j >= K - 1) {
        dz = d[K - 1]; pX1 = T(0); pd1 = T(0); pX0 = -d[K - 1]; pd0 = z - X[K - 1];
        return U[K - 1] + d[K - 1] * (z - X[K - 1]);
    }
    T h = X[j + 1] - X[j];
    T t = (z - X[j]) / h;
    T t2 = t * t, t3 = t2 * t;
    T h00 = T(2) * t3 - T(3) * t2 + T(1), h10 = t3 - T(2) * t2 + t;
    T h01 = T(-2) * t3 + T(3) * t2, h11 = t3 - t2;
    T h00p = T(6) * t2 - T(6) * t, h10p = T(3) * t2 - T(4) * t + T(1);
    T h01p = T(-6) * t2 + T(6) * t, h11p = T(3) * t2 - T(2) * t;
    T Dz = (h00p * U[j] + h01p * U[j + 1]) / h + h10p * d[j] + h11p * d[j + 1];
    T Hd = h10 * d[j] + h11 * d[j + 1];
    dz = Dz;
    pX0 = Dz * (t - T(1)) - Hd;
    pX1 = -Dz * t + Hd;
    pd0 = h * h10;
    pd1 = h * h11;
    return h00 * U[j] + h10 * h * d[j] + h01 * U[j + 1] + h11 * h * d[j + 1];
}

// transform (mu, sigma, knots, slopes) and node values into shared memory
template <typename T>
__device__ __forceinline__ void load_transform(const EvalArgs& E, T* trs, T* U) {
    const int K = E.n_nodes + 2;
    const int nt = TR_HDR + 4 * K;
    for (int i = threadIdx.x; i < nt; i += blockDim.x)
        trs[i] = sizeof(T) == 4 ? (T)E.trf[i] : (T)E.trd[i];
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double u = j == 0 ? 0.0
                 : (j == K - 1 ? 1.0
                               : (1.0 - cos((2.0 * j - 1.0) * 3.14159265358979323846 / (2.0 * E.n_nodes))) / 2.0);
        U[j] = (T)u;
    }
}

// S7 + S11: one thread per image pixel, s^2 sub-rays each.
// Near-edge FP64 island: a float ray whose grid coordinate lies within
// EDGE_DELTA (in cells) of a cell edge or of the grid boundary is traced again in
// double, so that the integer cell of every ray (the rays-per-cell histogram and
// the kink of the bilinear slope used by the adjoint) is decided in double.
constexpr double EDGE_DELTA = 2e-3;

__device__ __forceinline__ bool near_edge(float gx, float gy, int n) {
    const float lo = -(float)EDGE_DELTA, hi = (float)(n - 1) + (float)EDGE_DELTA;
    if (gx < lo || gx > hi || gy < lo || gy > hi) return false;     // clearly outside
    const float fx = gx - floorf(gx), fy = gy - floorf(gy);
    return fx < (float)EDGE_DELTA || fx > 1.0f - (float)EDGE_DELTA || fy < (float)EDGE_DELTA ||
           fy > 1.0f - (float)EDGE_DELTA;
}

template <typename T>
__global__ void __launch_bounds__(CTA_R) k_render(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sgrid = reinterpret_cast<T*>(smem_raw);
    __shared__ T trs[TR_HDR + 4 * (MAXM + 2)];
    __shared__ T U[MAXM + 2];
    __shared__ double trs_d[sizeof(T) == 4 ? TR_HDR + 4 * (MAXM + 2) : 1];
    __shared__ double U_d[sizeof(T) == 4 ? MAXM + 2 : 1];
    __shared__ LensP L;
    __shared__ __align__(8) uint64_t mbar;
    const int n = E.n_src, K = E.n_nodes + 2;
    if (threadIdx.x == 0) load_lens(L, E.lens, E.sub_kind ? E.n_sub : 0);
    load_transform<T>(E, trs, U);
    if (sizeof(T) == 4) load_transform<double>(E, trs_d, U_d);
    if (!stage_to_smem(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar, E.flags)) return;
    const int npix = E.n_img * E.n_img;
    const int pixel = tile * CTA_R + threadIdx.x;
    if (pixel >= npix) return;
    const T mux = trs[0], muy = trs[1], isg = T(1) / trs[2];
    const T* Xx = trs + TR_HDR;
    const T* Xy = Xx + K;
    const T* dx_ = Xx + 2 * K;
    const T* dy_ = Xx + 3 * K;
    const int s = E.s, s2 = s * s;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const T nm1 = T(n - 1);
    T acc = T(0);
    for (int q = 0; q < s2; ++q) {
        double xd, yd;
        ray_pos(E.n_img, E.pix, s, pixel, q, xd, yd);
        T bx, by;
        trace_value<T>(L, E.profile, nsub, E.sub_kind, xd, yd, bx, by);
        const T zx = (bx - mux) * isg, zy = (by - muy) * isg;
        const T yx = cdf_value<T>(Xx, U, dx_, K, cdf_interval<T>(Xx, K, zx), zx);
        const T yy = cdf_value<T>(Xy, U, dy_, K, cdf_interval<T>(Xy, K, zy), zy);
        if (sizeof(T) == 4 && near_edge((float)(yx * nm1), (float)(yy * nm1), n)) {
            double dbx, dby;
            trace_value_T<double>(L, E.profile, nsub, E.sub_kind, xd, yd, dbx, dby);
            const double* Xd = trs_d + TR_HDR;
            const double dzx = (dbx - trs_d[0]) / trs_d[2], dzy = (dby - trs_d[1]) / trs_d[2];
            const double gxd = (double)cdf_value<double>(Xd, U_d, Xd + 2 * K, K, cdf_interval<double>(Xd, K, dzx), dzx);
            const double gyd = (double)cdf_value<double>(Xd + K, U_d, Xd + 3 * K, K, cdf_interval<double>(Xd + K, K, dzy), dzy);
            int cellx = -1;
            if (gxd >= 0.0 && gxd <= 1.0 && gyd >= 0.0 && gyd <= 1.0) {
                int i0 = (int)(gxd * (n - 1)), j0 = (int)(gyd * (n - 1));
                i0 = i0 > n - 2 ? n - 2 : i0;
                j0 = j0 > n - 2 ? n - 2 : j0;
                const T fx = (T)(gxd * (n - 1) - i0), fy = (T)(gyd * (n - 1) - j0);
                const T* r0 = sgrid + j0 * n + i0;
                acc += (T(1) - fx) * (T(1) - fy) * r0[0] + fx * (T(1) - fy) * r0[1] +
                       (T(1) - fx) * fy * r0[n] + fx * fy * r0[n + 1];
                cellx = j0 * (n - 1) + i0;
                atomicAdd(E.ccount + cellx, 1);
            }
            E.cell[(size_t)pixel * s2 + q] = cellx;
            continue;
        }
        int cell = -1;
        if (yx >= T(0) && yx <= T(1) && yy >= T(0) && yy <= T(1)) {
            const T gx = yx * nm1, gy = yy * nm1;
            int i0 = (int)gx, j0 = (int)gy;
            i0 = i0 > n - 2 ? n - 2 : i0;
            j0 = j0 > n - 2 ? n - 2 : j0;
            const T fx = gx - T(i0), fy = gy - T(j0);
            const T* r0 = sgrid + j0 * n + i0;
            const T v = (T(1) - fx) * (T(1) - fy) * r0[0] + fx * (T(1) - fy) * r0[1] +
                        (T(1) - fx) * fy * r0[n] + fx * fy * r0[n + 1];
            acc += v;
            cell = j0 * (n - 1) + i0;
            atomicAdd(E.ccount + cell, 1);
        }
        E.cell[(size_t)pixel * s2 + q] = cell;
    }
    const T val = acc / T(s2);
    reinterpret_cast<T*>(E.img)[pixel] = val;
    if (E.image_out) reinterpret_cast<T*>(E.image_out)[pixel] = val;
}

// exclusive scan of the per-cell ray counts into offsets; cursors zeroed
constexpr int SCAN_NT = 1024;
__global__ void __launch_bounds__(SCAN_NT) k_scan_cells(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
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
    __shared__ int wtot[SCAN_NT / 32];
    if ((tid & 31) == 31) wtot[tid >> 5] = incl;
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int w = 0; w < SCAN_NT / 32; ++w) { int t = wtot[w]; wtot[w] = acc; acc += t; }
    }
    __syncthreads();
    int base = wtot[tid >> 5] + incl - own;
    int* off = E.ccount + nc;              // counts [0, ncell), offsets [ncell, 2 ncell + 1)
    for (int i = 0; i < per; ++i) {
        int c = tid * per + i;
        if (c < nc) { off[c] = base; base += E.ccount[c]; E.cursor[c] = 0; }
    }
    if (tid == SCAN_NT - 1) off[nc] = base;
}

// S9 (image -> source/transform/lens part).  One thread per pixel, rays
// recomputed with forward-mode derivatives of the main lens.  Writes one
// counting-sorted record per in-grid ray and fixed-order per-CTA partial sums
// of the lens, standardisation and spline-knot gradients.
template <typename T>
__global__ void __launch_bounds__(CTA_R) k_render_adj(const __grid_constant__ Batch B) {
    typedef typename real4_of<T>::type R4;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int n = E.n_src, K = E.n_nodes + 2, nc = n - 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sgrid = reinterpret_cast<T*>(smem_raw);
    const size_t gbytes = ((size_t)n * n * sizeof(T) + 127) & ~(size_t)127;
    double* tab = reinterpret_cast<double*>(smem_raw + gbytes);           // [NW][2 axes][2][K]
    constexpr int NW = CTA_R / 32;
    T* gbs = reinterpret_cast<T*>(tab + NW * 4 * K);                      // [CTA_R][s2][2]
    __shared__ T trs[TR_HDR + 4 * (MAXM + 2)];
    __shared__ T U[MAXM + 2];
    __shared__ LensP L;
    __shared__ double wacc[NW][NACC_FIX];
    __shared__ double wsub[NW][5];
    __shared__ __align__(8) uint64_t mbar;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) load_lens(L, E.lens, E.sub_kind ? E.n_sub : 0);
    load_transform<T>(E, trs, U);
    for (int i = threadIdx.x; i < NW * 4 * K; i += blockDim.x) tab[i] = 0.0;
    const bool staged = stage_to_smem(sgrid, E.src, (uint32_t)(n * n * sizeof(T)), &mbar, E.flags);
    const int nacc = NACC_FIX + 4 * K + 5 * (E.sub_kind ? E.n_sub : 0);
    double* out = E.apart + (size_t)tile * nacc;
    if (!staged) {
        for (int i = threadIdx.x; i < nacc; i += blockDim.x) out[i] = 0.0;
        return;
    }
    const int npix = E.n_img * E.n_img;
    const int pixel = tile * CTA_R + threadIdx.x;
    const bool valid = pixel < npix;
    const int s = E.s, s2 = s * s;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const T mux = trs[0], muy = trs[1], sg = trs[2], isg = T(1) / sg;
    const T* Xa[2] = {trs + TR_HDR, trs + TR_HDR + K};
    const T* Da[2] = {trs + TR_HDR + 2 * K, trs + TR_HDR + 3 * K};
    const T nm1 = T(n - 1);
    const T gpix = valid ? reinterpret_cast<const T*>(E.gimg)[pixel] / T(s2) : T(0);
    const int* off = E.ccount + nc * nc;
    R4* rec = reinterpret_cast<R4*>(E.rec);

    T acc[NACC_FIX];
#pragma unroll
    for (int i = 0; i < NACC_FIX; ++i) acc[i] = T(0);
    int cj[2] = {-2, -2};
    T ca[2][4] = {{T(0), T(0), T(0), T(0)}, {T(0), T(0), T(0), T(0)}};
    double* mytab = tab + wid * 4 * K;

    auto flush = [&](int a, bool need) {
        unsigned m = __ballot_sync(0xffffffffu, need);
        while (m) {
            const int l = __ffs(m) - 1;
            if (lane == l) {
                double* tX = mytab + a * K;
                double* tD = mytab + 2 * K + a * K;
                const int j = cj[a];
                if (j >= 0) { tX[j] += (double)ca[a][0]; tD[j] += (double)ca[a][2]; }
                if (j + 1 <= K - 1) { tX[j + 1] += (double)ca[a][1]; tD[j + 1] += (double)ca[a][3]; }
            }
            __syncwarp();
            m &= m - 1;
        }
        if (need) { ca[a][0] = ca[a][1] = ca[a][2] = ca[a][3] = T(0); }
    };

    for (int q = 0; q < s2; ++q) {
        int cell = -1;
        double xd = 0.0, yd = 0.0;
        T gb0 = T(0), gb1 = T(0);
        int jn[2] = {cj[0], cj[1]};
        T pn[2][4];
        bool have = false;
        if (valid) {
            ray_pos(E.n_img, E.pix, s, pixel, q, xd, yd);
            cell = E.cell[(size_t)pixel * s2 + q];
            if (cell >= nc * nc) cell = -1;     // only a forward pass on this slot writes cells
        }
        if (cell >= 0) {
            Dual<T, 6> bx, by;
            trace_dual<T>(L, E.profile, nsub, E.sub_kind, xd, yd, bx, by);
            const T z[2] = {(bx.v - mux) * isg, (by.v - muy) * isg};
            T y[2], dz[2];
            for (int a = 0; a < 2; ++a) {
                jn[a] = cdf_interval<T>(Xa[a], K, z[a]);
                y[a] = cdf_grad<T>(Xa[a], U, Da[a], K, jn[a], z[a], dz[a], pn[a][0], pn[a][1], pn[a][2],
                                   pn[a][3]);
            }
            const int i0 = cell % nc, j0 = cell / nc;
            const T fx = y[0] * nm1 - T(i0), fy = y[1] * nm1 - T(j0);
            const T* r0 = sgrid + j0 * n + i0;
            const T dsdx = nm1 * ((T(1) - fy) * (r0[1] - r0[0]) + fy * (r0[n + 1] - r0[n]));
            const T dsdy = nm1 * ((T(1) - fx) * (r0[n] - r0[0]) + fx * (r0[n + 1] - r0[1]));
            const T gy[2] = {gpix * dsdx, gpix * dsdy};
            const T gz0 = gy[0] * dz[0], gz1 = gy[1] * dz[1];
            gb0 = gz0 * isg;
            gb1 = gz1 * isg;
            acc[8] -= gb0;
            acc[9] -= gb1;
            acc[10] -= (gz0 * z[0] + gz1 * z[1]) * isg;
#pragma unroll
            for (int p = 0; p < 6; ++p) acc[p] += gb0 * bx.d[p] + gb1 * by.d[p];
            const T xf = T(xd), yf = T(yd);
            acc[6] += -gb0 * xf + gb1 * yf;
            acc[7] += -gb0 * yf - gb1 * xf;
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 4; ++c) pn[a][c] *= gy[a];
            have = true;
            const int slot = off[cell] + atomicAdd(E.cursor + cell, 1);
            if (slot >= 0 && slot < off[cell + 1] && slot < npix * s2) {
                R4 r;
                r.x = fx; r.y = fy; r.z = gpix; r.w = T(0);
                rec[slot] = r;
            }
        }
        for (int a = 0; a < 2; ++a) {
            const bool need = have && jn[a] != cj[a] && cj[a] != -2;
            flush(a, need);
            if (have) {
                cj[a] = jn[a];
                for (int c = 0; c < 4; ++c) ca[a][c] += pn[a][c];
            }
        }
        if (nsub) {
            gbs[(threadIdx.x * s2 + q) * 2] = gb0;
            gbs[(threadIdx.x * s2 + q) * 2 + 1] = gb1;
        }
    }
    for (int a = 0; a < 2; ++a) flush(a, cj[a] != -2);
    // fixed-order reductions: warp tree -> per-warp slots -> warps in order
#pragma unroll
    for (int i = 0; i < NACC_FIX; ++i) {
        double v = (double)acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wacc[wid][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NACC_FIX + 4 * K; i += blockDim.x) {
        double r = 0.0;
        if (i < NACC_FIX) {
            for (int w = 0; w < NW; ++w) r += wacc[w][i];
        } else {
            const int k = i - NACC_FIX;     // [0, 2K) knots X (axis-major), [2K, 4K) slopes d
            for (int w = 0; w < NW; ++w) r += tab[w * 4 * K + k];
        }
        out[i] = r;
    }
    // subhalo parameters: one pass per subhalo over the stored d logL / d beta
    for (int h = 0; h < nsub; ++h) {
        T a5[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (valid) {
            for (int q = 0; q < s2; ++q) {
                const T g0 = gbs[(threadIdx.x * s2 + q) * 2], g1 = gbs[(threadIdx.x * s2 + q) * 2 + 1];
                if (g0 == T(0) && g1 == T(0)) continue;
                double xd, yd;
                ray_pos(E.n_img, E.pix, s, pixel, q, xd, yd);
                Dual<T, 5> ax, ay;
                sub_dual<T>(L, h, E.sub_kind, xd, yd, ax, ay);
#pragma unroll
                for (int c = 0; c < 5; ++c) a5[c] -= g0 * ax.d[c] + g1 * ay.d[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            double v = (double)a5[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) wsub[wid][c] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double r = 0.0;
            for (int w = 0; w < NW; ++w) r += wsub[w][threadIdx.x];
            out[NACC_FIX + 4 * K + 5 * h + threadIdx.x] = r;
        }
        __syncthreads();
    }
}

// per-cell bilinear corner sums over the counting-sorted records: one warp per
// cell, fixed lane-stride order and a fixed warp tree, in double
constexpr int GATHER_NT = 256;
template <typename T>
__global__ void __launch_bounds__(GATHER_NT) k_cell_gather(const __grid_constant__ Batch B) {
    typedef typename real4_of<T>::type R4;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int nc = E.n_src - 1, ncell = nc * nc;
    const int cell = tile * (GATHER_NT / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= ncell) return;
    const int* off = E.ccount + ncell;
    const R4* rec = reinterpret_cast<const R4*>(E.rec);
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    const int n_rays = E.n_img * E.n_img * E.s * E.s;
    const int lo = max(0, off[cell]), hi = min(off[cell + 1], n_rays);
    for (int i = lo + lane; i < hi; i += 32) {
        const R4 r = rec[i];
        const double fx = r.x, fy = r.y, g = r.z;
        c0 += (1.0 - fx) * (1.0 - fy) * g;
        c1 += fx * (1.0 - fy) * g;
        c2 += (1.0 - fx) * fy * g;
        c3 += fx * fy * g;
    }
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(0xffffffffu, c0, o);
        c1 += __shfl_down_sync(0xffffffffu, c1, o);
        c2 += __shfl_down_sync(0xffffffffu, c2, o);
        c3 += __shfl_down_sync(0xffffffffu, c3, o);
    }
    if (lane == 0) {
        double* c = E.corner + (size_t)cell * 4;
        c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3;
    }
}

}  // namespace rtu
