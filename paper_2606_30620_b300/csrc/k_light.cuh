// k_light.cuh -- the MGE lens light (App. A.3): the forward adds the supersample mean
// of the light to the unconvolved image; in the adjoint every component's six weighted moments of
// its sub-ray offsets (dx, dy) from the centre are summed,
//   M = sum w, (sum w dx, sum w dy), (sum w dx^2, sum w dx dy, sum w dy^2),
//   w = (d log L / d image) / s^2 * L_n(sub-ray),
// and k_grad_final maps them to d log L / d (A, sigma, q, phi, x_n, y_n): every
// partial of L_n is L_n times a polynomial of degree <= 2 in (dx, dy).
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

// The forward: one thread per pixel adds the supersample mean of the light to the
// unconvolved image the render kernel wrote (after the near-edge pass), before the PSF.
constexpr int LIGHT_FWD_NT = 256;
constexpr int LIGHT_MAXS = 8;          // the largest supersampling factor s

// the s sub-ray coordinates of pixel index i along one axis (registers; s <= 8)
template <typename T>
__device__ __forceinline__ void subray_coords(const PixGeom<T>& G, int i, int s, T* c) {
    const T hi = G.hi, lo = G.lo, e0 = T(i) - G.ci;
#pragma unroll
    for (int q = 0; q < LIGHT_MAXS; ++q) {
        const T e = e0 + G.offp[q < s ? q : 0];
        c[q] = fma(e, hi, e * lo);
    }
}

template <typename T>
__global__ void __launch_bounds__(LIGHT_FWD_NT) k_light_fwd(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LightK<T> L;
    __shared__ PixGeom<T> G;
    light_setup<T>(L, E.light, E.n_light);
    pixgeom_setup<T>(G, E.pix, E.n_img, E.s);
    __syncthreads();
    const int npix = E.n_img * E.n_img, s = E.s;
    const int pixel = tile * LIGHT_FWD_NT + threadIdx.x;
    if (L.n == 0 || pixel >= npix) return;
    const int pj = pixel / E.n_img, pi = pixel - pj * E.n_img;
    T xs[LIGHT_MAXS], ys[LIGHT_MAXS];
    subray_coords(G, pi, s, xs);
    subray_coords(G, pj, s, ys);
    T v = T(0);
    for (int n = 0; n < L.n; ++n) {
        const T xn = L.xn[n], yn = L.yn[n], a = L.e2a[n], b = L.e2b[n], c = L.e2c[n];
        T vn = T(0);
#pragma unroll
        for (int qb = 0; qb < LIGHT_MAXS; ++qb) {
            if (qb >= s) break;
            const T dy = ys[qb] - yn;
            const T cy = c * dy * dy, by = b * dy;
#pragma unroll
            for (int qa = 0; qa < LIGHT_MAXS; ++qa) {
                if (qa >= s) break;
                const T dx = xs[qa] - xn;
                vn += r_exp2(-(dx * (a * dx + by) + cy));
            }
        }
        v += L.amp[n] * vn;
    }
    T* img = reinterpret_cast<T*>(E.img);
    const T val = img[pixel] + v / T(s * s);
    img[pixel] = val;
    if (E.image_out) reinterpret_cast<T*>(E.image_out)[pixel] = val;
}

// One thread per LIGHT_PPT pixels (CTA_R apart: coalesced), components one after
// the other; per pixel the s^2 sub-rays are summed in T, then added to compensated
// (hi, lo) accumulators, then fixed-order warp and CTA sums.
template <typename T>
__global__ void __launch_bounds__(CTA_R) k_light_adj(const __grid_constant__ Batch B) {
    typedef typename real2_of<T>::type TP;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LightK<T> L;
    __shared__ PixGeom<T> G;
    __shared__ TP wred[CTA_R / 32][6];
    __shared__ UDiv dv_n;
    light_setup<T>(L, E.light, E.n_light);
    pixgeom_setup<T>(G, E.pix, E.n_img, E.s);
    if (threadIdx.x == 0) dv_n = udiv_make((uint32_t)E.n_img);
    __syncthreads();
    const int nl = L.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s = E.s, s2 = s * s, npix = E.n_img * E.n_img;
    const T inv_s2 = T(1) / T(s2);
    const T* gimg = reinterpret_cast<const T*>(E.gimg);
    for (int n = 0; n < nl; ++n) {
        const T xn = L.xn[n], yn = L.yn[n], a = L.e2a[n], b = L.e2b[n], c = L.e2c[n], amp = L.amp[n];
        TP acc[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { acc[k].x = T(0); acc[k].y = T(0); }
        for (int r = 0; r < LIGHT_PPT; ++r) {
            const int pixel = (tile * LIGHT_PPT + r) * CTA_R + threadIdx.x;
            if (pixel >= npix) break;
            const T g = gimg[pixel] * inv_s2;
            const int pj = (int)udiv((uint32_t)pixel, dv_n), pi = pixel - pj * E.n_img;
            T xs[LIGHT_MAXS], ys[LIGHT_MAXS];
            subray_coords(G, pi, s, xs);
            subray_coords(G, pj, s, ys);
            T m[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int qb = 0; qb < LIGHT_MAXS; ++qb) {
                if (qb >= s) break;
                const T dy = ys[qb] - yn;
                const T cy = c * dy * dy, by = b * dy;
#pragma unroll
                for (int qa = 0; qa < LIGHT_MAXS; ++qa) {
                    if (qa >= s) break;
                    const T dx = xs[qa] - xn;
                    const T w = amp * r_exp2(-(dx * (a * dx + by) + cy));
                    const T wx = w * dx, wy = w * dy;
                    m[0] += w;
                    m[1] += wx;
                    m[2] += wy;
                    m[3] += wx * dx;
                    m[4] += wx * dy;
                    m[5] += wy * dy;
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) pair_add(acc[k], g * m[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            TP v = warp_pair_sum(acc[k].x);
            pair_add(v, warp_pair_sum(acc[k].y));
            if (lane == 0) wred[wid][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            TP r;
            r.x = T(0); r.y = T(0);
            for (int w = 0; w < CTA_R / 32; ++w) pair_add(r, wred[w][threadIdx.x]);
            E.lpartl[(size_t)tile * 6 * nl + 6 * n + threadIdx.x] = (double)r.x + (double)r.y;
        }
        __syncthreads();
    }
}

}  // namespace rtu
