// k_light.cuh -- adjoint of the MGE lens light (App. A.3): d log L / d (A, sigma,
// q, phi, x_n, y_n) of every component, one thread per image pixel over its
// sub-rays (the forward adds the light inside the render kernel), fixed-order sums.
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

// L = A/(2 pi) exp(-E), E = (q x'^2 + y'^2/q)/(2 sigma^2):
//   dL/dA = L/A,  dL/dsigma = 2 E L/sigma,  dL/dq = -L (x'^2 - y'^2/q^2)/(2 sigma^2),
//   dL/dphi = -L x' y' (q - 1/q)/sigma^2,
//   dL/dx_n = L (q x' cos phi - y' sin phi / q)/sigma^2,
//   dL/dy_n = L (q x' sin phi + y' cos phi / q)/sigma^2
template <typename T>
__global__ void __launch_bounds__(CTA_R) k_light_adj(const __grid_constant__ Batch B) {
    typedef typename real2_of<T>::type TP;
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LightK<T> L;
    __shared__ PixGeom<T> G;
    __shared__ TP wred[CTA_R / 32][6 * MAX_LIGHT];
    light_setup<T>(L, E.light, E.n_light);
    pixgeom_setup<T>(G, E.pix, E.n_img, E.s);
    __syncthreads();
    const int nl = L.n;
    if (nl == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s = E.s, s2 = s * s;
    bool valid;
    const int pixel = render_pixel(E.n_img, tile, threadIdx.x, valid);
    T acc[6 * MAX_LIGHT];
#pragma unroll
    for (int k = 0; k < 6 * MAX_LIGHT; ++k) acc[k] = T(0);
    if (valid) {
        const T g = reinterpret_cast<const T*>(E.gimg)[pixel] / T(s2);
        const int pj = pixel / E.n_img, pi = pixel - pj * E.n_img;
        for (int q = 0; q < s2; ++q) {
            const T x = ray_coord(G, pi, q % s), y = ray_coord(G, pj, q / s);
#pragma unroll
            for (int n = 0; n < MAX_LIGHT; ++n) {
                if (n < nl) {
                    const T* c = L.c[n];
                    const T dx = x - c[6], dy = y - c[7];
                    const T xp = c[4] * dx + c[5] * dy, yp = c[4] * dy - c[5] * dx;
                    const T Ex = c[1] * (c[2] * xp * xp + c[3] * yp * yp);
                    const T gl = g * c[0] * r_exp(-Ex);          // g L
                    const T k2 = T(2) * c[1];                     // 1/sigma^2
                    acc[6 * n + 0] += gl * c[8];
                    acc[6 * n + 1] += gl * T(2) * Ex * c[9];
                    acc[6 * n + 2] -= gl * c[1] * (xp * xp - yp * yp * c[3] * c[3]);
                    acc[6 * n + 3] -= gl * k2 * xp * yp * (c[2] - c[3]);
                    acc[6 * n + 4] += gl * k2 * (c[2] * xp * c[4] - yp * c[5] * c[3]);
                    acc[6 * n + 5] += gl * k2 * (c[2] * xp * c[5] + yp * c[4] * c[3]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 6 * MAX_LIGHT; ++k) {
        if (k < 6 * nl) {
            const TP v = warp_pair_sum(acc[k]);
            if (lane == 0) wred[wid][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 6 * nl; k += blockDim.x) {
        TP r;
        r.x = T(0); r.y = T(0);
        for (int w = 0; w < CTA_R / 32; ++w) pair_add(r, wred[w][k]);
        E.lpartl[(size_t)tile * 6 * nl + k] = (double)r.x + (double)r.y;
    }
}

}  // namespace rtu
