// k_adj.cuh -- S9, transform part: back through the Hermite knots and slopes,
// the monotonicity guard, the Chebyshev fit and the type-7 order statistics to
// the selected centre rays, the mean and sigma_min (App. C i-iv), then through
// the centre-ray trace to the lens; final fixed-order lens-gradient sums.
#pragma once
#include "rtu_internal.cuh"
#include "k_grid.cuh"

namespace rtu {

// tadj layout: [0] dmu_x/N  [1] dmu_y/N  [2] dsigma/(N sigma)  [3] amin
//              [8 + a*2MAXM + t]  d logL / d beta of the ray selected at (axis a, target t)
constexpr int TADJ_SEL = 8;

__global__ void __launch_bounds__(256) k_cdf_adj(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    const int M = E.n_nodes, D = E.degree, K = M + 2, N = E.n_mask;
    const int nacc = NACC_FIX + 4 * K + 5 * (E.sub_kind ? E.n_sub : 0);
    __shared__ double tot[NACC_FIX + 4 * (MAXM + 2)];
    // column sums over the render-adjoint CTAs in fixed order
    for (int col = threadIdx.x; col < NACC_FIX + 4 * K; col += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < E.n_cta_r; ++t) s += E.apart[(size_t)t * nacc + col];
        tot[col] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double* tr = E.trd;
    const double sigma = tr[2];
    double dmu[2] = {tot[8], tot[9]};
    double dsig = tot[10];
    for (int a = 0; a < 2; ++a) {
        const double* Xf = tr + TR_HDR + a * K;          // guarded knots
        const double* Xr = tr + TR_HDR + (6 + a) * K;    // raw knots
        const double* pr = tr + TR_HDR + (4 + a) * K;    // raw p'
        const double* sl = tr + TR_HDR + (2 + a) * K;    // slopes 1/p'
        const double* gX = tot + NACC_FIX + a * K;
        const double* gd = tot + NACC_FIX + 2 * K + a * K;
        double span = Xr[K - 1] - Xr[0];
        const bool span_ok = span > 0.0;
        if (!span_ok) span = fabs(span) + 1e-300;
        const double floor_d = 1e-6 * span;
        double gfl = 0.0;
        double gpr[MAXM + 2], gXr[MAXM + 2], gXf[MAXM + 2];
        for (int j = 0; j < K; ++j) {
            // slope d = 1/p'  ->  d L/d p' = -gd d^2
            const double gp = -gd[j] * sl[j] * sl[j];
            if (pr[j] < floor_d) { gpr[j] = 0.0; gfl += gp; } else gpr[j] = gp;
            gXf[j] = gX[j];
        }
        for (int j = K - 1; j >= 1; --j) {
            if (Xf[j] != Xr[j]) { gXf[j - 1] += gXf[j]; gfl += gXf[j]; gXr[j] = 0.0; }
            else gXr[j] = gXf[j];
        }
        gXr[0] = gXf[0];
        if (span_ok) { gXr[K - 1] += 1e-6 * gfl; gXr[0] -= 1e-6 * gfl; }
        // X(t) = sum c_k T_k(t), p'(u) = 2 sum c_k T_k'(t), t = -1, t_j, +1
        double gc[MAXM];
        for (int k = 0; k <= D; ++k) gc[k] = 0.0;
        for (int j = 0; j < K; ++j) {
            const double t = j == 0 ? -1.0 : (j == K - 1 ? 1.0 : 2.0 * cheb_node(j, M) - 1.0);
            double T0 = 1.0, T1 = t, U0 = 1.0, U1 = 2.0 * t;
            gc[0] += gXr[j];
            if (D >= 1) gc[1] += gXr[j] * t + gpr[j] * 2.0 * 1.0 * U0;
            for (int k = 2; k <= D; ++k) {
                const double T2 = 2.0 * t * T1 - T0;
                gc[k] += gXr[j] * T2 + gpr[j] * 2.0 * k * U1;
                const double U2 = 2.0 * t * U1 - U0;
                T0 = T1; T1 = T2; U0 = U1; U1 = U2;
            }
        }
        // c_k = (2/M) sum_i Q_i T_k(t_i)  (halved for k = 0)
        const double* Q = tr + TR_HDR + 8 * K + 2 * MAXM + a * MAXM;
        for (int i = 0; i < M; ++i) {
            const double ti = 2.0 * cheb_node(i + 1, M) - 1.0;
            double T0 = 1.0, T1 = ti, g = 0.5 * gc[0];
            if (D >= 1) g += gc[1] * ti;
            for (int k = 2; k <= D; ++k) {
                const double T2 = 2.0 * ti * T1 - T0;
                g += gc[k] * T2;
                T0 = T1; T1 = T2;
            }
            const double gQ = g * 2.0 / M;
            // Q_i = z_lo + frac (z_hi - z_lo), z = (beta - mu)/sigma
            const double h = cheb_node(i + 1, M) * (N - 1);
            const double frac = h - floor(h);
            E.tadj[TADJ_SEL + a * 2 * MAXM + 2 * i] = gQ * (1.0 - frac) / sigma;
            E.tadj[TADJ_SEL + a * 2 * MAXM + 2 * i + 1] = gQ * frac / sigma;
            dmu[a] -= gQ / sigma;
            dsig -= gQ * Q[i] / sigma;
        }
    }
    E.tadj[0] = dmu[0] / N;
    E.tadj[1] = dmu[1] / N;
    E.tadj[2] = dsig / (N * sigma);
    E.tadj[3] = tr[3];
}

// centre rays: d logL / d beta_i = selected-rank terms + dmu/N
//   + [a = argmin sigma] dsigma (beta_i,a - mu_a)/(N sigma_min); then the lens
template <typename T>
__global__ void __launch_bounds__(CTA_C) k_centre_adj(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int M = E.n_nodes, N = E.n_mask;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nl = 8 + 5 * nsub;
    __shared__ LensP L;
    __shared__ int sidx[2][2 * MAXM];
    __shared__ double sg[2][2 * MAXM];
    __shared__ double hdr[4], mu[2];
    __shared__ double red[CTA_C / 32][8];
    if (threadIdx.x == 0) load_lens(L, E.lens, nsub);
    for (int i = threadIdx.x; i < 2 * 2 * MAXM; i += blockDim.x) {
        const int a = i / (2 * MAXM), t = i - a * 2 * MAXM;
        const bool on = t < 2 * M;
        sidx[a][t] = on ? E.sel_idx[a * 2 * MAXM + t] : -1;
        sg[a][t] = on ? E.tadj[TADJ_SEL + a * 2 * MAXM + t] : 0.0;
    }
    if (threadIdx.x < 4) hdr[threadIdx.x] = E.tadj[threadIdx.x];
    if (threadIdx.x < 2) mu[threadIdx.x] = E.trd[threadIdx.x];
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    double gb[2] = {0.0, 0.0};
    double xd = 0.0, yd = 0.0;
    if (k < N) {
        const double b[2] = {E.beta[k], E.beta[N + k]};
        const int amin = hdr[3] > 0.5 ? 1 : 0;
        for (int a = 0; a < 2; ++a) {
            double g = hdr[a];
            if (a == amin) g += hdr[2] * (b[a] - mu[a]);
            for (int t = 0; t < 2 * M; ++t)
                if (sidx[a][t] == k) g += sg[a][t];
            gb[a] = g;
        }
        ray_pos(E.n_img, E.pix, 1, E.centre_idx[k], 0, xd, yd);
    }
    T acc[8];
    for (int p = 0; p < 8; ++p) acc[p] = T(0);
    if (k < N) {
        Dual<T, 6> bx, by;
        trace_dual<T>(L, E.profile, nsub, E.sub_kind, xd, yd, bx, by);
        const T g0 = (T)gb[0], g1 = (T)gb[1];
        for (int p = 0; p < 6; ++p) acc[p] = g0 * bx.d[p] + g1 * by.d[p];
        acc[6] = -g0 * T(xd) + g1 * T(yd);
        acc[7] = -g0 * T(yd) - g1 * T(xd);
    }
    double* out = E.cadj + (size_t)tile * nl;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = 0; p < 8; ++p) {
        double v = (double)acc[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double r = 0.0;
        for (int w = 0; w < CTA_C / 32; ++w) r += red[w][threadIdx.x];
        out[threadIdx.x] = r;
    }
    for (int h = 0; h < nsub; ++h) {
        __syncthreads();
        T a5[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (k < N) {
            Dual<T, 5> ax, ay;
            sub_dual<T>(L, h, E.sub_kind, xd, yd, ax, ay);
            for (int c = 0; c < 5; ++c) a5[c] = -((T)gb[0] * ax.d[c] + (T)gb[1] * ay.d[c]);
        }
        for (int c = 0; c < 5; ++c) {
            double v = (double)a5[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[wid][c] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double r = 0.0;
            for (int w = 0; w < CTA_C / 32; ++w) r += red[w][threadIdx.x];
            out[8 + 5 * h + threadIdx.x] = r;
        }
    }
}

// g_lens = (render-adjoint lens sums) + (centre-adjoint lens sums), fixed order
__global__ void __launch_bounds__(64) k_grad_final(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    const int K = E.n_nodes + 2;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nacc = NACC_FIX + 4 * K + 5 * nsub;
    const int nl = 8 + 5 * nsub;
    for (int p = threadIdx.x; p < nl; p += blockDim.x) {
        const int col = p < 8 ? p : NACC_FIX + 4 * K + (p - 8);
        double s = 0.0;
        for (int t = 0; t < E.n_cta_r; ++t) s += E.apart[(size_t)t * nacc + col];
        double c = 0.0;
        for (int t = 0; t < E.n_cta_c; ++t) c += E.cadj[(size_t)t * nl + p];
        double g = s + c;
        if (p == 1 && E.profile == 0) g = 0.0;
        E.g_lens[p] = g;
    }
}

}  // namespace rtu
