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

constexpr int CDF_NT = 1024;
__global__ void __launch_bounds__(CDF_NT) k_cdf_adj(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    const int M = E.n_nodes, D = E.degree, K = M + 2, N = E.n_mask;
    const int nacc = NACC_FIX + 4 * K + 5 * (E.sub_kind ? E.n_sub : 0);
    const int ncol = NACC_FIX + 4 * K;
    __shared__ double tot[NACC_FIX + 4 * (MAXM + 2)];
    __shared__ double gXr[2][MAXM + 2], gpr[2][MAXM + 2], gc[2][MAXM], gQ[2][MAXM];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // column sums over the render-adjoint CTAs: one warp per column, fixed lane
    // stride and a fixed shuffle tree
    for (int col = wid; col < ncol; col += CDF_NT / 32) {
        double s = 0.0;
        for (int t = lane; t < E.n_cta_adj; t += 32) s += E.apart[(size_t)t * nacc + col];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) tot[col] = s;
    }
    __syncthreads();
    const double* tr = E.trd;
    const double sigma = tr[2];
    if (E.transform) {
        // uniform grid: X_j = (lo_a + U_j L - mu_a)/sigma, slopes sigma/L, with
        // lo_a = (min_a + max_a)/2 - L/2 and L the larger range (axis amax)
        if (threadIdx.x == 0) {
            const int amax = tr[5] > 0.5 ? 1 : 0;
            const double L = tr[6];
            double dmu[2] = {tot[8], tot[9]}, dsig = tot[10], dL = 0.0, dc[2] = {0.0, 0.0};
            for (int a = 0; a < 2; ++a) {
                const double* X = tr + TR_HDR + a * K;
                for (int j = 0; j < K; ++j) {
                    const double U = j == 0 ? 0.0 : (j == K - 1 ? 1.0 : E.cheb[cheb_u(M, D) + j - 1]);
                    const double gX = tot[NACC_FIX + a * K + j], gd = tot[NACC_FIX + 2 * K + a * K + j];
                    dc[a] += gX / sigma;
                    dL += gX * (U - 0.5) / sigma - gd * sigma / (L * L);
                    dmu[a] -= gX / sigma;
                    dsig += -gX * X[j] / sigma + gd / L;
                }
            }
            for (int a = 0; a < 2; ++a) {
                double gmin = 0.5 * dc[a], gmax = 0.5 * dc[a];
                if (a == amax) { gmax += dL; gmin -= dL; }
                E.tadj[TADJ_SEL + a * 2 * MAXM + 0] = gmin;
                E.tadj[TADJ_SEL + a * 2 * MAXM + 1] = gmax;
                for (int t = 2; t < 2 * MAXM; ++t) E.tadj[TADJ_SEL + a * 2 * MAXM + t] = 0.0;
            }
            E.tadj[0] = dmu[0] / N;
            E.tadj[1] = dmu[1] / N;
            E.tadj[2] = dsig / (N * sigma);
            E.tadj[3] = tr[3];
        }
        return;
    }
    // back through the guard (sequential in the knots; one thread per axis)
    if (threadIdx.x < 2) {
        const int a = threadIdx.x;
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
        double gXf[MAXM + 2];
        for (int j = 0; j < K; ++j) {
            const double gp = -gd[j] * sl[j] * sl[j];        // slope d = 1/p'
            if (pr[j] < floor_d) { gpr[a][j] = 0.0; gfl += gp; } else gpr[a][j] = gp;
            gXf[j] = gX[j];
        }
        for (int j = K - 1; j >= 1; --j) {
            if (Xf[j] != Xr[j]) { gXf[j - 1] += gXf[j]; gfl += gXf[j]; gXr[a][j] = 0.0; }
            else gXr[a][j] = gXf[j];
        }
        gXr[a][0] = gXf[0];
        if (span_ok) { gXr[a][K - 1] += 1e-6 * gfl; gXr[a][0] -= 1e-6 * gfl; }
    }
    __syncthreads();
    // knots X = V c and slopes p' = dV c  ->  gc = V^T gX + dV^T gp'
    const double* Vt = E.cheb + cheb_V(M, D);
    const double* dVt = E.cheb + cheb_dV(M, D);
    for (int w = threadIdx.x; w < 2 * (D + 1); w += CDF_NT) {
        const int a = w / (D + 1), k = w % (D + 1);
        double g = 0.0;
        for (int j = 0; j < K; ++j) g += Vt[j * (D + 1) + k] * gXr[a][j] + dVt[j * (D + 1) + k] * gpr[a][j];
        gc[a][k] = g;
    }
    __syncthreads();
    // c = C Q  ->  gQ = C^T gc; Q = z_lo + frac (z_hi - z_lo), z = (beta - mu)/sigma
    const double* Ct = E.cheb + cheb_C(M, D);
    for (int w = threadIdx.x; w < 2 * M; w += CDF_NT) {
        const int a = w / M, i = w % M;
        double g = 0.0;
        for (int k = 0; k <= D; ++k) g += Ct[k * M + i] * gc[a][k];
        gQ[a][i] = g;
        const double h = E.cheb[cheb_u(M, D) + i] * (N - 1);
        const double frac = h - floor(h);
        E.tadj[TADJ_SEL + a * 2 * MAXM + 2 * i] = g * (1.0 - frac) / sigma;
        E.tadj[TADJ_SEL + a * 2 * MAXM + 2 * i + 1] = g * frac / sigma;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dmu[2] = {tot[8], tot[9]};
        double dsig = tot[10];
        for (int a = 0; a < 2; ++a) {
            const double* Q = tr + TR_HDR + 8 * K + 2 * MAXM + a * MAXM;
            for (int i = 0; i < M; ++i) {
                dmu[a] -= gQ[a][i] / sigma;
                dsig -= gQ[a][i] * Q[i] / sigma;
            }
        }
        E.tadj[0] = dmu[0] / N;
        E.tadj[1] = dmu[1] / N;
        E.tadj[2] = dsig / (N * sigma);
        E.tadj[3] = tr[3];
    }
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
    __shared__ LensK<T> L;
    __shared__ LensK<double> Ld;
    __shared__ int sidx[2][2 * MAXM];
    __shared__ double sg[2][2 * MAXM];
    __shared__ double hdr[4], mu[2];
    __shared__ double red[CTA_C / 32][8];
    load_lensk(L, lensk_src<T>(E.lensk));
    if (sizeof(T) == 4) load_lensk(Ld, E.lensk);
    for (int i = threadIdx.x; i < 2 * 2 * MAXM; i += blockDim.x) {
        const int a = i / (2 * MAXM), t = i - a * 2 * MAXM;
        const bool on = t < 2 * M && E.sel_idx[a * 2 * MAXM + t] >= 0;
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
        const T x = (T)xd, y = (T)yd;
        if (sizeof(T) == 4 && lens_near_core(L, x, y)) {
            EplJ<double> J;
            double bx, by, o8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            lens_beta_eval(Ld, xd, yd, J, bx, by);
            lens_beta_vjp(Ld, J, xd, yd, gb[0], gb[1], o8);
            for (int p = 0; p < 8; ++p) acc[p] = (T)o8[p];
        } else {
            EplJ<T> J;
            T bx, by;
            lens_beta_eval(L, x, y, J, bx, by);
            lens_beta_vjp(L, J, x, y, (T)gb[0], (T)gb[1], acc);
        }
    }
    double* out = E.cadj + (size_t)tile * nl;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = 0; p < 8; ++p) {
        const double v = warp_sum(acc[p]);
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
        if (k < N) sub_vjp<T>(L, h, (T)xd, (T)yd, (T)gb[0], (T)gb[1], a5);
        for (int c = 0; c < 5; ++c) {
            const double v = warp_sum(a5[c]);
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
        for (int t = 0; t < E.n_cta_adj; ++t) s += E.apart[(size_t)t * nacc + col];
        double c = 0.0;
        for (int t = 0; t < E.n_cta_c; ++t) c += E.cadj[(size_t)t * nl + p];
        double g = s + c;
        if (p == 1 && E.profile == 0) g = 0.0;
        E.g_lens[p] = g;
    }
}

}  // namespace rtu
