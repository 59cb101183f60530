// k_adj.cuh -- S9, transform part: back through the Hermite knots and slopes,
// the monotonicity guard, the Chebyshev fit and the type-7 order statistics to
// the selected centre rays, the mean and sigma_min (App. C i-iv), then through
// the centre-ray trace to the lens; for the unsmoothed eCDF, from the sorted
// positions' gradients to every centre ray; final fixed-order lens-gradient sums.
#pragma once
#include "rtu_internal.cuh"
#include "k_grid.cuh"
#include "k_gp.cuh"

namespace rtu {

// tadj layout: [0] dmu_x/N  [1] dmu_y/N  [3] amin  [4], [5] the x and y parts of
//              dsigma (their sum / (N sigma) multiplies beta - mu on the amin axis)
//              [8 + a*2MAXM + t]  d logL / d beta of the ray selected at (axis a, target t)
constexpr int TADJ_SEL = 8;

// one warp: column sums over the render-adjoint CTAs (the partials are column-major,
// so the lanes read consecutive CTAs), fixed lane stride and a fixed shuffle tree
__device__ __forceinline__ double apart_col(const EvalArgs& E, int col) {
    return warp_rows_sum(E.apart + (size_t)col * E.n_row_adj, E.n_row_adj, 1);
}

// the selected-rank lens terms of axis a: sum over targets t of tadj[sel a t] jsel[a
// t], into row n_cta_c + a of cadj; one warp per lens parameter, lanes over the targets
// (fixed lane stride and shuffle tree)
__device__ __forceinline__ void sel_terms(const EvalArgs& E, int a) {
    const int T2 = min(2 * E.n_nodes, 2 * MAXM);
    const int nl = 8 + 5 * (E.sub_kind ? E.n_sub : 0);
    const int lane = threadIdx.x & 31;
    for (int p = threadIdx.x >> 5; p < nl; p += blockDim.x >> 5) {
        double s = 0.0;
        for (int t = lane; t < T2; t += 32)
            s += E.tadj[TADJ_SEL + a * 2 * MAXM + t] * E.jsel[(size_t)(a * 2 * MAXM + t) * nl + p];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) E.cadj[(size_t)(E.n_cta_c + a) * nl + p] = s;
    }
}

// One CTA per (evaluation, axis); the uniform-grid transform couples the axes
// (one box side) and is done by the axis-0 CTA alone.
constexpr int CDF_NT = 256;
constexpr int CDF_CHEB_STAGE = 2048;      // doubles of the fit's matrices staged in shared memory
__global__ void __launch_bounds__(CDF_NT) k_cdf_adj(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int ax = blockIdx.x - B.tile0[ev];
    const int M = E.n_nodes, D = E.degree, K = M + 2, N = E.n_mask;
    __shared__ double tot[NACC_FIX + 4 * (MAXM + 2)];
    __shared__ double gXr[MAXM + 2], gpr[MAXM + 2], gc[MAXM], gQ[MAXM];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double* tr = E.trd;
    const double sigma = tr[2];
    if (E.transform == RTU_TRANSFORM_UNIFORM) {
        if (ax != 0) return;
        const double isig = 1.0 / sigma;
        for (int col = wid; col < NACC_FIX + 4 * K; col += CDF_NT / 32) {
            const double v = apart_col(E, col);
            if (lane == 0) tot[col] = v;
        }
        __syncthreads();
        // uniform grid: X_j = (lo_a + U_j L - mu_a)/sigma, slopes sigma/L, with
        // lo_a = (min_a + max_a)/2 - L/2 and L the larger range (axis amax)
        if (threadIdx.x == 0) {
            const int amax = tr[5] > 0.5 ? 1 : 0;
            const double L = tr[6], iL = 1.0 / L;
            double dmu[2] = {tot[8], tot[9]}, dsig = tot[10], dL = 0.0, dc[2] = {0.0, 0.0};
            for (int a = 0; a < 2; ++a) {
                const double* X = tr + TR_HDR + a * K;
                for (int j = 0; j < K; ++j) {
                    const double U = j == 0 ? 0.0 : (j == K - 1 ? 1.0 : E.cheb[cheb_u(M, D) + j - 1]);
                    const double gX = tot[NACC_FIX + a * K + j], gd = tot[NACC_FIX + 2 * K + a * K + j];
                    dc[a] += gX * isig;
                    dL += gX * (U - 0.5) * isig - gd * sigma * iL * iL;
                    dmu[a] -= gX * isig;
                    dsig += -gX * X[j] * isig + gd * iL;
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
            E.tadj[3] = tr[3];
            E.tadj[4] = dsig;
            E.tadj[5] = 0.0;
        }
        __syncthreads();
        sel_terms(E, 0);
        sel_terms(E, 1);
        return;
    }
    // this axis's guarded knots, raw knots, raw p' and slopes, staged (the serial
    // parts below walk them), and the fit's matrices when they fit the staging buffer
    __shared__ double sXf[MAXM + 2], sXr[MAXM + 2], spr[MAXM + 2], ssl[MAXM + 2];
    __shared__ double scheb[CDF_CHEB_STAGE];
    for (int j = threadIdx.x; j < K; j += CDF_NT) {
        sXf[j] = tr[TR_HDR + ax * K + j];
        sXr[j] = tr[TR_HDR + (6 + ax) * K + j];
        spr[j] = tr[TR_HDR + (4 + ax) * K + j];
        ssl[j] = tr[TR_HDR + (2 + ax) * K + j];
    }
    const int ncheb = cheb_C(M, D) + (D + 1) * M;
    const bool cstaged = ncheb <= CDF_CHEB_STAGE;
    if (cstaged)
        for (int i = threadIdx.x; i < ncheb; i += CDF_NT) scheb[i] = E.cheb[i];
    const double* cheb = cstaged ? scheb : E.cheb;
    // 1/sigma by one thread (an FP64 divide in every warp would queue 8 of them on
    // the SM's FP64 pipe, which takes one warp instruction at a time)
    __shared__ double isig_sh;
    if (threadIdx.x == 0) isig_sh = 1.0 / sigma;
    // this axis's columns: dmu_a, dsigma (axis 0), knots X and slopes d; each column's
    // rows in CDF_PARTS contiguous parts, one per lane of a group of adjacent lanes
    // (in order), the parts combined by a fixed shuffle tree -- about a third of the
    // FP64 instructions of a lane-strided warp tree per column
    constexpr int CDF_PARTS = 4;
    const int ncol = 2 + 2 * K;
    {
        const int rows = E.n_row_adj;
        const int q = (rows + CDF_PARTS - 1) / CDF_PARTS;
        for (int base = wid * 32; base < ncol * CDF_PARTS; base += CDF_NT) {      // warp-uniform
            const int it = base + lane, w = it / CDF_PARTS, part = it - w * CDF_PARTS;
            int col = 0;
            double v = 0.0;
            if (w < ncol) {
                col = w == 0 ? 8 + ax : (w == 1 ? 10 : (w < 2 + K ? NACC_FIX + ax * K + (w - 2)
                                                                 : NACC_FIX + 2 * K + ax * K + (w - 2 - K)));
                const double* a = E.apart + (size_t)col * rows;
                const int r0 = part * q, r1 = min(rows, r0 + q);
#pragma unroll 8
                for (int t = r0; t < r1; ++t) v += a[t];
            }
            v += __shfl_xor_sync(0xffffffffu, v, 1);     // (p0 + p1), (p2 + p3)
            v += __shfl_xor_sync(0xffffffffu, v, 2);     // then their sum
            if (w < ncol && part == 0) tot[col] = v;
        }
    }
    __syncthreads();
    const double isig = isig_sh;
    const double* gX = tot + NACC_FIX + ax * K;
    const double* gd = tot + NACC_FIX + 2 * K + ax * K;
    const double* Xf = sXf;      // guarded knots
    const double* Xr = sXr;      // raw knots
    const double* pr = spr;      // raw p'
    const double* sl = ssl;      // slopes 1/p'
    // the floor's span: formed by the threads that use it (one warp for K <= 32)
    double span = 0.0, floor_d = 0.0;
    bool span_ok = true;
    if (threadIdx.x < ((K + 31) & ~31)) {
        span = Xr[K - 1] - Xr[0];
        span_ok = span > 0.0;
        if (!span_ok) span = fabs(span) + 1e-300;
        floor_d = 1e-6 * span;
    }
    // back through the slope floor (per point) ...
    for (int j = threadIdx.x; j < K; j += CDF_NT) {
        const double gp = -gd[j] * sl[j] * sl[j];    // slope d = 1/p'
        gpr[j] = pr[j] < floor_d ? 0.0 : gp;
        gXr[j] = gX[j];
    }
    __syncthreads();
    // ... and the knot floor (sequential in the knots; the floor's span terms): the
    // floored slopes' terms summed by warp 0 (lane stride, fixed tree), the carry down
    // the floored knots by its lane 0
    double gfl = 0.0;
    if (wid == 0) {
        for (int j = lane; j < K; j += 32)
            if (pr[j] < floor_d) gfl += -gd[j] * sl[j] * sl[j];
        for (int o = 16; o > 0; o >>= 1) gfl += __shfl_down_sync(0xffffffffu, gfl, o);
    }
    if (threadIdx.x == 0) {
        for (int j = K - 1; j >= 1; --j)
            if (Xf[j] != Xr[j]) { gXr[j - 1] += gXr[j]; gfl += gXr[j]; gXr[j] = 0.0; }
        // floor = 1e-6 |span| (+ 1e-300 when the span is not positive): d floor / d span
        const double ds = span_ok ? 1e-6 : -1e-6;
        gXr[K - 1] += ds * gfl;
        gXr[0] -= ds * gfl;
    }
    __syncthreads();
    // knots X = V c and slopes p' = dV c  ->  gc = V^T gX + dV^T gp'
    const double* Vt = cheb + cheb_V(M, D);
    const double* dVt = cheb + cheb_dV(M, D);
    for (int k = threadIdx.x; k <= D; k += CDF_NT) {
        double g = 0.0;
#pragma unroll 8
        for (int j = 0; j < K; ++j) g += Vt[j * (D + 1) + k] * gXr[j] + dVt[j * (D + 1) + k] * gpr[j];
        gc[k] = g;
    }
    __syncthreads();
    // c = C Q  ->  gQ = C^T gc; Q = z_lo + frac (z_hi - z_lo), z = (beta - mu)/sigma
    const double* Ct = cheb + cheb_C(M, D);
    for (int i = threadIdx.x; i < M; i += CDF_NT) {
        double g = 0.0;
#pragma unroll 8
        for (int k = 0; k <= D; ++k) g += Ct[k * M + i] * gc[k];
        gQ[i] = g;
        const double h = cheb[cheb_u(M, D) + i] * (E.wtot - 1);
        const double frac = h - floor(h);
        E.tadj[TADJ_SEL + ax * 2 * MAXM + 2 * i] = g * (1.0 - frac) * isig;
        E.tadj[TADJ_SEL + ax * 2 * MAXM + 2 * i + 1] = g * frac * isig;
    }
    __syncthreads();
    // mu and sigma parts: fixed lane stride over the nodes, fixed tree
    if (wid == 0) {
        const double* Q = tr + TR_HDR + 8 * K + 2 * MAXM + ax * MAXM;
        double sq = 0.0, sqq = 0.0;
        for (int i = lane; i < M; i += 32) {
            sq += gQ[i];
            sqq += gQ[i] * Q[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_down_sync(0xffffffffu, sq, o);
            sqq += __shfl_down_sync(0xffffffffu, sqq, o);
        }
        if (lane == 0) {
            E.tadj[ax] = (tot[8 + ax] - sq * isig) / N;
            E.tadj[4 + ax] = (ax == 0 ? tot[10] : 0.0) - sqq * isig;
            if (ax == 0) E.tadj[3] = tr[3];
        }
    }
    sel_terms(E, ax);      // the selected-rank tadj entries were written before the barrier
}

// centre rays: d logL / d beta_i = dmu/N + [a = argmin sigma] dsigma (beta_i,a -
//   mu_a)/(N sigma_min) here, then the lens (the selected-rank terms, large and
//   few, come from k_sel_jac's rows, in double)
template <typename T>
__global__ void __launch_bounds__(CTA_C) k_centre_adj(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int N = E.n_mask;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nl = 8 + 5 * nsub;
    __shared__ LensK<T> L;
    __shared__ LensK<double> Ld;
    __shared__ double hdr[4], mu[2];
    // per-warp partials as (compensated, for float) pairs of the kernel's type: every
    // FP64 instruction takes a slot of the SM's FP64 pipe for the whole warp however
    // few lanes are active, so the conversion to double waits for the CTA's sums
    typedef decltype(warp_pair_sum(T(0))) P;
    __shared__ P red[CTA_C / 32][8];
    load_lensk(L, lensk_src<T>(E.lensk));
    if (sizeof(T) == 4) load_lensk(Ld, E.lensk);
    if (threadIdx.x < 4) hdr[threadIdx.x] = E.tadj[threadIdx.x];
    if (threadIdx.x == 2) hdr[2] = (E.tadj[4] + E.tadj[5]) / (N * E.trd[2]);
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
            gb[a] = g;
        }
        // the pixel centre (sub-ray offset 0 at s = 1)
        const int pix = E.centre_idx[k];
        const int pj = pix / E.n_img, pi = pix - pj * E.n_img;
        const double c = 0.5 * (E.n_img - 1);
        xd = (pi - c) * E.pix;
        yd = (pj - c) * E.pix;
    }
    T acc[8];
    for (int p = 0; p < 8; ++p) acc[p] = T(0);
    // a near-core centre ray of the float path: its lens vector-Jacobian product in
    // double, kept in double (near the core d alpha / d lens grows without bound, and
    // one such term rounded to float can outweigh the rest of the sum)
    double accd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool nearc = false;
    if (k < N) {
        const T x = (T)xd, y = (T)yd;
        if (sizeof(T) == 4 && lens_near_core(L, x, y)) {
            EplJ<double> J;
            double bx, by;
            lens_beta_eval(Ld, xd, yd, J, bx, by);
            lens_beta_vjp(Ld, J, xd, yd, gb[0], gb[1], accd);
            nearc = true;
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
        const P v = warp_pair_sum(acc[p]);
        if (lane == 0) red[wid][p] = v;
    }
    // the double terms of the warps that hold a near-core ray (fixed shuffle tree)
    __shared__ double redd[CTA_C / 32][8];
    const bool anyd = __any_sync(0xffffffffu, nearc);
    for (int p = 0; p < 8; ++p) {
        const double v = anyd ? warp_sum(accd[p]) : 0.0;
        if (lane == 0) redd[wid][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        P r = red[0][threadIdx.x];
        for (int w = 1; w < CTA_C / 32; ++w) pair_add(r, red[w][threadIdx.x]);
        double rd = (double)r.x + (double)r.y;
        for (int w = 0; w < CTA_C / 32; ++w) rd += redd[w][threadIdx.x];
        out[threadIdx.x] = rd;
    }
    for (int h = 0; h < nsub; ++h) {
        __syncthreads();
        T a5[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (k < N) sub_vjp<T>(L, h, (T)xd, (T)yd, (T)gb[0], (T)gb[1], a5);
        for (int c = 0; c < 5; ++c) {
            const P v = warp_pair_sum(a5[c]);
            if (lane == 0) red[wid][c] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            P r = red[0][threadIdx.x];
            for (int w = 1; w < CTA_C / 32; ++w) pair_add(r, red[w][threadIdx.x]);
            out[8 + 5 * h + threadIdx.x] = (double)r.x + (double)r.y;
        }
    }
}

// The selected-rank lens Jacobians: every (axis a, target t) whose order statistic
// the QF interpolates contributes (d logL / d beta_a of its ray) times the row
// d beta_a / d lens of that ray, in double (these few terms are large and partly
// cancel the image terms).  The rows depend on the lens and the selection only, so the
// forward computes them (beside the render, after the selection) and the transform
// adjoint takes the weighted sum once the cotangents are known.  One CTA per
// evaluation, one thread per (axis, target): jsel[(a 2 MAXM + t) nl + p].
constexpr int SEL_ADJ_NT = 4 * MAXM;
__global__ void __launch_bounds__(SEL_ADJ_NT) k_sel_jac(const __grid_constant__ Batch B) {
    // systems of the unsmoothed transform launch no CTA here: map through the prefix
    const EvalArgs& E = B.e[find_eval(B, blockIdx.x)];
    const int M = E.n_nodes;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nl = 8 + 5 * nsub;
    __shared__ LensK<double> Ld;
    __shared__ LensK<DF> Ldf;
    load_lensk(Ld, E.lensk);
    __syncthreads();
    // the float path without subhaloes evaluates these rows in double-float (about
    // 48 bits) on the FP32 pipes: FP64 instructions are scarce on this part
    const bool use_df = !E.f64 && Ld.nsub == 0;
    if (use_df) {
        load_lensk(Ldf, lensk_df_src(E.lensk));
        __syncthreads();
    }
    const int a = threadIdx.x / (2 * MAXM), t = threadIdx.x - a * 2 * MAXM;
    const int ray = t < 2 * M ? E.sel_idx[a * 2 * MAXM + t] : -1;
    double o8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double xd = 0.0, yd = 0.0;
    const bool ok = ray >= 0 && ray < E.n_mask;
    if (ok) {
        const int pix = E.centre_idx[ray];
        const int pj = pix / E.n_img, pi = pix - pj * E.n_img;
        const double c = 0.5 * (E.n_img - 1);
        xd = (pi - c) * E.pix;
        yd = (pj - c) * E.pix;
        if (use_df) {
            EplJ<DF> J;
            DF bx, by;
            const DF xf(xd), yf(yd), one(1.0f), zero(0.0f, 0.0f);
            lens_beta_eval_smooth(Ldf, xf, yf, J, bx, by);
            DF o8f[8] = {zero, zero, zero, zero, zero, zero, zero, zero};
            lens_beta_vjp(Ldf, J, xf, yf, a == 0 ? one : zero, a == 1 ? one : zero, o8f);
            for (int p = 0; p < 8; ++p) o8[p] = o8f[p].to_double();
        } else {
            EplJ<double> J;
            double bx, by;
            lens_beta_eval(Ld, xd, yd, J, bx, by);
            lens_beta_vjp(Ld, J, xd, yd, a == 0 ? 1.0 : 0.0, a == 1 ? 1.0 : 0.0, o8);
        }
    }
    double* row = E.jsel + (size_t)threadIdx.x * nl;
    for (int p = 0; p < 8; ++p) row[p] = o8[p];
    for (int h = 0; h < nsub; ++h) {
        double a5[5] = {0, 0, 0, 0, 0};
        if (ok) sub_vjp<double>(Ld, h, xd, yd, a == 0 ? 1.0 : 0.0, a == 1 ? 1.0 : 0.0, a5);
        for (int c = 0; c < 5; ++c) row[8 + 5 * h + c] = a5[c];
    }
}

// The unsmoothed eCDF (App. C, first paragraph): centre ray i holds rank r_a(i) on
// axis a, so d logL / d beta_i = (gk_x[r_x(i)], gk_y[r_y(i)]); then the lens (and
// subhaloes), in double: every centre ray carries terms of the size of the image
// terms they cancel.  One thread per centre ray, rows 0..n_cta_c-1 of cadj; the
// CTA of tile 0 also clears rows n_cta_c and n_cta_c + 1 (the selected-rank rows of
// the smoothed grid).
__global__ void __launch_bounds__(CTA_C) k_lin_centre_adj(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int N = E.n_mask;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nl = 8 + 5 * nsub;
    __shared__ LensK<double> Ld;
    __shared__ double red[CTA_C / 32][8];
    load_lensk(Ld, E.lensk);
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    double o8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double xd = 0.0, yd = 0.0, gx = 0.0, gy = 0.0;
    if (k < N) {
        gx = fix128_value(E.gk + 2 * (size_t)E.lrank[k]);
        gy = fix128_value(E.gk + 2 * ((size_t)N + E.lrank[N + k]));
        const int pix = E.centre_idx[k];
        const int pj = pix / E.n_img, pi = pix - pj * E.n_img;
        const double c = 0.5 * (E.n_img - 1);
        xd = (pi - c) * E.pix;
        yd = (pj - c) * E.pix;
        EplJ<double> J;
        double bx, by;
        lens_beta_eval(Ld, xd, yd, J, bx, by);
        lens_beta_vjp(Ld, J, xd, yd, gx, gy, o8);
    }
    double* out = E.cadj + (size_t)tile * nl;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = 0; p < 8; ++p) {
        const double v = warp_sum(o8[p]);
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
        double a5[5] = {0, 0, 0, 0, 0};
        if (k < N) sub_vjp<double>(Ld, h, xd, yd, gx, gy, a5);
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
    if (tile == 0)
        for (int p = threadIdx.x; p < 2 * nl; p += CTA_C) E.cadj[(size_t)E.n_cta_c * nl + p] = 0.0;
}

// g_lens = (render-adjoint lens sums) + (centre-adjoint lens sums), one warp per
// parameter (lane-strided rows, fixed shuffle tree); lens-light moments likewise
constexpr int GRAD_NT = 256;
__global__ void __launch_bounds__(GRAD_NT) k_grad_final(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    const int K = E.n_nodes + 2;
    const int nsub = E.sub_kind ? E.n_sub : 0;
    const int nl = 8 + 5 * nsub;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = GRAD_NT / 32;
    if (threadIdx.x == 0) *E.gmax = 0ull;     // the next adjoint's PSF pass starts from zero
    for (int p = wid; p < nl; p += NW) {
        const int col = p < 8 ? p : NACC_FIX + 4 * K + (p - 8);
        const double s = apart_col(E, col);
        const double c = warp_rows_sum(E.cadj + p, E.n_cta_c + 2, nl);   // + the selected-rank rows
        double g = s + c;
        if (p == 1 && E.profile == 0) g = 0.0;
        if (lane == 0) E.g_lens[p] = g;
    }
    // spectrum parameters and alpha_src: the GP adjoint's per-CTA partials
    {
        const int nf = E.family == 2 ? 3 : 2;
        const int ngl = gp_part_rows(E.n_src);
        for (int c = wid; c <= nf; c += NW) {
            const double v = warp_rows_sum(E.gpart + (c < nf ? c : 3), ngl, 4);
            if (lane == 0) E.g_ps[c] = v;
        }
    }
    // lens light: per component the moment sums of k_light_adj, then d log L / d (A,
    // sigma, q, phi, x_n, y_n) with L_n = A/(2 pi) exp(-E), E = (q x'^2 + y'^2/q)/(2
    // sigma^2), x' = cos phi dx + sin phi dy, y' = cos phi dy - sin phi dx
    const int nlp = E.light ? 6 * E.n_light : 0;
    if (nlp == 0) return;
    __shared__ double mom[6 * MAX_LIGHT];
    const int nlc = light_ctas(E.n_img);
    for (int i = wid; i < nlp; i += NW) {
        const double v = warp_rows_sum(E.lpartl + i, nlc, nlp);
        if (lane == 0) mom[i] = v;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < nlp / 6; n += GRAD_NT) {
        const double* m = mom + 6 * n;
        const double* p = E.light + 6 * n;
        const double A = p[0], sg = p[1], q = p[2], cs = cos(p[3]), sn = sin(p[3]);
        const double c1 = 0.5 / (sg * sg);
        const double wx = cs * m[1] + sn * m[2], wy = cs * m[2] - sn * m[1];
        const double wxx = cs * cs * m[3] + 2.0 * cs * sn * m[4] + sn * sn * m[5];
        const double wyy = sn * sn * m[3] - 2.0 * cs * sn * m[4] + cs * cs * m[5];
        const double wxy = -cs * sn * m[3] + (cs * cs - sn * sn) * m[4] + cs * sn * m[5];
        const double wE = c1 * (q * wxx + wyy / q);
        double g[6];
        g[0] = m[0] / A;
        g[1] = 2.0 * wE / sg;
        g[2] = -c1 * (wxx - wyy / (q * q));
        g[3] = -2.0 * c1 * (q - 1.0 / q) * wxy;
        g[4] = 2.0 * c1 * (q * cs * wx - sn / q * wy);
        g[5] = 2.0 * c1 * (q * sn * wx + cs / q * wy);
        if (E.g_light)
            for (int k = 0; k < 6; ++k) E.g_light[6 * n + k] = g[k];
    }
}

}  // namespace rtu
