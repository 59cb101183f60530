// k_grid.cuh -- building the RTU transform (Sec. 2.2, App. C steps i-iv).
//
//  k_trace_centres  trace the arc-mask pixel centres (double), per-CTA sums and
//                   ranges of beta
//  k_centre_hist    level-1 integer histograms of beta per axis (HB bins over
//                   [min, max]) and per-CTA sums of squared deviations
//  k_select_fit     one CTA per evaluation: prefix scan of the histograms, exact
//                   order statistics at the Chebyshev-node ranks, the Chebyshev
//                   fit of the quantile function (discrete cosine sums, exact
//                   interpolation for M = D+1), Hermite knots/slopes, guard.
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

__device__ __forceinline__ int beta_bin(double b, double lo, double scale) {
    // scale = HB / (hi - lo); identical expression in every kernel that bins
    double t = (b - lo) * scale;
    int k = (int)t;
    return k < 0 ? 0 : (k >= HB ? HB - 1 : k);
}

__global__ void __launch_bounds__(CTA_C) k_trace_centres(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LensK<double> L;
    __shared__ double red[6][CTA_C / 32];
    load_lensk(L, E.lensk);
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    double bx = 0.0, by = 0.0;
    double v[6];
    if (k < E.n_mask) {
        double x, y;
        ray_pos(E.n_img, E.pix, 1, E.centre_idx[k], 0, x, y);
        lens_beta(L, x, y, bx, by);
        E.beta[k] = bx;
        E.beta[E.n_mask + k] = by;
        v[0] = bx; v[1] = by; v[2] = bx; v[3] = bx; v[4] = by; v[5] = by;
    } else {
        v[0] = 0.0; v[1] = 0.0; v[2] = 1e300; v[3] = -1e300; v[4] = 1e300; v[5] = -1e300;
    }
    // fixed-order reduction: warp tree, then warps in order
    for (int o = 16; o > 0; o >>= 1) {
        v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
        v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
        v[2] = fmin(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
        v[3] = fmax(v[3], __shfl_down_sync(0xffffffffu, v[3], o));
        v[4] = fmin(v[4], __shfl_down_sync(0xffffffffu, v[4], o));
        v[5] = fmax(v[5], __shfl_down_sync(0xffffffffu, v[5], o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 6; ++q) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        double r = red[q][0];
        for (int i = 1; i < CTA_C / 32; ++i) {
            double o = red[q][i];
            r = q < 2 ? r + o : ((q & 1) == 0 ? fmin(r, o) : fmax(r, o));
        }
        E.cpart[tile * 8 + q] = r;
    }
}

// reduce the per-CTA centre sums: mean and range per axis (same order everywhere)
__device__ __forceinline__ void centre_moments(const EvalArgs& E, double* out6) {
    double s0 = 0.0, s1 = 0.0, lo0 = 1e300, hi0 = -1e300, lo1 = 1e300, hi1 = -1e300;
    for (int t = 0; t < E.n_cta_c; ++t) {
        const double* c = E.cpart + t * 8;
        s0 += c[0]; s1 += c[1];
        lo0 = fmin(lo0, c[2]); hi0 = fmax(hi0, c[3]);
        lo1 = fmin(lo1, c[4]); hi1 = fmax(hi1, c[5]);
    }
    out6[0] = s0 / E.n_mask; out6[1] = s1 / E.n_mask;
    out6[2] = lo0; out6[3] = hi0; out6[4] = lo1; out6[5] = hi1;
}

__device__ __forceinline__ double bin_scale(double lo, double hi) {
    return hi > lo ? (double)HB / (hi - lo) : 0.0;
}

__global__ void __launch_bounds__(CTA_C) k_centre_hist(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ double m[6];
    __shared__ double red[2][CTA_C / 32];
    if (threadIdx.x == 0) centre_moments(E, m);
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    double d0 = 0.0, d1 = 0.0;
    if (k < E.n_mask) {
        double bx = E.beta[k], by = E.beta[E.n_mask + k];
        atomicAdd(E.hist + beta_bin(bx, m[2], bin_scale(m[2], m[3])), 1);
        atomicAdd(E.hist + HB + beta_bin(by, m[4], bin_scale(m[4], m[5])), 1);
        d0 = (bx - m[0]) * (bx - m[0]);
        d1 = (by - m[1]) * (by - m[1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = d0; red[1][threadIdx.x >> 5] = d1; }
    __syncthreads();
    if (threadIdx.x < 2) {
        double r = 0.0;
        for (int i = 0; i < CTA_C / 32; ++i) r += red[threadIdx.x][i];
        E.cpart2[tile * 2 + threadIdx.x] = r;
    }
}

constexpr int SEL_NT = 1024;

// One CTA per evaluation.  Dynamic shared memory:
//   double ck[SEL_CAP]; int ci[SEL_CAP]; unsigned bitmap[HB/32];
__global__ void __launch_bounds__(SEL_NT) k_select_fit(const __grid_constant__ Batch B) {
    const EvalArgs& E = B.e[blockIdx.x];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double* ck = reinterpret_cast<double*>(smem_raw);
    int* ci = reinterpret_cast<int*>(ck + SEL_CAP);
    unsigned* bitmap = reinterpret_cast<unsigned*>(ci + SEL_CAP);
    __shared__ double mom[6];
    __shared__ double sig[3];
    __shared__ int chunk_off[SEL_NT + 1];
    __shared__ int t_bin[2 * MAXM], t_below[2 * MAXM], t_rank[2 * MAXM], t_slot[2 * MAXM];
    __shared__ int d_bin[2 * MAXM], d_off[2 * MAXM + 1], d_fill[2 * MAXM];
    __shared__ int n_d;
    __shared__ double Qs[2][MAXM];
    __shared__ double coef[2][MAXM];
    __shared__ int flag_sh;
    const int tid = threadIdx.x;
    const int N = E.n_mask, M = E.n_nodes, D = E.degree, K = M + 2;

    if (tid == 0) {
        centre_moments(E, mom);
        double v0 = 0.0, v1 = 0.0;
        for (int t = 0; t < E.n_cta_c; ++t) { v0 += E.cpart2[2 * t]; v1 += E.cpart2[2 * t + 1]; }
        double sx = sqrt(v0 / N), sy = sqrt(v1 / N);
        sig[0] = sx <= sy ? sx : sy;            // sigma_min, tie -> x (App. C i)
        sig[1] = sx <= sy ? 0.0 : 1.0;
        flag_sh = 0;
    }
    __syncthreads();
    const double sigma = sig[0];

    for (int a = 0; a < 2; ++a) {
        const int* hist = E.hist + a * HB;
        const double* beta = E.beta + a * N;
        const double lo = mom[2 + 2 * a], hi = mom[3 + 2 * a];
        const double scale = bin_scale(lo, hi);
        // exclusive scan of HB bins: 64 consecutive bins per thread
        constexpr int PER = HB / SEL_NT;
        int own = 0;
        for (int i = 0; i < PER; ++i) own += hist[tid * PER + i];
        // block scan (warp inclusive scans, then warp totals)
        int incl = own;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o) incl += y;
        }
        __shared__ int wtot[SEL_NT / 32];
        if ((tid & 31) == 31) wtot[tid >> 5] = incl;
        for (int i = tid; i < 2 * MAXM; i += SEL_NT) d_fill[i] = 0;
        for (int i = tid; i < HB / 32; i += SEL_NT) bitmap[i] = 0u;
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < SEL_NT / 32; ++w) { int t = wtot[w]; wtot[w] = acc; acc += t; }
            chunk_off[SEL_NT] = acc;
        }
        __syncthreads();
        chunk_off[tid] = wtot[tid >> 5] + incl - own;
        __syncthreads();
        // target ranks: node j -> floor(u_j (N-1)) and the next one (RTU grid); the
        // smallest and largest ray (uniform grid: the square box, Sec. 2.1)
        const int nt = E.transform ? 2 : 2 * M;
        for (int t = tid; t < nt; t += SEL_NT) {
            int k;
            if (E.transform) {
                k = t == 0 ? 0 : N - 1;
            } else {
                double h = E.cheb[cheb_u(M, D) + t / 2] * (N - 1);
                k = (int)floor(h);
                k = k < 0 ? 0 : (k > N - 1 ? N - 1 : k);
                if (t & 1) k = k + 1 > N - 1 ? N - 1 : k + 1;
            }
            t_rank[t] = k;
        }
        for (int t = nt + tid; t < 2 * MAXM; t += SEL_NT) E.sel_idx[a * 2 * MAXM + t] = -1;
        for (int t = tid; t < nt; t += SEL_NT) { t_bin[t] = 0; t_below[t] = 0; }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const int r = t_rank[t];
            if (chunk_off[tid] <= r && r < chunk_off[tid + 1]) {
                int c = chunk_off[tid];
                for (int i = 0; i < PER; ++i) {
                    int h = hist[tid * PER + i];
                    if (r < c + h) { t_bin[t] = tid * PER + i; t_below[t] = c; break; }
                    c += h;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            // distinct target bins (ranks are non-decreasing, so are their bins)
            int nd = 0, off = 0;
            for (int t = 0; t < nt; ++t) {
                if (nd == 0 || d_bin[nd - 1] != t_bin[t]) {
                    d_bin[nd] = t_bin[t];
                    d_off[nd] = off;
                    int cnt = hist[t_bin[t]];
                    off += cnt;
                    bitmap[t_bin[t] >> 5] |= 1u << (t_bin[t] & 31);
                    ++nd;
                }
                t_slot[t] = nd - 1;
            }
            d_off[nd] = off;
            n_d = nd;
            if (off > SEL_CAP) flag_sh |= F_SELECT;
        }
        __syncthreads();
        const int nd = n_d;
        // gather the candidates of the target bins
        for (int k = tid; k < N; k += SEL_NT) {
            const double b = beta[k];
            const int bn = beta_bin(b, lo, scale);
            if (bitmap[bn >> 5] & (1u << (bn & 31))) {
                int d = 0;
                while (d < nd - 1 && d_bin[d] != bn) ++d;
                const int pos = atomicAdd(&d_fill[d], 1);
                const int at = d_off[d] + pos;
                if (at < SEL_CAP && pos < d_off[d + 1] - d_off[d]) { ck[at] = b; ci[at] = k; }
            }
        }
        __syncthreads();
        // the element of rank (r - below) inside its bin, ties ordered by index
        for (int t = 0; t < nt; ++t) {
            const int d = t_slot[t];
            const int o = d_off[d], cnt = min(d_off[d + 1], SEL_CAP) - o;
            const int want = t_rank[t] - t_below[t];
            for (int c = tid; c < cnt; c += SEL_NT) {
                const double kc = ck[o + c];
                const int ic = ci[o + c];
                int rank = 0;
                for (int c2 = 0; c2 < cnt; ++c2) {
                    const double k2 = ck[o + c2];
                    rank += (k2 < kc) || (k2 == kc && ci[o + c2] < ic);
                }
                if (rank == want) {
                    E.sel_val[a * 2 * MAXM + t] = kc;
                    E.sel_idx[a * 2 * MAXM + t] = ic;
                }
            }
        }
        __syncthreads();
        // empirical QF at the nodes in standardized coordinates (type-7 interpolation)
        for (int j = tid; j < M && !E.transform; j += SEL_NT) {
            double h = E.cheb[cheb_u(M, D) + j] * (N - 1);
            double frac = h - floor(h);
            double zl = (E.sel_val[a * 2 * MAXM + 2 * j] - mom[a]) / sigma;
            double zh = (E.sel_val[a * 2 * MAXM + 2 * j + 1] - mom[a]) / sigma;
            Qs[a][j] = zl + frac * (zh - zl);
        }
        __syncthreads();
    }

    double* tr = E.trd;
    if (E.transform) {
        // uniform grid: the smallest square box around the masked rays, centred on
        // each axis's range, mapped affinely onto [0, 1]^2 -- written as Hermite
        // knots X_j = (lo + U_j L - mu)/sigma with equal slopes sigma/L (linear)
        if (tid < 2) {
            const int a = tid;
            const double mn0 = E.sel_val[0], mx0 = E.sel_val[1];
            const double mn1 = E.sel_val[2 * MAXM], mx1 = E.sel_val[2 * MAXM + 1];
            const double r0 = mx0 - mn0, r1 = mx1 - mn1;
            const double L = r0 >= r1 ? r0 : r1;
            const double mn = a == 0 ? mn0 : mn1, mx = a == 0 ? mx0 : mx1;
            const double lo = 0.5 * (mn + mx) - 0.5 * L;
            for (int j = 0; j < K; ++j) {
                const double U = j == 0 ? 0.0 : (j == K - 1 ? 1.0 : E.cheb[cheb_u(M, D) + j - 1]);
                const double X = (lo + U * L - mom[a]) / sigma;
                tr[TR_HDR + a * K + j] = X;
                tr[TR_HDR + (6 + a) * K + j] = X;
                tr[TR_HDR + (2 + a) * K + j] = sigma / L;
                tr[TR_HDR + (4 + a) * K + j] = L / sigma;
            }
            if (a == 0) { tr[5] = r0 >= r1 ? 0.0 : 1.0; tr[6] = L; }
        }
        if (tid == 0) {
            tr[0] = mom[0]; tr[1] = mom[1]; tr[2] = sigma; tr[3] = sig[1]; tr[4] = K;
        }
        __syncthreads();
        for (int i = tid; i < TR_HDR + 4 * K; i += SEL_NT) E.trf[i] = (float)tr[i];
        if (E.cdf_out) {
            for (int i = tid; i < 3; i += SEL_NT) E.cdf_out[i] = tr[i];
            for (int i = tid; i < 4 * K; i += SEL_NT) E.cdf_out[3 + i] = tr[TR_HDR + i];
        }
        if (tid == 0 && flag_sh) atomicOr(E.flags, flag_sh);
        return;
    }
    // App. C iii: Chebyshev coefficients of the QF from M = D+1 nodes by the
    // discrete orthogonality of T_k on the nodes: c = C Q (one thread per coefficient)
    const double* Ct = E.cheb + cheb_C(M, D);
    for (int w = tid; w < 2 * (D + 1); w += SEL_NT) {
        const int a = w / (D + 1), k = w % (D + 1);
        double sacc = 0.0;
        for (int j = 0; j < M; ++j) sacc += Ct[k * M + j] * Qs[a][j];
        coef[a][k] = sacc;
    }
    __syncthreads();
    // App. C iv: knots p(0), p(u_j), p(1) and p'(u) there (one thread per point)
    __shared__ double Xs[2][MAXM + 2], Ps[2][MAXM + 2];
    const double* Vt = E.cheb + cheb_V(M, D);
    const double* dVt = E.cheb + cheb_dV(M, D);
    for (int w = tid; w < 2 * K; w += SEL_NT) {
        const int a = w / K, j = w % K;
        double p = 0.0, d = 0.0;
        for (int k = 0; k <= D; ++k) {
            p += Vt[j * (D + 1) + k] * coef[a][k];
            d += dVt[j * (D + 1) + k] * coef[a][k];
        }
        Xs[a][j] = p;
        Ps[a][j] = d;
        tr[TR_HDR + (6 + a) * K + j] = p;       // raw knots
        tr[TR_HDR + (4 + a) * K + j] = d;       // raw p'
    }
    __syncthreads();
    // monotonicity guard, sequential in the knots (one thread per axis)
    if (tid < 2) {
        const int a = tid;
        double* X = Xs[a];
        double* dp = Ps[a];
        int fl = 0;
        double span = X[K - 1] - X[0];
        if (!(span > 0.0)) { fl |= F_NONMONO; span = fabs(span) + 1e-300; }
        const double floor_d = 1e-6 * span;
        for (int j = 0; j < K; ++j)
            if (dp[j] < floor_d) { dp[j] = floor_d; fl |= F_NONMONO; }
        for (int j = 1; j < K; ++j) {
            double lim = X[j - 1] + floor_d;
            if (X[j] < lim) { X[j] = lim; fl |= F_NONMONO; }
        }
        for (int j = 0; j < K; ++j) {
            tr[TR_HDR + a * K + j] = X[j];
            tr[TR_HDR + (2 + a) * K + j] = 1.0 / dp[j];
        }
        for (int k = 0; k <= D; ++k) tr[TR_HDR + 8 * K + a * MAXM + k] = coef[a][k];
        for (int j = 0; j < M; ++j) tr[TR_HDR + 8 * K + 2 * MAXM + a * MAXM + j] = Qs[a][j];
        if (fl) atomicOr(&flag_sh, fl);
    }
    if (tid == 0) {
        tr[0] = mom[0]; tr[1] = mom[1]; tr[2] = sigma; tr[3] = sig[1]; tr[4] = K;
    }
    __syncthreads();
    // float copy for the float render path, the optional CDF output, flags
    for (int i = tid; i < TR_HDR + 4 * K; i += SEL_NT) E.trf[i] = (float)tr[i];
    if (E.cdf_out) {
        for (int i = tid; i < 3; i += SEL_NT) E.cdf_out[i] = tr[i];
        for (int i = tid; i < 4 * K; i += SEL_NT) E.cdf_out[3 + i] = tr[TR_HDR + i];
    }
    if (tid == 0 && flag_sh) atomicOr(E.flags, flag_sh);
}

}  // namespace rtu
