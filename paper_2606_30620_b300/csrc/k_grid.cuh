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
//  k_lin_sort       the unsmoothed transform (App. C, first paragraph): every
//                   order statistic, by a counting sort on the level-1 histogram
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

__device__ __forceinline__ int beta_bin(double b, double lo, double scale) {
    // scale = HB / (hi - lo); identical expression in every kernel that bins
    double t = (b - lo) * scale;
    int k = (int)t;
    return k < 0 ? 0 : (k >= HB ? HB - 1 : k);
}

// reduce the per-CTA centre sums: mean and range per axis.  Called by one whole
// warp; lane l takes the CTAs t = l mod 32 in order, then a fixed shuffle tree, so
// every call gets the same bits.  Lane 0 writes out6.
__device__ __forceinline__ void centre_moments(const EvalArgs& E, double* out6) {
    const int lane = threadIdx.x & 31;
    double s0 = 0.0, s1 = 0.0, lo0 = 1e300, hi0 = -1e300, lo1 = 1e300, hi1 = -1e300;
    for (int t = lane; t < E.n_cta_c; t += 32) {
        const double* c = E.cpart + t * 8;          // written by other CTAs: read through L2
        s0 += __ldcg(c); s1 += __ldcg(c + 1);
        lo0 = fmin(lo0, __ldcg(c + 2)); hi0 = fmax(hi0, __ldcg(c + 3));
        lo1 = fmin(lo1, __ldcg(c + 4)); hi1 = fmax(hi1, __ldcg(c + 5));
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        lo0 = fmin(lo0, __shfl_down_sync(0xffffffffu, lo0, o));
        hi0 = fmax(hi0, __shfl_down_sync(0xffffffffu, hi0, o));
        lo1 = fmin(lo1, __shfl_down_sync(0xffffffffu, lo1, o));
        hi1 = fmax(hi1, __shfl_down_sync(0xffffffffu, hi1, o));
    }
    if (lane == 0) {
        out6[0] = s0 / E.n_mask; out6[1] = s1 / E.n_mask;
        out6[2] = lo0; out6[3] = hi0; out6[4] = lo1; out6[5] = hi1;
    }
}

// 5 CTAs per SM (48 registers): the c2 batch's 678 CTAs then run in one wave
__global__ void __launch_bounds__(CTA_C, 5) k_trace_centres(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ LensK<double> L;
    __shared__ LensK<DF> Ldf;
    __shared__ double red[6][CTA_C / 32];
    __shared__ DF red_df[6][CTA_C / 32];
    // the float path traces its centre rays in double-float (about 48 bits) unless
    // subhaloes are present (and loads only that lens block); the double path in double
    const bool use_df = !E.f64 && !(E.sub_kind && E.n_sub > 0);
    __shared__ DF pix_df;
    if (use_df) {
        load_lensk(Ldf, lensk_df_src(E.lensk));
        if (threadIdx.x == 0) pix_df = DF(E.pix);
    } else {
        load_lensk(L, E.lensk);
    }
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    const bool ok = k < E.n_mask;
    if (use_df) {
        // positions and the warp reductions in double-float as well: on this part an
        // FP64 instruction holds the FP64 pipe for many cycles, and a warp tree of six
        // doubles per ray cost more than the lens itself
        DF bxf(0.0f, 0.0f), byf(0.0f, 0.0f);
        if (ok) {
            const int pix = E.centre_idx[k];
            const int pj = pix / E.n_img, pi = pix - pj * E.n_img;
            const float c = 0.5f * (float)(E.n_img - 1);      // pixel offsets are exact in float
            lens_beta_smooth<DF>(Ldf, DF((float)pi - c) * pix_df, DF((float)pj - c) * pix_df, bxf, byf);
            E.beta[k] = bxf.to_double();
            E.beta[E.n_mask + k] = byf.to_double();
        }
        const DF inf(INFINITY, 0.0f), ninf(-INFINITY, 0.0f), zero(0.0f, 0.0f);
        DF a[6] = {ok ? bxf : zero, ok ? byf : zero, ok ? bxf : inf, ok ? bxf : ninf, ok ? byf : inf, ok ? byf : ninf};
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const DF t(__shfl_down_sync(0xffffffffu, a[q].hi, o), __shfl_down_sync(0xffffffffu, a[q].lo, o));
                if (q < 2) a[q] = a[q] + t;
                else if ((q & 1) == 0) a[q] = t < a[q] ? t : a[q];
                else a[q] = a[q] < t ? t : a[q];
            }
        }
        // the CTA's partials in double-float as well, one conversion to double each:
        // every FP64 instruction, even with one lane active, takes a slot of the SM's
        // FP64 pipe for the whole warp
        if ((threadIdx.x & 31) == 0)
            for (int q = 0; q < 6; ++q) red_df[q][threadIdx.x >> 5] = a[q];
        __syncthreads();
        if (threadIdx.x < 6) {
            const int q = threadIdx.x;
            DF r = red_df[q][0];
            for (int i = 1; i < CTA_C / 32; ++i) {
                const DF o = red_df[q][i];
                r = q < 2 ? r + o : ((q & 1) == 0 ? (o < r ? o : r) : (r < o ? o : r));
            }
            E.cpart[tile * 8 + q] = r.to_double();
            __threadfence();
        }
    } else {
        double v[6];   // sum x, sum y, min x, max x, min y, max y of the warp (lane 0)
        double bx = 0.0, by = 0.0;
        if (ok) {
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
            __threadfence();
        }
    }
    // the last CTA of the evaluation to finish reduces the partials once (fixed order)
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(E.ccnt, 1) == E.n_cta_c - 1;
    __syncthreads();
    if (last && threadIdx.x < 32) {
        double m6[6];
        centre_moments(E, m6);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 6; ++q) E.mom[q] = m6[q];
            E.ccnt[0] = 0;
        }
    }
}

__device__ __forceinline__ double bin_scale(double lo, double hi) {
    return hi > lo ? (double)HB / (hi - lo) : 0.0;
}

__global__ void __launch_bounds__(CTA_C) k_centre_hist(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ double m[6], sc[2];
    __shared__ double dev[2][CTA_C];
    if (threadIdx.x < 6) m[threadIdx.x] = __ldcg(E.mom + threadIdx.x);
    __syncthreads();
    // the bin scales once per CTA (an FP64 divide each)
    if (threadIdx.x < 2) sc[threadIdx.x] = bin_scale(m[2 + 2 * threadIdx.x], m[3 + 2 * threadIdx.x]);
    __syncthreads();
    const int k = tile * CTA_C + threadIdx.x;
    double d0 = 0.0, d1 = 0.0;
    if (k < E.n_mask) {
        double bx = E.beta[k], by = E.beta[E.n_mask + k];
        const int w = E.cwt ? (int)E.cwt[k] : 1;      // weighted grid: the ray counts w times
        const int b0 = beta_bin(bx, m[2], sc[0]);
        const int b1 = beta_bin(by, m[4], sc[1]);
        atomicAdd(E.hist + b0, w);
        atomicAdd(E.hist + HB + b1, w);
        // the count of each bin's row of 32, so the selection reads 2 HROWS counts
        // instead of summing the 2 HB bins
        atomicAdd(E.hist + 2 * HB + (b0 >> 5), w);
        atomicAdd(E.hist + 2 * HB + HROWS + (b1 >> 5), w);
        E.cbin[k] = b0;
        E.cbin[E.n_mask + k] = b1;
        d0 = (bx - m[0]) * (bx - m[0]);
        d1 = (by - m[1]) * (by - m[1]);
    }
    // the CTA's sums of squared deviations by warp 0 alone (lane l adds the rays
    // l, l + 32, ... in order, then a shuffle tree): the SM's FP64 pipe takes one warp
    // instruction at a time, whatever its active lanes, so a tree in every warp
    // would cost eight times the instructions
    dev[0][threadIdx.x] = d0;
    dev[1][threadIdx.x] = d1;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double s0 = dev[0][lane], s1 = dev[1][lane];
#pragma unroll
        for (int i = 1; i < CTA_C / 32; ++i) { s0 += dev[0][lane + 32 * i]; s1 += dev[1][lane + 32 * i]; }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {                            // the tree's totals are in lane 0
            E.cpart2[tile * 2] = s0;
            E.cpart2[tile * 2 + 1] = s1;
            __threadfence();
        }
    }
    // the last CTA to finish: sums of squared deviations over the CTAs (lanes over
    // CTAs, fixed tree), once per evaluation
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(E.ccnt + 1, 1) == E.n_cta_c - 1;
    __syncthreads();
    if (last && threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double v0 = 0.0, v1 = 0.0;
        for (int t = lane; t < E.n_cta_c; t += 32) { v0 += __ldcg(E.cpart2 + 2 * t); v1 += __ldcg(E.cpart2 + 2 * t + 1); }
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_down_sync(0xffffffffu, v0, o);
            v1 += __shfl_down_sync(0xffffffffu, v1, o);
        }
        if (lane == 0) {
            E.mom[6] = v0;
            E.mom[7] = v1;
            E.ccnt[1] = 0;
        }
    }
}

// the optional build outputs of axis a: its level-1 histogram and traced centre positions
__device__ __forceinline__ void export_selection(const EvalArgs& E, int a, const int* hist, const double* beta) {
    if (E.sel_hist_out)
        for (int i = threadIdx.x; i < HB; i += blockDim.x) E.sel_hist_out[(size_t)a * HB + i] = hist[i];
    if (E.centres_out)
        for (int k = threadIdx.x; k < E.n_mask; k += blockDim.x) E.centres_out[(size_t)a * E.n_mask + k] = beta[k];
}

constexpr int SEL_NT = 1024;
constexpr int SEL_ROWS = HROWS;       // the histogram as rows of 32 bins (one per lane)
constexpr int SEL_SMALL = SEL_CAP / (2 * MAXM);   // candidates ranked directly per target bin (48)
constexpr int SEL_DIG = 11;            // bits per radix-refinement level
constexpr int SEL_HB = 1 << SEL_DIG;   // digit histogram bins (2 per thread)
static_assert(SEL_HB == 2 * SEL_NT, "two digits per thread in the refinement scan");
static_assert(2 * SEL_HB * 4 + SEL_SMALL * 8 <= SEL_CAP * 8, "refinement scratch fits the candidate arrays");
constexpr int SEL_CHEB = cheb_size(MAXM, MAXM - 1);   // the largest fit tables (doubles, shared memory)
constexpr int SEL_LPT = 8;             // centre-ray bins loaded per thread at a time
// dynamic shared memory of k_select_fit: candidates, bitmap, the fit tables
constexpr int SEL_SMEM = SEL_CAP * 16 + HB / 8 + SEL_CHEB * 8;

// 8-byte asynchronous global -> shared copy (both addresses 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Order-preserving 64-bit image of a double (-0 taken as +0): a < b iff key(a) < key(b).
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// One CTA per (evaluation, axis).  Dynamic shared memory:
//   double ck[SEL_CAP]; int ci[SEL_CAP]; unsigned bitmap[HB/32]; uint32_t cw[SEL_CAP];
// Histogram entries are ray counts, or weight sums for a weighted grid; ranks run
// over the weight-expanded sample (W = total weight).
__global__ void __launch_bounds__(SEL_NT) k_select_fit(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int a = blockIdx.x - B.tile0[ev];          // axis
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double* ck = reinterpret_cast<double*>(smem_raw);
    int* ci = reinterpret_cast<int*>(ck + SEL_CAP);
    unsigned* bitmap = reinterpret_cast<unsigned*>(ci + SEL_CAP);
    uint32_t* cwc = reinterpret_cast<uint32_t*>(bitmap + HB / 32);
    double* chb = reinterpret_cast<double*>(cwc + SEL_CAP);      // [SEL_CHEB] the fit's tables
    __shared__ double mom[6];
    __shared__ double sig[4];
    __shared__ int rowoff[SEL_ROWS + 1];
    __shared__ int wtot[SEL_NT / 32];
    __shared__ int t_bin[2 * MAXM], t_below[2 * MAXM], t_rank[2 * MAXM], t_slot[2 * MAXM];
    __shared__ int d_bin[2 * MAXM], d_num[2 * MAXM];
    __shared__ int n_d, big_sh;
    __shared__ double Qs[MAXM];
    __shared__ double coef[MAXM];
    __shared__ double Xs[MAXM + 2], Ps[MAXM + 2];
    __shared__ double selv[2 * MAXM];        // the selected order statistics
    __shared__ int flag_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int N = E.n_mask, M = E.n_nodes, D = E.degree, K = M + 2;
    const int W = E.wtot;                            // ranks of the (weight-expanded) sample

    // the fit's tables (Chebyshev nodes, C, V, V') copied into shared memory
    // asynchronously while the histogram is scanned
    const int ncheb = cheb_size(M, D);
    const bool chb_ok = ncheb <= SEL_CHEB;
    if (chb_ok) {
        for (int i = tid; i < ncheb; i += SEL_NT) cp_async8(chb + i, E.cheb + i);
        cp_async_commit();
    }
    // this axis's row counts, two per thread (scanned below)
    static_assert(SEL_ROWS == 2 * SEL_NT, "two rows per thread");
    const int* hrow = E.hist + 2 * HB + a * HROWS;
    const int r0 = __ldcg(hrow + 2 * tid), r1 = __ldcg(hrow + 2 * tid + 1);
    if (tid < 6) mom[tid] = __ldcg(E.mom + tid);
    // the two axes' standard deviations and their inverses on two warps (FP64 divides
    // and roots are long dependent chains on this part)
    if (tid == 0 || tid == 32) {
        const int q = tid >> 5;
        const double sq = sqrt(__ldcg(E.mom + 6 + q) / N);
        sig[q] = sq;
        sig[2 + q] = 1.0 / sq;
    }
    if (tid == 64) { flag_sh = 0; big_sh = 0; }
    __syncthreads();
    // sigma_min, tie -> x (App. C i); the two are positive, so their bit patterns
    // order as they do (an integer compare: an FP64 one executed by all 32 warps
    // would queue 32 instructions on the SM's FP64 pipe)
    const bool sxmin = __double_as_longlong(sig[0]) <= __double_as_longlong(sig[1]);
    const double sigma = sxmin ? sig[0] : sig[1], isig = sxmin ? sig[2] : sig[3];
    double* tr = E.trd;
    const int* hist = E.hist + a * HB;
    const double* beta = E.beta + a * N;
    const double lo = mom[2 + 2 * a];
    export_selection(E, a, hist, beta);
    for (int i = tid; i < 2 * MAXM; i += SEL_NT) d_num[i] = 0;
    for (int i = tid; i < HB / 32; i += SEL_NT) bitmap[i] = 0u;
    if (chb_ok) cp_async_wait();
    __syncthreads();
    const double* cb = chb_ok ? chb : E.cheb;
    // exclusive scan of the row counts (k_centre_hist kept them beside the bins): two
    // rows per thread, warp scans, warp totals
    const int own = r0 + r1;
    int incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int v = wtot[lane];
        int wi = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wtot[lane] = wi - v;
        if (lane == 31) rowoff[SEL_ROWS] = wi;
    }
    __syncthreads();
    {
        const int ex = wtot[wid] + incl - own;
        rowoff[2 * tid] = ex;
        rowoff[2 * tid + 1] = ex + r0;
    }
    // target ranks: node j -> floor(u_j (N-1)) and the next one (RTU grid); the
    // smallest and largest ray (uniform grid: the square box, Sec. 2.1)
    const int nt = E.transform == RTU_TRANSFORM_UNIFORM ? 2 : 2 * M;
    for (int t = tid; t < nt; t += SEL_NT) {
        int k;
        if (E.transform == RTU_TRANSFORM_UNIFORM) {
            k = t == 0 ? 0 : W - 1;
        } else {
            double h = cb[cheb_u(M, D) + t / 2] * (W - 1);
            k = (int)floor(h);
            k = k < 0 ? 0 : (k > W - 1 ? W - 1 : k);
            if (t & 1) k = k + 1 > W - 1 ? W - 1 : k + 1;
        }
        t_rank[t] = k;
    }
    for (int t = nt + tid; t < 2 * MAXM; t += SEL_NT) E.sel_idx[a * 2 * MAXM + t] = -1;
    __syncthreads();
    // the bin of each target rank: one warp per target -- the 64-row section, the
    // row, then the bin inside the row by a warp scan of its 32 counts
    for (int t = wid; t < nt; t += SEL_NT / 32) {
        const int r = t_rank[t];
        constexpr int SEC = SEL_ROWS / 32;
        const unsigned m1 = __ballot_sync(0xffffffffu, rowoff[lane * SEC] <= r && r < rowoff[lane * SEC + SEC]);
        const int sec = __ffs(m1) - 1;
        const int ra = sec * SEC + 2 * lane;
        const unsigned m2 = __ballot_sync(0xffffffffu, rowoff[ra] <= r && r < rowoff[ra + 2]);
        const int rr = sec * SEC + 2 * (__ffs(m2) - 1);
        const int row = r < rowoff[rr + 1] ? rr : rr + 1;
        const int v = hist[row * 32 + lane];
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int ex = rowoff[row] + inc - v;
        const unsigned m3 = __ballot_sync(0xffffffffu, ex <= r && r < ex + v);
        if (lane == __ffs(m3) - 1) {
            t_bin[t] = row * 32 + lane;
            t_below[t] = ex;
        }
    }
    __syncthreads();
    if (wid == 0) {
        // distinct target bins (ranks are non-decreasing, so are their bins): a new bin
        // where it differs from the previous target's; slots by a running ballot count
        int base = 0;
        for (int t0 = 0; t0 < nt; t0 += 32) {
            const int t = t0 + lane;
            const bool isnew = t < nt && (t == 0 || t_bin[t] != t_bin[t - 1]);
            const unsigned nb = __ballot_sync(0xffffffffu, isnew);
            const int slot = base + __popc(nb & ((2u << lane) - 1u)) - 1;
            if (t < nt) {
                t_slot[t] = slot;
                if (isnew) {
                    d_bin[slot] = t_bin[t];
                    atomicOr(&bitmap[t_bin[t] >> 5], 1u << (t_bin[t] & 31));
                }
            }
            base += __popc(nb);
        }
        if (lane == 0) n_d = base;
    }
    for (int t = tid; t < nt; t += SEL_NT) selv[t] = lo;     // overwritten by the selection
    __syncthreads();
    const int nd = n_d;
    // candidates of the target bins, in one pass over the centre rays: each is counted
    // in its bin and, while the bin has at most SEL_SMALL, kept in the bin's segment of
    // SEL_SMALL slots.  A bin of at most SEL_SMALL candidates has its targets ranked
    // there; a larger one is resolved below by radix refinement (so the selection is
    // exact whatever the distribution: one far outlier can squeeze most rays into a
    // few level-1 bins).  SEL_LPT bins per thread are loaded at a time, then the
    // positions of the hits.
    static_assert(2 * MAXM * SEL_SMALL <= SEL_CAP, "a segment per distinct bin");
    const int* cbin = E.cbin + (size_t)a * N;    // the bins k_centre_hist used
    for (int k0 = 0; k0 < N; k0 += SEL_NT * SEL_LPT) {
        int bn[SEL_LPT];
#pragma unroll
        for (int u = 0; u < SEL_LPT; ++u) {
            const int k = k0 + u * SEL_NT + tid;
            bn[u] = k < N ? __ldcg(cbin + k) : -1;
        }
        double bv[SEL_LPT];
#pragma unroll
        for (int u = 0; u < SEL_LPT; ++u) {
            const bool hit = bn[u] >= 0 && (bitmap[bn[u] >> 5] & (1u << (bn[u] & 31)));
            if (!hit) bn[u] = -1;
            bv[u] = hit ? __ldcg(beta + k0 + u * SEL_NT + tid) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < SEL_LPT; ++u) {
            if (bn[u] < 0) continue;
            const int k = k0 + u * SEL_NT + tid;
            // the bin's slot (the distinct bins increase)
            int d = 0, dh = nd - 1;
            while (d < dh) {
                const int mid = (d + dh) >> 1;
                if (d_bin[mid] < bn[u]) d = mid + 1;
                else dh = mid;
            }
            const int at = atomicAdd(&d_num[d], 1);
            if (at < SEL_SMALL) {
                const int o = d * SEL_SMALL + at;
                ck[o] = bv[u];
                ci[o] = k;
                cwc[o] = E.cwt ? E.cwt[k] : 1u;
            }
        }
    }
    __syncthreads();
    // the element covering rank (r - below) of its bin: candidates ordered by
    // (value, index), each covering as many ranks as its weight (at most SEL_SMALL
    // candidates: two per lane, each compared with all)
    for (int t = wid; t < nt; t += SEL_NT / 32) {
        const int d = t_slot[t];
        if (d_num[d] > SEL_SMALL) {
            if (lane == 0) big_sh = 1;
            continue;
        }
        const int o = d * SEL_SMALL, cnt = d_num[d];
        const int want = t_rank[t] - t_below[t];
        for (int c = lane; c < cnt; c += 32) {
            const double kc = ck[o + c];
            const int ic = ci[o + c];
            int rank = 0;
            for (int c2 = 0; c2 < cnt; ++c2) {
                const double k2 = ck[o + c2];
                if ((k2 < kc) || (k2 == kc && ci[o + c2] < ic)) rank += (int)cwc[o + c2];
            }
            if (rank <= want && want < rank + (int)cwc[o + c]) {
                E.sel_idx[a * 2 * MAXM + t] = ic;
                selv[t] = kc;
            }
        }
    }
    __syncthreads();
    // Targets in a bin of more than SEL_SMALL candidates, one at a time by the whole
    // CTA: MSD radix selection on the key (order-preserving 64-bit image of the value,
    // then the ray index among equal values), SEL_DIG bits per level starting at the
    // highest bit in which the candidates' keys differ.  Each level reads the candidates
    // once for their key range and once for a histogram of the next digit (counts and
    // weights), keeps the digit holding the wanted rank, and stops when at most
    // SEL_SMALL candidates remain, which are ranked like the small bins.  Scratch: the
    // candidate arrays (the small bins are done).  Skipped (a uniform branch) when
    // every target bin was small.
    if (big_sh) {
        int* hc = reinterpret_cast<int*>(ck);                 // [SEL_HB] counts
        int* hw = hc + SEL_HB;                                // [SEL_HB] weights
        double* fv = ck + SEL_HB;                             // [SEL_SMALL] final candidates
        int* fi = ci;
        uint32_t* fw = cwc;
        __shared__ unsigned long long r_pfx, r_mn, r_mx, r_keq;
        __shared__ int r_psh, r_stage, r_want, r_cnt, r_fn, r_done;
        for (int t = 0; t < nt; ++t) {
            const int d = t_slot[t];
            if (d_num[d] <= SEL_SMALL) continue;
            const int b = t_bin[t];
            if (tid == 0) {
                r_want = t_rank[t] - t_below[t];
                r_cnt = d_num[d];
                r_stage = 0;
                r_psh = 64;
                r_pfx = 0ull;
                r_done = 0;
            }
            __syncthreads();
            for (int lev = 0; lev < 16 && !r_done; ++lev) {
                const bool gather = r_cnt <= SEL_SMALL;
                const int stage = r_stage, psh = r_psh;
                const unsigned long long pfx = r_pfx, keq = r_keq;
                if (tid == 0) { r_mn = ~0ull; r_mx = 0ull; r_fn = 0; }
                __syncthreads();
                // pass 1: the key range of the candidates (and, when few remain, the candidates)
                unsigned long long mn = ~0ull, mx = 0ull;
                for (int k = tid; k < N; k += SEL_NT) {
                    if (cbin[k] != b) continue;
                    const unsigned long long key = order_key(beta[k]);
                    const unsigned long long kk = stage == 0 ? key : (unsigned long long)k;
                    if (stage == 1 && key != keq) continue;
                    if (psh < 64 && (kk >> psh) != pfx) continue;
                    mn = kk < mn ? kk : mn;
                    mx = kk > mx ? kk : mx;
                    if (gather) {
                        const int at = atomicAdd(&r_fn, 1);
                        if (at < SEL_SMALL) {
                            fv[at] = beta[k];
                            fi[at] = k;
                            fw[at] = E.cwt ? E.cwt[k] : 1u;
                        }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mn, o);
                    const unsigned long long x2 = __shfl_xor_sync(0xffffffffu, mx, o);
                    mn = m2 < mn ? m2 : mn;
                    mx = x2 > mx ? x2 : mx;
                }
                if (lane == 0) { atomicMin(&r_mn, mn); atomicMax(&r_mx, mx); }
                __syncthreads();
                if (gather) {
                    if (wid == 0) {
                        const int cnt = min(r_fn, SEL_SMALL), want = r_want;
                        for (int c = lane; c < cnt; c += 32) {
                            const double kc = fv[c];
                            const int ic = fi[c];
                            int rank = 0;
                            for (int c2 = 0; c2 < cnt; ++c2)
                                if ((fv[c2] < kc) || (fv[c2] == kc && fi[c2] < ic)) rank += (int)fw[c2];
                            if (rank <= want && want < rank + (int)fw[c]) {
                                E.sel_idx[a * 2 * MAXM + t] = ic;
                                selv[t] = kc;
                            }
                        }
                        if (lane == 0) r_done = 1;
                    }
                    __syncthreads();
                    break;
                }
                const unsigned long long lo_k = r_mn, hi_k = r_mx;
                if (lo_k == hi_k) {
                    // equal values: the rank runs over the ray index among them
                    if (tid == 0) { r_stage = 1; r_keq = lo_k; r_psh = 64; r_pfx = 0ull; }
                    __syncthreads();
                    continue;
                }
                const int hb = 63 - __clzll((long long)(lo_k ^ hi_k));
                const int sh = hb - (SEL_DIG - 1) > 0 ? hb - (SEL_DIG - 1) : 0;
                for (int i = tid; i < 2 * SEL_HB; i += SEL_NT) hc[i] = 0;
                __syncthreads();
                // pass 2: histogram of the digit below the common prefix
                for (int k = tid; k < N; k += SEL_NT) {
                    if (cbin[k] != b) continue;
                    const unsigned long long key = order_key(beta[k]);
                    const unsigned long long kk = stage == 0 ? key : (unsigned long long)k;
                    if (stage == 1 && key != keq) continue;
                    if (psh < 64 && (kk >> psh) != pfx) continue;
                    const int dg = (int)((kk >> sh) & (SEL_HB - 1));
                    atomicAdd(&hc[dg], 1);
                    atomicAdd(&hw[dg], E.cwt ? (int)E.cwt[k] : 1);
                }
                __syncthreads();
                // the digit holding the wanted rank: exclusive scan of the weights, two
                // digits per thread
                {
                    const int w0 = hw[2 * tid], w1 = hw[2 * tid + 1];
                    int inc = w0 + w1;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (lane == 31) wtot[wid] = inc;
                    __syncthreads();
                    int base = 0;
                    for (int i = 0; i < wid; ++i) base += wtot[i];
                    const int e0 = base + inc - w0 - w1, e1 = e0 + w0, want = r_want;
                    int hit = -1, below = 0;
                    if (w0 > 0 && e0 <= want && want < e1) { hit = 2 * tid; below = e0; }
                    if (w1 > 0 && e1 <= want && want < e1 + w1) { hit = 2 * tid + 1; below = e1; }
                    __syncthreads();
                    if (hit >= 0) {
                        r_want = want - below;
                        r_cnt = hc[hit];
                        r_pfx = ((lo_k >> sh) & ~(unsigned long long)(SEL_HB - 1)) | (unsigned long long)hit;
                        r_psh = sh;
                    }
                }
                __syncthreads();
            }
            if (tid == 0 && !r_done) flag_sh |= F_SELECT;      // not reached: at most 8 levels
            __syncthreads();
        }
    }
    if (E.transform == RTU_TRANSFORM_UNIFORM) {
        // uniform grid: the smallest square box around the masked rays, centred on
        // each axis's range, mapped affinely onto [0, 1]^2 -- written as Hermite
        // knots X_j = (lo + U_j L - mu)/sigma with equal slopes sigma/L (linear).
        // The ranges are the order statistics of ranks 0 and N-1 (= min, max).
        const double r0x = mom[3] - mom[2], r1y = mom[5] - mom[4];
        const double L = r0x >= r1y ? r0x : r1y;
        const double mn = mom[2 + 2 * a], mx = mom[3 + 2 * a];
        const double lo_a = 0.5 * (mn + mx) - 0.5 * L;
        for (int j = tid; j < K; j += SEL_NT) {
            const double U = j == 0 ? 0.0 : (j == K - 1 ? 1.0 : cb[cheb_u(M, D) + j - 1]);
            const double X = (lo_a + U * L - mom[a]) * isig;
            tr[TR_HDR + a * K + j] = X;
            tr[TR_HDR + (6 + a) * K + j] = X;
            tr[TR_HDR + (2 + a) * K + j] = sigma / L;
            tr[TR_HDR + (4 + a) * K + j] = L * isig;
        }
        if (a == 0 && tid == 0) {
            tr[0] = mom[0]; tr[1] = mom[1]; tr[2] = sigma; tr[3] = sxmin ? 0.0 : 1.0; tr[4] = K;
            tr[5] = r0x >= r1y ? 0.0 : 1.0; tr[6] = L;
        }
    } else {
        // empirical QF at the nodes in standardized coordinates (type-7 interpolation)
        for (int j = tid; j < M; j += SEL_NT) {
            const double h = cb[cheb_u(M, D) + j] * (W - 1);
            const double frac = h - floor(h);
            const double zl = (selv[2 * j] - mom[a]) * isig;
            const double zh = (selv[2 * j + 1] - mom[a]) * isig;
            Qs[j] = zl + frac * (zh - zl);
        }
        __syncthreads();
        // App. C iii: Chebyshev coefficients of the QF from M = D+1 nodes by the
        // discrete orthogonality of T_k on the nodes: c = C Q (one thread per coefficient)
        const double* Ct = cb + cheb_C(M, D);
        for (int k = tid; k <= D; k += SEL_NT) {
            double sacc = 0.0;
            for (int j = 0; j < M; ++j) sacc += Ct[k * M + j] * Qs[j];
            coef[k] = sacc;
        }
        __syncthreads();
        // App. C iv: knots p(0), p(u_j), p(1) and p'(u) there (one thread per point),
        // the slope floor of the guard and the slopes 1/p' (per point)
        const double* Vt = cb + cheb_V(M, D);
        const double* dVt = cb + cheb_dV(M, D);
        for (int j = tid; j < K; j += SEL_NT) {
            double p = 0.0, d = 0.0;
            for (int k = 0; k <= D; ++k) {
                p += Vt[j * (D + 1) + k] * coef[k];
                d += dVt[j * (D + 1) + k] * coef[k];
            }
            Xs[j] = p;
            Ps[j] = d;
            tr[TR_HDR + (6 + a) * K + j] = p;       // raw knots
            tr[TR_HDR + (4 + a) * K + j] = d;       // raw p'
        }
        __syncthreads();
        // monotonicity guard (App. C iv): p' >= 1e-6 span per point (in parallel),
        // strictly increasing knots (sequential in the knots, one thread).  By warp 0
        // alone: FP64 instructions of all 32 warps would queue on the SM's FP64 pipe.
        if (wid == 0) {
            double span = Xs[K - 1] - Xs[0];
            const bool span_ok = span > 0.0;
            if (!span_ok) span = fabs(span) + 1e-300;
            const double floor_d = 1e-6 * span;
            if (!span_ok && lane == 0) atomicOr(&flag_sh, F_NONMONO);
            for (int j = lane; j < K; j += 32) {
                double dp = Ps[j];
                if (dp < floor_d) { dp = floor_d; atomicOr(&flag_sh, F_NONMONO); }
                tr[TR_HDR + (2 + a) * K + j] = 1.0 / dp;
            }
            // when no fitted knot is below its predecessor + floor (checked by one warp
            // in parallel) all stay as fitted; else they are raised in order by one lane
            bool low = false;
            for (int j = 1 + lane; j < K; j += 32) low |= Xs[j] < Xs[j - 1] + floor_d;
            if (!__any_sync(0xffffffffu, low)) {
                for (int j = lane; j < K; j += 32) tr[TR_HDR + a * K + j] = Xs[j];
            } else if (lane == 0) {
                int fl = 0;
                double prev = Xs[0];
                tr[TR_HDR + a * K] = prev;
                for (int j = 1; j < K; ++j) {
                    double x = Xs[j];
                    const double lim = prev + floor_d;
                    if (x < lim) { x = lim; fl |= F_NONMONO; }
                    tr[TR_HDR + a * K + j] = x;
                    prev = x;
                }
                if (fl) atomicOr(&flag_sh, fl);
            }
        }
        for (int k = tid; k <= D; k += SEL_NT) tr[TR_HDR + 8 * K + a * MAXM + k] = coef[k];
        for (int j = tid; j < M; j += SEL_NT) tr[TR_HDR + 8 * K + 2 * MAXM + a * MAXM + j] = Qs[j];
        if (a == 0 && tid == 0) {
            tr[0] = mom[0]; tr[1] = mom[1]; tr[2] = sigma; tr[3] = sxmin ? 0.0 : 1.0; tr[4] = K;
        }
    }
    __syncthreads();
    // float copy of this axis's knots and slopes (and the header) for the float
    // render path, the optional CDF output, flags
    for (int j = tid; j < K; j += SEL_NT) {
        E.trf[TR_HDR + a * K + j] = (float)tr[TR_HDR + a * K + j];
        E.trf[TR_HDR + (2 + a) * K + j] = (float)tr[TR_HDR + (2 + a) * K + j];
    }
    if (a == 0)
        for (int i = tid; i < TR_HDR; i += SEL_NT) E.trf[i] = (float)tr[i];
    if (E.cdf_out) {
        if (a == 0)
            for (int i = tid; i < 3; i += SEL_NT) E.cdf_out[i] = tr[i];
        for (int j = tid; j < K; j += SEL_NT) {
            E.cdf_out[3 + a * K + j] = tr[TR_HDR + a * K + j];
            E.cdf_out[3 + (2 + a) * K + j] = tr[TR_HDR + (2 + a) * K + j];
        }
    }
    if (tid == 0 && flag_sh) atomicOr(E.flags, flag_sh);
    // the last of the evaluation's two CTAs to finish (an atomic counter after a fence)
    // tests every render tile against the grid's reach, reading the other axis's float
    // transform through L2: k_render reads one byte per tile
    __shared__ int last_sf;
    __shared__ float reach[4];
    __threadfence();
    __syncthreads();
    if (tid == 0) last_sf = atomicAdd(E.ccnt + 3, 1) == 1;
    __syncthreads();
    if (!last_sf) return;
    if (tid == 0) {
        grid_reach(E, true, reach);
        E.ccnt[3] = 0;
    }
    __syncthreads();
    for (int t = tid; t < E.n_cta_r; t += SEL_NT) E.tcull[t] = tile_out_of_reach(E, t, reach) ? 1 : 0;
}

// ------------------------------------------------ the unsmoothed eCDF transform
// App. C (first paragraph): the k-th smallest centre ray of an axis maps to
// k/(n-1), linearly in between and with the end segments' slopes beyond.  The map
// commutes with the standardisation of step i, so the observations are kept as raw
// source-plane positions (mu = 0, sigma = 1 in the transform header).
//
// One CTA per (evaluation, axis): the level-1 histogram (every ray once, bins over
// [min, max]) becomes a counting sort -- exclusive scan in place, scatter through
// the bin cursors (afterwards hist[b] is the end of bin b), then each bin's few
// rays sorted by (position, ray index), a total order, so the result does not
// depend on the scatter's arrival order.  Writes the sorted positions (double and
// float hi + lo), the ray at each rank, the rank of each ray, and a transform
// header the render kernels read like the Hermite one: end knots X_0 = first and
// X_{K-1} = last observation with the end-segment slopes (the reach of the grid),
// plus the bin origin and scale of the histogram for the renderers' bin lookup.
constexpr int LIN_NT = 1024;
__global__ void __launch_bounds__(LIN_NT) k_lin_sort(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int a = blockIdx.x - B.tile0[ev];
    const int N = E.n_mask, K = E.n_nodes + 2, tid = threadIdx.x;
    __shared__ double mom[6];
    __shared__ double sig[2];
    __shared__ int wtot[LIN_NT / 32];
    if (tid < 6) mom[tid] = __ldcg(E.mom + tid);
    if (tid == 0) {
        const double sx = sqrt(__ldcg(E.mom + 6) / N), sy = sqrt(__ldcg(E.mom + 7) / N);
        sig[0] = sx <= sy ? sx : sy;            // sigma_min, tie -> x (App. C i)
        sig[1] = sx <= sy ? 0.0 : 1.0;
    }
    __syncthreads();
    int* h = E.hist + a * HB;
    export_selection(E, a, h, E.beta + (size_t)a * N);
    __syncthreads();
    // exclusive scan of the HB bin counts, in place: warp w owns the contiguous segment
    // [w SEG, (w+1) SEG) and walks it in 32-bin chunks (coalesced); segment totals,
    // then their exclusive scan, then each warp rescans its segment with its offset
    {
        constexpr int SEG = HB / (LIN_NT / 32);
        const int lane = tid & 31, w = tid >> 5;
        int* hs = h + w * SEG;
        int tot = 0;
        for (int c = 0; c < SEG; c += 32) tot += hs[c + lane];
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
        if (lane == 0) wtot[w] = tot;
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int i = 0; i < LIN_NT / 32; ++i) { const int t = wtot[i]; wtot[i] = acc; acc += t; }
        }
        __syncthreads();
        int carry = wtot[w];
        for (int c = 0; c < SEG; c += 32) {
            const int v = hs[c + lane];
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            hs[c + lane] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    // scatter through the bin cursors (the bins k_centre_hist used)
    const double lo = mom[2 + 2 * a], sc = bin_scale(mom[2 + 2 * a], mom[3 + 2 * a]);
    double* key = E.lkey + (size_t)a * N;
    int* idx = E.lidx + (size_t)a * N;
    for (int i = tid; i < N; i += LIN_NT) {
        const double b = E.beta[(size_t)a * N + i];
        const int pos = atomicAdd(h + E.cbin[(size_t)a * N + i], 1);
        if (pos < N) { key[pos] = b; idx[pos] = i; }
    }
    __syncthreads();
    // sort inside each bin by (position, ray index): insertion sort, one thread per bin
    for (int bin = tid; bin < HB; bin += LIN_NT) {
        const int e = min(h[bin], N), s0 = bin ? min(h[bin - 1], N) : 0;
        for (int i = s0 + 1; i < e; ++i) {
            const double kv = key[i];
            const int iv = idx[i];
            int j = i - 1;
            while (j >= s0 && (key[j] > kv || (key[j] == kv && idx[j] > iv))) {
                key[j + 1] = key[j];
                idx[j + 1] = idx[j];
                --j;
            }
            key[j + 1] = kv;
            idx[j + 1] = iv;
        }
    }
    __syncthreads();
    float2* kf = reinterpret_cast<float2*>(E.lkf) + (size_t)a * N;
    for (int j = tid; j < N; j += LIN_NT) {
        const double v = key[j];
        const float hi = (float)v;
        kf[j] = make_float2(hi, (float)(v - (double)hi));
        E.lrank[(size_t)a * N + idx[j]] = j;
    }
    // transform header: mu = 0, sigma = 1; end knots and end-segment slopes; the
    // interior knots are spread evenly between them (unused by the linear map)
    double* tr = E.trd;
    const double x0 = key[0], x1 = key[N - 1];
    const double hl = key[1] - key[0], hr = key[N - 1] - key[N - 2];
    const double dl = hl > 0.0 ? 1.0 / ((N - 1) * hl) : 0.0;
    const double dr = hr > 0.0 ? 1.0 / ((N - 1) * hr) : 0.0;
    for (int j = tid; j < K; j += LIN_NT) {
        const double X = j == K - 1 ? x1 : x0 + (x1 - x0) * ((double)j / (K - 1));
        const double d = j == 0 ? dl : (j == K - 1 ? dr : 1.0 / (x1 - x0 > 0.0 ? x1 - x0 : 1.0));
        tr[TR_HDR + a * K + j] = X;
        tr[TR_HDR + (2 + a) * K + j] = d;
        E.trf[TR_HDR + a * K + j] = (float)X;
        E.trf[TR_HDR + (2 + a) * K + j] = (float)d;
    }
    if (tid == 0) {
        tr[TR_HDR + 6 * K + a] = lo;
        tr[TR_HDR + 6 * K + 2 + a] = sc;
        E.trf[TR_HDR + 6 * K + a] = (float)lo;
        E.trf[TR_HDR + 6 * K + 2 + a] = (float)sc;
    }
    if (a == 0 && tid < TR_HDR) {
        const double v = tid == 2 ? 1.0 : (tid == 4 ? (double)N : 0.0);
        tr[tid] = v;
        E.trf[tid] = (float)v;
    }
    // CDF output: the standardisation (App. C i); knots and slopes are not used
    if (E.cdf_out) {
        if (a == 0 && tid < 3) E.cdf_out[tid] = tid < 2 ? mom[tid] : sig[0];
        for (int j = tid; j < K; j += LIN_NT) {
            E.cdf_out[3 + a * K + j] = 0.0;
            E.cdf_out[3 + (2 + a) * K + j] = 0.0;
        }
    }
}

}  // namespace rtu
