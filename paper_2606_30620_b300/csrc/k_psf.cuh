// k_psf.cuh -- S8: PSF convolution ('same', zero padding) fused with the
// Gaussian residual and the likelihood partial sums (Sec. 3.1, Sec. 4); its
// adjoint (correlation with the PSF); the per-evaluation final reductions (by the
// likelihood kernel's last CTA).
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

constexpr int PSF_NT = PSF_T * PSF_T / 4;   // each thread: 4 horizontally adjacent outputs
constexpr int PSF_MAXK = 31;
constexpr int PSF_IN = PSF_T + PSF_MAXK - 1;

__device__ __forceinline__ double warp_rows_sum_cg(const double* a, int rows, size_t stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int t = lane; t < rows; t += 32) s += __ldcg(a + (size_t)t * stride);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return __shfl_sync(0xffffffffu, s, 0);
}

// The end of the forward, run by the last CTA of the likelihood kernel to finish
// (any block of at least 64 threads): log L = -1/2 sum r^2 - N log(sigma sqrt(2 pi)),
// chi^2_img = sum_mask r^2 / N_mask, N_in_grid, flags, the ray histogram.  The per-tile
// partials were written by the other CTAs: read through L2.
__device__ void like_final_cta(const EvalArgs& E) {
    __shared__ int red_i[32];
    __shared__ double sums[2];
    int cnt = 0;
    for (int t = threadIdx.x; t < E.n_cta_r; t += blockDim.x) cnt += __ldcg(E.cta_cnt + t);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red_i[threadIdx.x >> 5] = cnt;
    // the per-tile sums of r^2 (all pixels) and of r^2 in the mask: warps 0 and 1,
    // lane-strided, fixed tree
    if (threadIdx.x < 64) {
        const double v = warp_rows_sum_cg(E.lpart + (threadIdx.x >> 5), E.n_cta_p, 2);
        if ((threadIdx.x & 31) == 0) sums[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0 && E.stats) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += red_i[w];
        E.stats[4] = tot;
        const double npx = (double)E.n_img * E.n_img;
        E.stats[0] = -0.5 * sums[0] - npx * log(E.sigma * sqrt(2.0 * 3.14159265358979323846));
        E.stats[1] = sums[1] / (E.n_mask > 0 ? E.n_mask : 1);
        E.stats[2] = E.n_mask;
        E.stats[3] = (double)(*E.flags);
    }
    if (E.hist_out) {
        const int nc = (E.n_src - 1) * (E.n_src - 1);
        for (int i = threadIdx.x; i < nc; i += blockDim.x) E.hist_out[i] = __ldcg(E.ccount + i);
    }
    if (threadIdx.x == 0) E.ccnt[2] = 0;
}

// after a CTA's likelihood partials: the last CTA of the evaluation finishes the forward
__device__ __forceinline__ void like_last_cta(const EvalArgs& E) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(E.ccnt + 2, 1) == E.n_cta_p - 1;
    __syncthreads();
    if (last) like_final_cta(E);
}

// The CTA's two likelihood partials (sum r^2, sum over the mask) from per-thread
// values: a warp tree (compensated pairs for float), the warps' pairs combined in
// order by two threads, then one conversion to double each.  (Every FP64
// instruction takes a slot of the SM's FP64 pipe for the whole warp, however few of
// its lanes are active, so the pairs stay in the kernel's type until the end.)  The
// double path's pairs carry a zero low part: the same sums as adding doubles in order.
template <typename T, int NT>
__device__ __forceinline__ void like_cta_partials(const EvalArgs& E, int tile, T r2t, T r2mt) {
    typedef decltype(warp_pair_sum(T(0))) P;
    __shared__ P red[2][NT / 32];
    const P p0 = warp_pair_sum(r2t), p1 = warp_pair_sum(r2mt);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = p0; red[1][threadIdx.x >> 5] = p1; }
    __syncthreads();
    if (threadIdx.x < 2) {
        P r = red[threadIdx.x][0];
        for (int w = 1; w < NT / 32; ++w) pair_add(r, red[threadIdx.x][w]);
        E.lpart[tile * 2 + threadIdx.x] = (double)r.x + (double)r.y;
        __threadfence();
    }
}

__device__ __forceinline__ void psf_tile_of(const EvalArgs& E, int tile, int& ti, int& tj) {
    const int nt = (E.n_img + PSF_T - 1) / PSF_T;
    tj = tile / nt;
    ti = tile - tj * nt;
}

// m[j,i] = sum_{b,a} psf[b,a] img[j-(b-c), i-(a-c)];  resid = (d - m)/sigma^2;
// per-CTA sums of r^2 (all pixels) and r^2 in the mask, r = (d - m)/sigma.
// Each thread computes 4 adjacent outputs with a sliding register window over a
// shared-memory input tile (K + 3 shared loads per 4 K fused multiply-adds).
template <typename T>
__global__ void __launch_bounds__(PSF_NT) k_psf_like(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ T in[PSF_IN][PSF_IN + 1];
    __shared__ T kp[PSF_MAXK * PSF_MAXK];
    __shared__ double red[2][PSF_NT / 32];
    const int K = E.psf_k, c = (K - 1) / 2, n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    const T* img = reinterpret_cast<const T*>(E.img);
    const T* psf = reinterpret_cast<const T*>(E.psf);
    for (int w = threadIdx.x; w < K * K; w += PSF_NT) kp[w] = psf[w];
    const int W = PSF_T + 2 * c;
    for (int w = threadIdx.x; w < W * W; w += PSF_NT) {
        const int r = w / W, q = w - r * W;
        const int gj = j0 - c + r, gi = i0 - c + q;
        in[r][q] = (gj >= 0 && gj < n && gi >= 0 && gi < n) ? img[gj * n + gi] : T(0);
    }
    __syncthreads();
    const int tx0 = 4 * (threadIdx.x % (PSF_T / 4)), ty = threadIdx.x / (PSF_T / 4);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int b = 0; b < K; ++b) {
        const T* row = in[ty - b + 2 * c] + tx0 + 2 * c;     // row[u - a] for output u, tap a
        T v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3];
        const T* kr = kp + b * K;
        for (int a = 0; a < K; ++a) {
            const T w = kr[a];
            acc[0] += w * v0; acc[1] += w * v1; acc[2] += w * v2; acc[3] += w * v3;
            v3 = v2; v2 = v1; v1 = v0;
            v0 = a + 1 < K ? row[-(a + 1)] : T(0);
        }
    }
    const T isg = T(1) / T(E.sigma);
    double r2 = 0.0, r2m = 0.0;
    const int j = j0 + ty;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + tx0 + u;
        if (i < n && j < n) {
            const T m = acc[u];
            const T d = reinterpret_cast<const T*>(E.data)[j * n + i];
            const T r = (d - m) * isg;
            reinterpret_cast<T*>(E.resid)[j * n + i] = r * isg;
            if (E.model_out) reinterpret_cast<T*>(E.model_out)[j * n + i] = m;
            const double rr = (double)r * (double)r;
            r2 += rr;
            if (E.mask[j * n + i]) r2m += rr;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_down_sync(0xffffffffu, r2, o);
        r2m += __shfl_down_sync(0xffffffffu, r2m, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = r2; red[1][threadIdx.x >> 5] = r2m; }
    __syncthreads();
    if (threadIdx.x < 2) {
        double sacc = 0.0;
        for (int w = 0; w < PSF_NT / 32; ++w) sacc += red[threadIdx.x][w];
        E.lpart[tile * 2 + threadIdx.x] = sacc;
        __threadfence();
    }
    like_last_cta(E);
}

// ---- float path with a compile-time tap count KT (9 or 21): a PSF of K <= KT
// taps is zero-padded to KT.  128 threads per 32 x 32 output tile, 8
// horizontally adjacent outputs per thread; for every PSF row the thread loads
// 8 + KT - 1 inputs and the KT weights with 16-byte shared loads and does
// 8 KT fused multiply-adds from registers.
constexpr int PSFT_NT = 128;
template <int KT> struct PsfT {
    static constexpr int C = (KT - 1) / 2;
    static constexpr int W = PSF_T + KT - 1;          // input tile side
    static constexpr int V = 8 + KT - 1;              // inputs per thread per row
    static constexpr int VP = (V + 3) / 4 * 4;
    // row pitch >= W with P = 4 (mod 8): 16-byte aligned rows, and the two rows
    // read in one 8-thread phase of a 16-byte load fall in disjoint banks
    static constexpr int P = (W + 3) / 8 * 8 + 4;
    static constexpr int KP = (KT + 3) / 4 * 4;       // weight row pitch
};

// weights of an eval's K x K PSF centred in the KT x KT table (zeros around it),
// psf[b][a] at [b][a]; the convolution flips by indexing the input
template <int KT>
__device__ __forceinline__ void psf_weights_t(const EvalArgs& E, float* kw) {
    const int K = E.psf_k, o = (KT - K) / 2;
    const float* psf = reinterpret_cast<const float*>(E.psf);
    for (int w = threadIdx.x; w < KT * PsfT<KT>::KP; w += blockDim.x) {
        const int b = w / PsfT<KT>::KP, a = w - b * PsfT<KT>::KP;
        const int bb = b - o, aa = a - o;
        kw[w] = (a < KT && bb >= 0 && bb < K && aa >= 0 && aa < K) ? psf[bb * K + aa] : 0.0f;
    }
}

template <int KT>
__device__ __forceinline__ void psf_stage_t(const float* src, int n, int i0, int j0, float (*in)[PsfT<KT>::P]) {
    constexpr int W = PsfT<KT>::W, C = PsfT<KT>::C;
    for (int w = threadIdx.x; w < W * PsfT<KT>::P; w += PSFT_NT) {
        const int r = w / PsfT<KT>::P, q = w - r * PsfT<KT>::P;
        const int gj = j0 - C + r, gi = i0 - C + q;
        in[r][q] = (q < W && gj >= 0 && gj < n && gi >= 0 && gi < n) ? src[gj * n + gi] : 0.0f;
    }
}

// acc[u] += sum_a kw_row[a] v[u + off(a)], off(a) = KT - 1 - a (convolution) or a
// (correlation), v = the thread's inputs of one row
template <int KT, bool CONV>
__device__ __forceinline__ void psf_row_t(const float* in_row, const float* kw_row, float* acc) {
    constexpr int VP = PsfT<KT>::VP, KP = PsfT<KT>::KP;
    float v[VP], w[KP];
#pragma unroll
    for (int i = 0; i < VP / 4; ++i) {
        const float4 t = reinterpret_cast<const float4*>(in_row)[i];
        v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
#pragma unroll
    for (int i = 0; i < KP / 4; ++i) {
        const float4 t = reinterpret_cast<const float4*>(kw_row)[i];
        w[4 * i] = t.x; w[4 * i + 1] = t.y; w[4 * i + 2] = t.z; w[4 * i + 3] = t.w;
    }
#pragma unroll
    for (int a = 0; a < KT; ++a)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += w[a] * v[u + (CONV ? KT - 1 - a : a)];
}

template <int KT>
__global__ void __launch_bounds__(PSFT_NT) k_psf_like_t(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ __align__(16) float in[PsfT<KT>::W][PsfT<KT>::P];
    __shared__ __align__(16) float kw[KT * PsfT<KT>::KP];
    const int n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    psf_weights_t<KT>(E, kw);
    psf_stage_t<KT>(reinterpret_cast<const float*>(E.img), n, i0, j0, in);
    __syncthreads();
    const int tx0 = 8 * (threadIdx.x & 3), ty = threadIdx.x >> 2;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // m[j, i] = sum_{b,a} psf[b][a] in[ty + 2C - b][x + 2C - a]
#pragma unroll 1
    for (int b = 0; b < KT; ++b)
        psf_row_t<KT, true>(&in[ty + KT - 1 - b][tx0], kw + b * PsfT<KT>::KP, acc);
    const float isg = 1.0f / (float)E.sigma;
    float r2f = 0.f, r2mf = 0.f;
    const int j = j0 + ty;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + tx0 + u;
        if (i < n && j < n) {
            const float m = acc[u];
            const float d = reinterpret_cast<const float*>(E.data)[j * n + i];
            const float r = (d - m) * isg;
            reinterpret_cast<float*>(E.resid)[j * n + i] = r * isg;
            if (E.model_out) reinterpret_cast<float*>(E.model_out)[j * n + i] = m;
            r2f += r * r;
            if (E.mask[j * n + i]) r2mf += r * r;
        }
    }
    // per-thread float partials of 8 pixels
    like_cta_partials<float, PSFT_NT>(E, tile, r2f, r2mf);
    like_last_cta(E);
}

// d L / d img[p, q] = dlogL sum_{b,a} psf[b][a] resid[p + b - C, q + a - C]
template <int KT>
__global__ void __launch_bounds__(PSFT_NT) k_psf_adj_t(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ __align__(16) float in[PsfT<KT>::W][PsfT<KT>::P];
    __shared__ __align__(16) float kw[KT * PsfT<KT>::KP];
    const int n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    psf_weights_t<KT>(E, kw);
    psf_stage_t<KT>(reinterpret_cast<const float*>(E.resid), n, i0, j0, in);
    __syncthreads();
    const int tx0 = 8 * (threadIdx.x & 3), ty = threadIdx.x >> 2;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int b = 0; b < KT; ++b) psf_row_t<KT, false>(&in[ty + b][tx0], kw + b * PsfT<KT>::KP, acc);
    const float sc = E.dlogL ? (float)(*E.dlogL) : 1.0f;
    const int j = j0 + ty;
    float gm = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + tx0 + u;
        if (i < n && j < n) {
            const float g = acc[u] * sc;
            reinterpret_cast<float*>(E.gimg)[j * n + i] = g;
            gm = fmaxf(gm, fabsf(g));
        }
    }
    note_gmax(E, gm);
}

// ---- rank-1 PSF, psf[b][a] = u[b] v[a]: two one-dimensional passes over a 32 x 32
// output tile staged with its halo -- the taps v along x into a shared row buffer,
// then the taps u along y -- K + K multiply-adds per output instead of K^2.  Each
// thread computes 4 adjacent outputs of a pass from a sliding register window.
// CONV: convolution (the forward model); else correlation (its adjoint).  KT: the
// tap count when known at compile time (21, 9: the loops unroll and the window's
// shifts cost nothing), 0 for any other.
constexpr int PSFS_NT = 256;
constexpr int PSFS_W = PSF_T + PSF_MAXK - 1;

template <typename T, bool CONV, int KT>
__device__ __forceinline__ void psf_sep_passes(const EvalArgs& E, const T* src, int i0, int j0,
                                               T (*in)[PSFS_W + 1], T (*h)[PSF_T + 1], T* u, T* v, T* out4,
                                               int& ox, int& oy0) {
    const int K = KT > 0 ? KT : E.psf_k, c = (K - 1) / 2, n = E.n_img, W = PSF_T + 2 * c;
    for (int i = threadIdx.x; i < 2 * K; i += PSFS_NT) {
        const T x = (T)E.psf_uv[i];
        if (i < K) u[i] = x; else v[i - K] = x;
    }
    // the input window with its halo: rows by warp, columns by lane (no division per
    // element), each thread's loads issued before its stores
    {
        constexpr int NWS = PSFS_NT / 32, RPW = (PSFS_W + NWS - 1) / NWS;
        static_assert(PSFS_W <= 64, "two columns per lane");
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        T val[RPW][2];
#pragma unroll
        for (int k = 0; k < RPW; ++k)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = wid + k * NWS, q = lane + 32 * hh;
                const int gj = j0 - c + r, gi = i0 - c + q;
                val[k][hh] = (r < W && q < W && gj >= 0 && gj < n && gi >= 0 && gi < n) ? src[gj * n + gi] : T(0);
            }
#pragma unroll
        for (int k = 0; k < RPW; ++k)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = wid + k * NWS, q = lane + 32 * hh;
                if (r < W && q < W) in[r][q] = val[k][hh];
            }
    }
    __syncthreads();
    // along x: h[r][x] = sum_a v[a] in[r][x + 2c - a] (convolution) or in[r][x + a]
    for (int t = threadIdx.x; t < W * (PSF_T / 4); t += PSFS_NT) {
        const int r = t / (PSF_T / 4), x0 = 4 * (t - r * (PSF_T / 4));
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        if (CONV) {
            const T* row = in[r] + x0 + 2 * c;          // row[u - a] for output x0 + u
            T w0 = row[0], w1 = row[1], w2 = row[2], w3 = row[3];
#pragma unroll
            for (int a = 0; a < K; ++a) {
                const T f = v[a];
                a0 += f * w0; a1 += f * w1; a2 += f * w2; a3 += f * w3;
                w3 = w2; w2 = w1; w1 = w0;
                w0 = a + 1 < K ? row[-(a + 1)] : T(0);
            }
        } else {
            const T* row = in[r] + x0;                  // row[u + a]
            T w0 = row[0], w1 = row[1], w2 = row[2], w3 = row[3];
#pragma unroll
            for (int a = 0; a < K; ++a) {
                const T f = v[a];
                a0 += f * w0; a1 += f * w1; a2 += f * w2; a3 += f * w3;
                w0 = w1; w1 = w2; w2 = w3;
                w3 = a + 1 < K ? row[a + 4] : T(0);
            }
        }
        h[r][x0] = a0; h[r][x0 + 1] = a1; h[r][x0 + 2] = a2; h[r][x0 + 3] = a3;
    }
    __syncthreads();
    // along y: 4 adjacent rows of one column per thread (256 threads = 8 x 32)
    const int x = threadIdx.x & (PSF_T - 1), y0 = 4 * (threadIdx.x >> 5);
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    if (CONV) {
        const int base = y0 + 2 * c;                    // h[y - b + 2c]
        T w0 = h[base][x], w1 = h[base + 1][x], w2 = h[base + 2][x], w3 = h[base + 3][x];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const T f = u[b];
            a0 += f * w0; a1 += f * w1; a2 += f * w2; a3 += f * w3;
            w3 = w2; w2 = w1; w1 = w0;
            w0 = b + 1 < K ? h[base - (b + 1)][x] : T(0);
        }
    } else {
        T w0 = h[y0][x], w1 = h[y0 + 1][x], w2 = h[y0 + 2][x], w3 = h[y0 + 3][x];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const T f = u[b];
            a0 += f * w0; a1 += f * w1; a2 += f * w2; a3 += f * w3;
            w0 = w1; w1 = w2; w2 = w3;
            w3 = b + 1 < K ? h[y0 + b + 4][x] : T(0);
        }
    }
    out4[0] = a0; out4[1] = a1; out4[2] = a2; out4[3] = a3;
    ox = x;
    oy0 = y0;
}

template <typename T, int KT>
__global__ void __launch_bounds__(PSFS_NT) k_psf_like_sep(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ T in[PSFS_W][PSFS_W + 1];
    __shared__ T h[PSFS_W][PSF_T + 1];
    __shared__ T u[PSF_MAXK], v[PSF_MAXK];
    const int n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    T m4[4];
    int x, y0;
    psf_sep_passes<T, true, KT>(E, reinterpret_cast<const T*>(E.img), i0, j0, in, h, u, v, m4, x, y0);
    const T isg = T(1) / T(E.sigma);
    T r2t = T(0), r2mt = T(0);
    const int i = i0 + x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + y0 + k;
        if (i < n && j < n) {
            const T m = m4[k];
            const T d = reinterpret_cast<const T*>(E.data)[j * n + i];
            const T r = (d - m) * isg;
            reinterpret_cast<T*>(E.resid)[j * n + i] = r * isg;
            if (E.model_out) reinterpret_cast<T*>(E.model_out)[j * n + i] = m;
            r2t += r * r;
            if (E.mask[j * n + i]) r2mt += r * r;
        }
    }
    // per-thread partials of 4 pixels
    like_cta_partials<T, PSFS_NT>(E, tile, r2t, r2mt);
    like_last_cta(E);
}

template <typename T, int KT>
__global__ void __launch_bounds__(PSFS_NT) k_psf_adj_sep(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ T in[PSFS_W][PSFS_W + 1];
    __shared__ T h[PSFS_W][PSF_T + 1];
    __shared__ T u[PSF_MAXK], v[PSF_MAXK];
    const int n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    T g4[4];
    int x, y0;
    psf_sep_passes<T, false, KT>(E, reinterpret_cast<const T*>(E.resid), i0, j0, in, h, u, v, g4, x, y0);
    const T sc = E.dlogL ? (T)(*E.dlogL) : T(1);
    const int i = i0 + x;
    T gm = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + y0 + k;
        if (i < n && j < n) {
            const T g = g4[k] * sc;
            reinterpret_cast<T*>(E.gimg)[j * n + i] = g;
            gm = fmax(gm, r_abs(g));
        }
    }
    note_gmax(E, gm);
}

// log L = -1/2 sum r^2 - N log(sigma sqrt(2 pi)); chi^2_img = sum_mask r^2 / N_mask

// d L / d img[p,q] = dlogL * sum_{b,a} psf[b,a] resid[p+b-c, q+a-c]
template <typename T>
__global__ void __launch_bounds__(PSF_NT) k_psf_adj(const __grid_constant__ Batch B) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    __shared__ T in[PSF_IN][PSF_IN + 1];
    __shared__ T kp[PSF_MAXK * PSF_MAXK];
    const int K = E.psf_k, c = (K - 1) / 2, n = E.n_img;
    int ti, tj;
    psf_tile_of(E, tile, ti, tj);
    const int i0 = ti * PSF_T, j0 = tj * PSF_T;
    const T* res = reinterpret_cast<const T*>(E.resid);
    const T* psf = reinterpret_cast<const T*>(E.psf);
    for (int w = threadIdx.x; w < K * K; w += PSF_NT) kp[w] = psf[w];
    const int W = PSF_T + 2 * c;
    for (int w = threadIdx.x; w < W * W; w += PSF_NT) {
        const int r = w / W, q = w - r * W;
        const int gj = j0 - c + r, gi = i0 - c + q;
        in[r][q] = (gj >= 0 && gj < n && gi >= 0 && gi < n) ? res[gj * n + gi] : T(0);
    }
    __syncthreads();
    const int tx0 = 4 * (threadIdx.x % (PSF_T / 4)), ty = threadIdx.x / (PSF_T / 4);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int b = 0; b < K; ++b) {
        const T* row = in[ty + b] + tx0;                    // row[u + a] for output u, tap a
        T v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3];
        const T* kr = kp + b * K;
        for (int a = 0; a < K; ++a) {
            const T w = kr[a];
            acc[0] += w * v0; acc[1] += w * v1; acc[2] += w * v2; acc[3] += w * v3;
            v0 = v1; v1 = v2; v2 = v3;
            v3 = a + 1 < K ? row[a + 4] : T(0);
        }
    }
    const T sc = E.dlogL ? (T)(*E.dlogL) : T(1);
    const int j = j0 + ty;
    T gm = T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + tx0 + u;
        if (i < n && j < n) {
            const T g = acc[u] * sc;
            reinterpret_cast<T*>(E.gimg)[j * n + i] = g;
            gm = fmax(gm, r_abs(g));
        }
    }
    note_gmax(E, gm);
}

}  // namespace rtu
