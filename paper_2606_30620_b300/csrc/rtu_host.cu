// rtu_host.cu -- the C ABI (include/rtu.h): workspace layout, system creation
// and the per-step batched launches.  Host code allocates nothing on the
// device; every buffer is carved out of the caller's workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "rtu.h"
#include "rtu_internal.cuh"
#include "k_grid.cuh"
#include "k_gp.cuh"
#include "k_render.cuh"
#include "k_psf.cuh"
#include "k_adj.cuh"
#include "k_elbo.cuh"
#include "k_light.cuh"

using namespace rtu;

static_assert(sizeof(Batch) <= 32000, "batch descriptor must fit the kernel-parameter limit");
static_assert(sizeof(ElboBatch) <= 32000, "ELBO batch descriptor must fit the kernel-parameter limit");
static_assert(sizeof(rtu_prior) == sizeof(PriorD), "prior layout");

namespace {

thread_local std::string g_err;

rtu_status fail(rtu_status code, const std::string& msg) {
    g_err = msg;
    return code;
}

}  // namespace

__attribute__((visibility("hidden"))) rtu_status rtu_fail_internal(rtu_status code, const char* msg) {
    return fail(code, msg);
}

namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

bool factor_radices(int n, std::vector<int>& rad) {
    rad.clear();
    while (n % 4 == 0) { rad.push_back(4); n /= 4; }
    while (n % 2 == 0) { rad.push_back(2); n /= 2; }
    while (n % 3 == 0) { rad.push_back(3); n /= 3; }
    return n == 1 && (int)rad.size() <= MAX_RADIX;
}

// position p holds input element rev(p) for the in-place DIT order used by
// fft_seq_smem: p = sum_s j_s L_{s-1} -> rev = j_S + r_S j_{S-1} + r_S r_{S-1} j_{S-2} + ...
std::vector<int> digit_reversal(int n, const std::vector<int>& rad) {
    std::vector<int> rev(n);
    const int S = (int)rad.size();
    for (int p = 0; p < n; ++p) {
        std::vector<int> js(S);
        int q = p;
        for (int s = 0; s < S; ++s) { js[s] = q % rad[s]; q /= rad[s]; }
        int v = 0, w = 1;
        for (int s = S - 1; s >= 0; --s) { v += js[s] * w; w *= rad[s]; }
        rev[p] = v;
    }
    return rev;
}

struct Sizes {
    int nm_max, n_cta_c_max, n_cta_r, n_cta_p, K, ncell, n_rays, nacc, nl, tb, n_cta_adj;
    int nps, n_sites, n_state, n_phys, n_fixed, n_cta_upd;
};

Sizes sizes_of(const rtu_system_desc& d) {
    Sizes z;
    z.nm_max = d.n_img * d.n_img;
    z.n_cta_c_max = (z.nm_max + CTA_C - 1) / CTA_C;
    z.n_cta_r = render_tiles(d.n_img);
    const int tiles = (d.n_img + PSF_T - 1) / PSF_T;
    z.n_cta_p = tiles * tiles;
    z.K = d.n_nodes + 2;
    z.ncell = (d.n_src - 1) * (d.n_src - 1);
    z.n_rays = d.n_img * d.n_img * d.s_super * d.s_super;
    // the adjoint's grid-stride CTAs: one chunk each when a quarter of the rays is in the
    // grid (c2: 79 CTAs per system; measured against an eighth, 0.289 vs 0.300 ms, and a
    // sixteenth or a half, both slower)
    z.n_cta_adj = std::max(1, (z.n_rays + ADJ_DIV * CTA_R * ADJ_RPT - 1) / (ADJ_DIV * CTA_R * ADJ_RPT));
    const int nsub = d.sub_kind ? d.n_sub : 0;
    z.nacc = NACC_FIX + 4 * z.K + 5 * nsub;
    z.nl = 8 + 5 * nsub;
    z.tb = d.precision == RTU_F64 ? 8 : 4;
    z.nps = (d.ps_family == RTU_PS_MATERN ? 3 : 2) + 1;
    z.n_sites = (d.profile == RTU_EPL ? 8 : 7) + 4 * nsub + z.nps;
    z.n_state = z.n_sites + d.n_src * d.n_src;
    z.n_phys = z.nl + z.nps;
    z.n_fixed = z.n_phys + 6 * d.n_light;
    z.n_cta_upd = (z.n_state + ELBO_NT - 1) / ELBO_NT;
    return z;
}

// per-slot layout; returns bytes.  If base != nullptr fills the slot pointers.
size_t slot_layout(const rtu_system_desc& d, char* base, EvalArgs* e) {
    const Sizes z = sizes_of(d);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return base ? base + at : nullptr; };
    char* p;
    p = take((size_t)2 * z.nm_max * 8);               if (e) e->beta = (double*)p;
    p = take((size_t)z.n_cta_c_max * 8 * 8);          if (e) e->cpart = (double*)p;
    p = take((size_t)z.n_cta_c_max * 2 * 8);          if (e) e->cpart2 = (double*)p;
    p = take(8 * 8);                                  if (e) e->mom = (double*)p;
    p = take(16);                                     if (e) e->ccnt = (int*)p;
    p = take((size_t)2 * z.nm_max * 4);               if (e) e->cbin = (int*)p;
    p = take((size_t)(z.n_cta_c_max + 2) * z.nl * 8); if (e) e->cadj = (double*)p;
    p = take((size_t)4 * MAXM * z.nl * 8);           if (e) e->jsel = (double*)p;

    p = take((size_t)2 * (HB + HROWS) * 4);           if (e) e->hist = (int*)p;
    p = take((size_t)tr_size(z.K) * 8);               if (e) e->trd = (double*)p;
    p = take((size_t)tr_size(z.K) * 4);               if (e) e->trf = (float*)p;
    p = take((size_t)4 * MAXM * 4);                   if (e) e->sel_idx = (int*)p;
    p = take((size_t)(TADJ_SEL + 4 * MAXM) * 8);      if (e) e->tadj = (double*)p;
    const size_t n2 = (size_t)d.n_src * d.n_src;
    p = take(n2 * 2 * 8);                             if (e) e->cbufA = p;     // complex double (the GP source)
    p = take(n2 * 2 * z.tb);                          if (e) e->cbufB = p;
    p = take((size_t)gp_part_rows(d.n_src) * 4 * 8); if (e) e->gpart = (double*)p;
    p = take(n2 * z.tb);                              if (e) e->fld = p;
    p = take(n2 * z.tb);                              if (e) e->src = p;
    const size_t ni = (size_t)d.n_img * d.n_img;
    p = take(ni * z.tb);                              if (e) e->img = p;
    p = take(ni * z.tb);                              if (e) e->resid = p;
    p = take(ni * z.tb);                              if (e) e->gimg = p;
    p = take((size_t)z.n_cta_p * 2 * 8);              if (e) e->lpart = (double*)p;
    p = take((size_t)z.n_cta_r * CTA_R * d.s_super * d.s_super * 4); if (e) e->cell = (int*)p;
    p = take((size_t)(2 * z.ncell + 1) * 4);          if (e) e->ccount = (int*)p;
    p = take((size_t)z.ncell * 4);                    if (e) e->cursor = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->elist = (int*)p;
    p = take((size_t)z.n_rays * 4 * z.tb);            if (e) e->rec = p;
    p = take((size_t)z.ncell * 4 * 2 * z.tb);         if (e) e->corner = p;
    // partial rows for the largest tunable adjoint split (one CTA per CTA_R ADJ_RPT rays)
    // and near-core pass
    const int adj_max = std::max(1, (z.n_rays + CTA_R * ADJ_RPT - 1) / (CTA_R * ADJ_RPT));
    p = take((size_t)std::max(z.n_cta_r, adj_max + NEAR_CTAS_MAX) * z.nacc * 8); if (e) e->apart = (double*)p;
    p = take(16);                                     if (e) e->flags = (int*)p;
    p = take(8);                                      if (e) e->gmax = (unsigned long long*)p;
    p = take(LENSK_BYTES);                            if (e) e->lensk = p;
    p = take(16);                                     if (e) e->ecount = (int*)p;
    p = take(ni * 8);                                 if (e) e->pdef = (unsigned long long*)p;
    p = take(ni * 4);                                 if (e) e->pcnt = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->rval = (float*)p;
    p = take((size_t)(z.n_cta_r + 1) * 4);            if (e) e->cta_cnt = (int*)p;
    p = take((size_t)z.n_cta_r);                      if (e) e->tcull = (unsigned char*)p;
    p = take((size_t)(z.n_cta_r * (CTA_R / 32) + 1) * 4); if (e) e->useg = (int*)p;
    p = take((size_t)(z.n_cta_r * (CTA_R / 32) + 1) * 4); if (e) e->nseg = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->nlist = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->kray = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->kcell = (int*)p;
    p = take((size_t)z.n_rays * 4);                   if (e) e->krank = (int*)p;
    p = take((size_t)z.n_rays * 2 * z.tb);            if (e) e->gbuf = p;
    p = take((size_t)light_ctas(d.n_img) * 6 * std::max(1, d.n_light) * 8); if (e) e->lpartl = (double*)p;
    if (d.transform == RTU_TRANSFORM_LINEAR) {
        // the unsmoothed eCDF: every order statistic and its gradient
        p = take((size_t)2 * z.nm_max * 8);           if (e) e->lkey = (double*)p;
        p = take((size_t)2 * z.nm_max * 4);           if (e) e->lidx = (int*)p;
        p = take((size_t)2 * z.nm_max * 4);           if (e) e->lrank = (int*)p;
        p = take((size_t)2 * z.nm_max * 8);           if (e) e->lkf = (float*)p;
        p = take((size_t)2 * z.nm_max * 16);          if (e) e->gk = (unsigned long long*)p;
    }
    return o;
}

// per-slot buffers of one guide sample: parameters in, statistics and gradients out
struct SampleBufs { double *lens, *ps, *stats, *glens, *gps, *glight; void *lat, *glat; };

size_t sample_layout(const rtu_system_desc& d, char* base, SampleBufs* b) {
    const Sizes z = sizes_of(d);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return base ? base + at : nullptr; };
    const size_t n2 = (size_t)d.n_src * d.n_src;
    char* p;
    p = take((size_t)z.nl * 8);   if (b) b->lens = (double*)p;
    p = take((size_t)z.nps * 8);  if (b) b->ps = (double*)p;
    p = take(n2 * z.tb);          if (b) b->lat = p;
    p = take(8 * 8);              if (b) b->stats = (double*)p;
    p = take((size_t)z.nl * 8);   if (b) b->glens = (double*)p;
    p = take((size_t)z.nps * 8);  if (b) b->gps = (double*)p;
    p = take(n2 * z.tb);          if (b) b->glat = p;
    p = take((size_t)6 * std::max(1, d.n_light) * 8); if (b) b->glight = (double*)p;
    return o;
}

size_t state_layout(const rtu_system_desc& d, char* base, ElboState* st) {
    const Sizes z = sizes_of(d);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return base ? base + at : nullptr; };
    char* p;
    p = take((size_t)z.n_state * 8);      if (st) st->loc = (double*)p;
    p = take((size_t)z.n_state * 8);      if (st) st->rho = (double*)p;
    p = take((size_t)2 * z.n_state * 8);  if (st) st->m = (double*)p;
    p = take((size_t)2 * z.n_state * 8);  if (st) st->v = (double*)p;
    p = take((size_t)z.n_sites * sizeof(PriorD)); if (st) st->prior = (PriorD*)p;
    p = take((size_t)z.n_fixed * 8);      if (st) st->fixed = (double*)p;
    p = take(8);                          if (st) st->t = (long long*)p;
    p = take((size_t)z.n_cta_upd * 8);    if (st) st->part = (double*)p;
    p = take((size_t)2 * z.n_state * 8);  if (st) st->grad = (double*)p;
    if (st) { st->n_sites = z.n_sites; st->n_state = z.n_state; st->n_phys = z.n_phys; st->tag = 0; }
    return o;
}

size_t static_layout(const rtu_system_desc& d, char* base, int** cidx, double** tw, int** rev, double** cheb,
                     uint32_t** cwt = nullptr, double** psf_uv = nullptr) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return base ? base + at : nullptr; };
    char* p = take((size_t)d.n_img * d.n_img * 4); if (cidx) *cidx = (int*)p;
    p = take((size_t)d.n_img * d.n_img * 4);       if (cwt) *cwt = (uint32_t*)p;
    p = take((size_t)2 * d.n_src * 8);             if (tw) *tw = (double*)p;
    p = take((size_t)d.n_src * 4);                 if (rev) *rev = (int*)p;
    p = take((size_t)cheb_size(d.n_nodes, d.degree) * 8); if (cheb) *cheb = (double*)p;
    p = take((size_t)2 * d.psf_k * 8);             if (psf_uv) *psf_uv = (double*)p;
    return o;
}

// A rank-1 PSF psf[b][a] = u[b] v[a] (a sampled circular or axis-aligned Gaussian, for
// one) is convolved in two one-dimensional passes.  The factors are a column and a row
// through the largest tap; the PSF counts as rank 1 when no tap differs from u[b] v[a]
// by more than 8 rounding units of its precision times the largest tap.
bool psf_rank1(const std::vector<double>& P, int K, bool f64, double* uv) {
    int b0 = 0, a0 = 0;
    for (int i = 0; i < K * K; ++i)
        if (std::fabs(P[i]) > std::fabs(P[b0 * K + a0])) { b0 = i / K; a0 = i % K; }
    const double p0 = P[b0 * K + a0];
    if (!(std::fabs(p0) > 0.0)) return false;
    for (int b = 0; b < K; ++b) uv[b] = P[b * K + a0];
    for (int a = 0; a < K; ++a) uv[K + a] = P[b0 * K + a] / p0;
    const double tol = 8.0 * (f64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24)) * std::fabs(p0);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a)
            if (!(std::fabs(P[b * K + a] - uv[b] * uv[K + a]) <= tol)) return false;
    return true;
}

// Chebyshev nodes and the matrices of the interpolating fit (App. C iii-iv), by
// the three-term recurrences in double
std::vector<double> chebyshev_tables(int M, int D) {
    const int K = M + 2;
    std::vector<double> t(cheb_size(M, D), 0.0);
    std::vector<double> u(M), tk(K);
    for (int j = 1; j <= M; ++j) u[j - 1] = (1.0 - std::cos((2.0 * j - 1.0) * M_PI / (2.0 * M))) / 2.0;
    for (int j = 0; j < M; ++j) t[cheb_u(M, D) + j] = u[j];
    for (int j = 0; j < K; ++j) tk[j] = j == 0 ? -1.0 : (j == K - 1 ? 1.0 : 2.0 * u[j - 1] - 1.0);
    for (int j = 0; j < K; ++j) {
        double T0 = 1.0, T1 = tk[j], U0 = 1.0, U1 = 2.0 * tk[j];
        for (int k = 0; k <= D; ++k) {
            double Tk, dTk;
            if (k == 0) { Tk = 1.0; dTk = 0.0; }
            else if (k == 1) { Tk = T1; dTk = U0; }
            else {
                Tk = 2.0 * tk[j] * T1 - T0; dTk = k * U1;
                T0 = T1; T1 = Tk;
                const double U2 = 2.0 * tk[j] * U1 - U0;
                U0 = U1; U1 = U2;
            }
            t[cheb_V(M, D) + j * (D + 1) + k] = Tk;
            t[cheb_dV(M, D) + j * (D + 1) + k] = 2.0 * dTk;     // d/du = 2 d/dt
        }
    }
    for (int j = 0; j < M; ++j) {
        const double tj = 2.0 * u[j] - 1.0;
        double T0 = 1.0, T1 = tj;
        for (int k = 0; k <= D; ++k) {
            double Tk = k == 0 ? 1.0 : (k == 1 ? tj : 2.0 * tj * T1 - T0);
            if (k >= 2) { T0 = T1; T1 = Tk; }
            t[cheb_C(M, D) + k * M + j] = (2.0 / M) * Tk * (k == 0 ? 0.5 : 1.0);
        }
    }
    return t;
}

const char* check_desc(const rtu_system_desc* d) {
    if (!d) return "desc is null";
    if (d->n_img < 2 || d->n_img > 4096) return "n_img must be in [2, 4096]";
    if (d->s_super < 1 || d->s_super > 8) return "s_super must be in [1, 8]";
    std::vector<int> rad;
    if (d->n_src < 4 || d->n_src > 256 || !factor_radices(d->n_src, rad)) return "n_src must be 2^a 3^b in [4, 256]";
    if (d->psf_k < 1 || d->psf_k > 31 || d->psf_k % 2 == 0) return "psf_k must be odd in [1, 31]";
    if (d->profile != RTU_SIE && d->profile != RTU_EPL) return "profile must be RTU_SIE or RTU_EPL";
    if (d->sub_kind < 0 || d->sub_kind > 2) return "bad sub_kind";
    if (d->n_sub < 0 || d->n_sub > RTU_MAX_SUB) return "n_sub must be in [0, 16]";
    if (d->ps_family < 0 || d->ps_family > 2) return "bad ps_family";
    if (d->precision != RTU_F32 && d->precision != RTU_F64) return "precision must be RTU_F32 or RTU_F64";
    if (d->n_nodes != d->degree + 1) return "this build supports n_nodes == degree + 1 (interpolating fit)";
    if (d->n_nodes < 2 || d->n_nodes > MAXM) return "n_nodes must be in [2, 64]";
    if (d->n_slots < 1) return "n_slots must be >= 1";
    if (d->transform != RTU_TRANSFORM_RTU && d->transform != RTU_TRANSFORM_UNIFORM &&
        d->transform != RTU_TRANSFORM_LINEAR)
        return "bad transform";
    if (d->transform == RTU_TRANSFORM_LINEAR && d->weights)
        return "the unsmoothed eCDF transform takes no ray weights";
    if (d->n_light < 0 || d->n_light > RTU_MAX_LIGHT) return "n_light must be in [0, 8]";
    if (!(d->pix > 0) || !(d->src_pitch > 0) || !(d->sigma > 0)) return "pix, src_pitch, sigma must be > 0";
    if (!d->data || !d->mask || !d->psf) return "data, mask and psf must be device pointers";
    return nullptr;
}

std::once_flag g_attr_once;
constexpr int MAX_DYN = 200 * 1024;

void set_attributes() {
    cudaFuncSetAttribute(k_select_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_SMEM);
    cudaFuncSetAttribute(k_render<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_gp_adj_cluster<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GP_CL_SMEM_MAX);
    cudaFuncSetAttribute(k_gp_adj_cluster<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GP_CL_SMEM_MAX);
    // 8 CTAs per SM at the c2 shape (24 KB each): the largest shared-memory carveout
    cudaFuncSetAttribute(k_render<float, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_render<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<float, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<double, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<double, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<float, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
    cudaFuncSetAttribute(k_render_adj<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN);
}

}  // namespace

struct rtu_system {
    rtu_system_desc d;
    Sizes z;
    int n_mask, n_cta_c, nrad;
    int rad[MAX_RADIX];
    int* cidx;
    uint32_t* cwt;                // weights of the centre rays (weighted grid), else null
    int wtot;                     // total weight of the centre rays (n_mask when unweighted)
    double* tw;
    int* rev;
    double* cheb;
    double* psf_uv;               // factors of a rank-1 PSF, or null
    std::vector<EvalArgs> slot;   // workspace pointers of each slot
    int adj_div = ADJ_DIV;        // launch shapes (rtu_system_tune)
    int n_near = NEAR_CTAS;
    int n_edge = EDGE_CTAS;
    std::vector<SampleBufs> sbuf; // guide-sample buffers of each slot
    ElboState st;
    bool elbo_ready = false;
};

// ------------------------------------------------------------ zero kernel
constexpr int ZERO_TILES = 16;
__global__ void __launch_bounds__(256) k_zero(const __grid_constant__ Batch B, int with_cells) {
    const int ev = find_eval(B, blockIdx.x);
    const EvalArgs& E = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int nh = 2 * (HB + HROWS);
    const int ncell = (E.n_src - 1) * (E.n_src - 1);
    const int tot = nh + (with_cells ? 2 * ncell : 0);
    // tiles 1.. zero; tile 0 builds the lens blocks (a chain of FP64 latencies)
    for (int i = (tile - 1) * 256 + threadIdx.x; tile > 0 && i < tot; i += (ZERO_TILES - 1) * 256) {
        if (i < nh) E.hist[i] = 0;
        else if (i < nh + ncell) E.ccount[i - nh] = 0;
        else E.cursor[i - nh - ncell] = 0;          // the compaction's rank cursors
    }
    if (tile == 0) {
        if (threadIdx.x == 0) {
            *E.flags = 0; *E.ecount = 0; E.ccnt[0] = 0; E.ccnt[1] = 0; E.ccnt[2] = 0; E.ccnt[3] = 0;
            *E.gmax = 0ull;
        }
        const int nsub = E.sub_kind ? E.n_sub : 0;
        char* kb = static_cast<char*>(E.lensk);
        lens_setup_par(reinterpret_cast<LensK<double>*>(kb), reinterpret_cast<LensK<float>*>(kb + LENSK_D_BYTES),
                       reinterpret_cast<LensK<DF>*>(kb + LENSK_DF_AT), E.lens, E.profile, E.sub_kind, nsub);
    }
}

extern "C" {

size_t rtu_workspace_size(const rtu_system_desc* d) {
    if (check_desc(d)) return 0;
    return static_layout(*d, nullptr, nullptr, nullptr, nullptr, nullptr) +
           (size_t)d->n_slots * (slot_layout(*d, nullptr, nullptr) + sample_layout(*d, nullptr, nullptr)) +
           state_layout(*d, nullptr, nullptr) + 256;
}

rtu_status rtu_system_create(const rtu_system_desc* d, void* ws, size_t ws_bytes, rtu_system** out) {
    // synchronous: the uploads have landed when the call returns
    const rtu_status r = rtu_system_create_on(d, nullptr, ws, ws_bytes, nullptr, out);
    if (r != RTU_OK) return r;
    const cudaError_t ce = cudaStreamSynchronize(nullptr);
    if (ce != cudaSuccess) {
        rtu_system_destroy(*out);
        *out = nullptr;
        return fail(RTU_E_CUDA, std::string("rtu_system_create: ") + cudaGetErrorString(ce));
    }
    return RTU_OK;
}

rtu_status rtu_system_create_on(const rtu_system_desc* d, const rtu_host_inputs* hin, void* ws, size_t ws_bytes,
                                void* stream, rtu_system** out) {
    if (!out) return fail(RTU_E_ARG, "out is null");
    *out = nullptr;
    if (const char* m = check_desc(d)) return fail(RTU_E_ARG, m);
    if (!ws) return fail(RTU_E_WORKSPACE, "workspace is null");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(RTU_E_WORKSPACE, "workspace must be 256-byte aligned");
    if (ws_bytes < rtu_workspace_size(d)) return fail(RTU_E_WORKSPACE, "workspace smaller than rtu_workspace_size()");
    std::call_once(g_attr_once, set_attributes);
    rtu_system* s = new rtu_system();
    s->d = *d;
    s->z = sizes_of(*d);
    std::vector<int> rad;
    factor_radices(d->n_src, rad);
    s->nrad = (int)rad.size();
    for (int i = 0; i < MAX_RADIX; ++i) s->rad[i] = i < s->nrad ? rad[i] : 1;
    char* base = static_cast<char*>(ws);
    uint32_t* cwt_buf = nullptr;
    double* uv_buf = nullptr;
    const size_t st = static_layout(*d, base, &s->cidx, &s->tw, &s->rev, &s->cheb, &cwt_buf, &uv_buf);
    // arc-mask pixel list (the CDF uses observed-pixel centres inside the mask)
    const size_t npx = (size_t)d->n_img * d->n_img;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaSuccess;
    // the caller's observation block first, so that the desc's buffers are filled in
    // stream order before any kernel that reads them
    if (hin && hin->upload_bytes) {
        if (!hin->upload_src || !hin->upload_dst) { delete s; return fail(RTU_E_ARG, "upload block without its pointers"); }
        if ((ce = cudaMemcpyAsync(hin->upload_dst, hin->upload_src, hin->upload_bytes, cudaMemcpyHostToDevice, cs)) !=
            cudaSuccess) {
            delete s;
            return fail(RTU_E_CUDA, std::string("observation upload: ") + cudaGetErrorString(ce));
        }
    }
    // host copies of the mask, the PSF and the weights when the caller has them (no
    // device-to-host copy, which would wait for the device), else read back from the device
    std::vector<uint8_t> mask_copy;
    const uint8_t* mask = hin ? hin->mask : nullptr;
    if (!mask) {
        mask_copy.resize(npx);
        ce = cudaMemcpy(mask_copy.data(), d->mask, npx, cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) { delete s; return fail(RTU_E_CUDA, std::string("mask copy: ") + cudaGetErrorString(ce)); }
        mask = mask_copy.data();
    }
    // the static tables are assembled on the host with the device layout and go up in
    // two copies; the pixel list is written straight into that image
    std::unique_ptr<char[]> img(new char[st]);
    int* hcidx;
    double *htw, *hcheb;
    int* hrev;
    uint32_t* hcwt;
    double* huv;
    static_layout(*d, img.get(), &hcidx, &htw, &hrev, &hcheb, &hcwt, &huv);
    const size_t tw_off = (size_t)(reinterpret_cast<char*>(htw) - img.get());
    memset(img.get() + tw_off, 0, st - tw_off);        // alignment gaps of the small tables
    size_t nm = 0;
    for (size_t i = 0; i < npx; ++i) {                 // branch-free compaction, pixel order
        hcidx[nm] = (int)i;
        nm += mask[i] != 0;
    }
    if (nm < 2) { delete s; return fail(RTU_E_ARG, "the arc mask must hold at least 2 pixels"); }
    s->n_mask = (int)nm;
    s->n_cta_c = (s->n_mask + CTA_C - 1) / CTA_C;
    // weighted grid: the centre rays' weights, checked, in arc-mask order
    s->cwt = nullptr;
    s->wtot = s->n_mask;
    if (d->weights) {
        std::vector<uint32_t> w_copy;
        const uint32_t* w = hin ? hin->weights : nullptr;
        if (!w) {
            w_copy.resize(npx);
            if ((ce = cudaMemcpy(w_copy.data(), d->weights, npx * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
                delete s;
                return fail(RTU_E_CUDA, std::string("weights copy: ") + cudaGetErrorString(ce));
            }
            w = w_copy.data();
        }
        unsigned long long tot = 0;
        for (size_t k = 0; k < nm; ++k) {
            hcwt[k] = w[hcidx[k]];
            tot += hcwt[k];
            if (hcwt[k] == 0) { delete s; return fail(RTU_E_ARG, "weights must be >= 1 on the arc mask"); }
        }
        if (tot >= (1ull << 31)) { delete s; return fail(RTU_E_ARG, "the mask's total weight must be < 2^31"); }
        s->cwt = cwt_buf;
        s->wtot = (int)tot;
    }
    for (int m = 0; m < d->n_src; ++m) {
        const double ang = -2.0 * M_PI * m / d->n_src;
        htw[2 * m] = std::cos(ang);
        htw[2 * m + 1] = std::sin(ang);
    }
    const std::vector<int> rev = digit_reversal(d->n_src, rad);
    memcpy(hrev, rev.data(), rev.size() * 4);
    const std::vector<double> cheb = chebyshev_tables(d->n_nodes, d->degree);
    memcpy(hcheb, cheb.data(), cheb.size() * 8);
    // the PSF: rank 1 or not
    const int K = d->psf_k;
    const bool f64 = d->precision == RTU_F64;
    std::vector<double> P(K * K);
    {
        std::vector<float> pf(f64 ? 0 : K * K);
        const void* hp = hin ? hin->psf : nullptr;
        if (hp) {
            if (f64) memcpy(P.data(), hp, K * K * 8);
            else memcpy(pf.data(), hp, K * K * 4);
        } else {
            ce = f64 ? cudaMemcpy(P.data(), d->psf, K * K * 8, cudaMemcpyDeviceToHost)
                     : cudaMemcpy(pf.data(), d->psf, K * K * 4, cudaMemcpyDeviceToHost);
        }
        if (ce != cudaSuccess) { delete s; return fail(RTU_E_CUDA, std::string("psf copy: ") + cudaGetErrorString(ce)); }
        if (!f64) for (int i = 0; i < K * K; ++i) P[i] = pf[i];
    }
    const bool sep = psf_rank1(P, K, f64, huv);
    s->psf_uv = sep ? uv_buf : nullptr;
    // the arc-mask pixel list with, on a weighted grid, the centre weights behind it
    // (their region starts one table further on), then the FFT / Chebyshev / PSF tables:
    // stream-ordered copies from pageable memory, staged by the driver before the call
    // returns, so `img` may go out of scope; legacy stream when none is given
    const size_t cwt_off = (size_t)(reinterpret_cast<char*>(hcwt) - img.get());
    if ((ce = cudaMemcpyAsync(base, img.get(), nm * 4, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
        (d->weights &&
         (ce = cudaMemcpyAsync(base + cwt_off, img.get() + cwt_off, nm * 4, cudaMemcpyHostToDevice, cs)) != cudaSuccess) ||
        (ce = cudaMemcpyAsync(base + tw_off, img.get() + tw_off, st - tw_off, cudaMemcpyHostToDevice, cs)) !=
            cudaSuccess) {
        delete s;
        return fail(RTU_E_CUDA, std::string("table upload: ") + cudaGetErrorString(ce));
    }
    const size_t per = slot_layout(*d, nullptr, nullptr);
    const size_t sper = sample_layout(*d, nullptr, nullptr);
    s->slot.resize(d->n_slots);
    s->sbuf.resize(d->n_slots);
    for (int k = 0; k < d->n_slots; ++k) {
        EvalArgs e;
        memset(&e, 0, sizeof(e));
        slot_layout(*d, base + st + (size_t)k * (per + sper), &e);
        s->slot[k] = e;
        sample_layout(*d, base + st + (size_t)k * (per + sper) + per, &s->sbuf[k]);
    }
    memset(&s->st, 0, sizeof(s->st));
    state_layout(*d, base + st + (size_t)d->n_slots * (per + sper), &s->st);
    *out = s;
    return RTU_OK;
}

rtu_status rtu_system_tune(rtu_system* s, const rtu_tuning* t) {
    if (!s || !t) return fail(RTU_E_ARG, "rtu_system_tune: null argument");
    if (t->adj_div < 1 || t->adj_div > 64) return fail(RTU_E_ARG, "rtu_system_tune: adj_div must be in [1, 64]");
    if (t->near_ctas < 1 || t->near_ctas > NEAR_CTAS_MAX)
        return fail(RTU_E_ARG, "rtu_system_tune: near_ctas must be in [1, 16]");
    if (t->edge_ctas < 1 || t->edge_ctas > 256) return fail(RTU_E_ARG, "rtu_system_tune: edge_ctas must be in [1, 256]");
    s->adj_div = t->adj_div;
    s->n_near = t->near_ctas;
    s->n_edge = t->edge_ctas;
    return RTU_OK;
}

rtu_status rtu_system_destroy(rtu_system* s) {
    delete s;
    return RTU_OK;
}

const char* rtu_last_error(void) { return g_err.c_str(); }
const char* rtu_version(void) { return "rtu-b300 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

rtu_status fill_args(rtu_system* s, const rtu_eval& v, EvalArgs& e) {
    if (v.slot < 0 || v.slot >= s->d.n_slots) return fail(RTU_E_ARG, "eval slot out of range");
    if (!v.lens || !v.latents || !v.ps) return fail(RTU_E_ARG, "lens, latents and ps must be set");
    e = s->slot[v.slot];
    const rtu_system_desc& d = s->d;
    e.n_img = d.n_img; e.s = d.s_super; e.n_src = d.n_src; e.psf_k = d.psf_k;
    e.profile = d.profile; e.sub_kind = d.sub_kind; e.n_sub = d.n_sub; e.family = d.ps_family;
    e.n_nodes = d.n_nodes; e.degree = d.degree; e.n_mask = s->n_mask; e.f64 = d.precision == RTU_F64;
    e.transform = d.transform;
    e.nrad = s->nrad; e.n_cta_c = s->n_cta_c; e.n_cta_r = s->z.n_cta_r; e.n_cta_p = s->z.n_cta_p;
    e.n_cta_adj = std::max(1, (s->z.n_rays + s->adj_div * CTA_R * ADJ_RPT - 1) / (s->adj_div * CTA_R * ADJ_RPT));
    e.n_near = s->n_near;
    e.n_edge = s->n_edge;
    e.n_row_adj = e.n_cta_adj + (d.precision == RTU_F64 ? 0 : s->n_near);
    for (int i = 0; i < MAX_RADIX; ++i) e.rad[i] = s->rad[i];
    e.pix = d.pix; e.pitch = d.src_pitch; e.sigma = d.sigma;
    e.data = d.data; e.mask = d.mask; e.psf = d.psf;
    e.centre_idx = s->cidx; e.tw = s->tw; e.digrev = s->rev; e.cheb = s->cheb;
    e.cwt = s->cwt; e.wtot = s->wtot;
    e.psf_uv = s->psf_uv;
    e.lens = v.lens; e.latents = v.latents; e.ps = v.ps; e.dlogL = v.dlogL;
    e.stats = v.stats; e.model_out = v.model; e.image_out = v.image; e.source_out = v.source;
    e.cdf_out = v.cdf; e.hist_out = v.ray_hist;
    e.sel_hist_out = v.sel_hist; e.centres_out = v.centres;
    e.g_lat = v.g_latents; e.g_lens = v.g_lens; e.g_ps = v.g_ps;
    e.n_light = d.n_light;
    e.light = d.n_light > 0 ? v.light : nullptr;
    e.g_light = d.n_light > 0 ? v.g_light : nullptr;
    if (d.n_light > 0 && !v.light) return fail(RTU_E_ARG, "light must be set when n_light > 0");
    return RTU_OK;
}

typedef int (*TileFn)(const EvalArgs&);

// ---- optional per-kernel event timing
struct ProfRec { const char* name; cudaEvent_t a, b; int side; };
cudaStream_t g_side_hint = nullptr;   // the side stream of the launching thread (timeline)
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<std::pair<std::string, std::pair<long, double>>> g_prof_acc;

template <typename Kern, typename... Extra>
rtu_status launch(const char* name, Kern kern, Batch& B, TileFn tiles, int threads, size_t smem,
                  cudaStream_t st, Extra... extra) {
    int tot = 0;
    for (int i = 0; i < B.n; ++i) { B.tile0[i] = tot; tot += tiles(B.e[i]); }
    B.tile0[B.n] = tot;
    if (tot == 0) return RTU_OK;
    ProfRec pr{name, nullptr, nullptr, st == nullptr ? 0 : (st == g_side_hint ? 1 : 0)};
    const bool prof = g_prof_on;
    if (prof) {
        cudaEventCreate(&pr.a);
        cudaEventCreate(&pr.b);
        cudaEventRecord(pr.a, st);
    }
    kern<<<tot, threads, smem, st>>>(B, extra...);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(RTU_E_CUDA, std::string("launch ") + name + ": " + cudaGetErrorString(ce));
    if (prof) {
        cudaEventRecord(pr.b, st);
        std::lock_guard<std::mutex> g(g_prof_mu);
        g_prof_pending.push_back(pr);
    }
    return RTU_OK;
}

int t_one(const EvalArgs&) { return 1; }
// smoothed (RTU, uniform box) or unsmoothed-eCDF systems only, in a mixed batch
bool is_lin(const EvalArgs& e) { return e.transform == RTU_TRANSFORM_LINEAR; }
int t_two_fit(const EvalArgs& e) { return is_lin(e) ? 0 : 2; }
int t_two_lin(const EvalArgs& e) { return is_lin(e) ? 2 : 0; }
int t_one_fit(const EvalArgs& e) { return is_lin(e) ? 0 : 1; }
int t_centre_fit(const EvalArgs& e) { return is_lin(e) ? 0 : e.n_cta_c; }
int t_centre_lin(const EvalArgs& e) { return is_lin(e) ? e.n_cta_c : 0; }
int t_light(const EvalArgs& e) { return e.light && e.n_light > 0 ? light_ctas(e.n_img) : 0; }
int t_light_fwd(const EvalArgs& e) {
    return e.light && e.n_light > 0 ? (e.n_img * e.n_img + LIGHT_FWD_NT - 1) / LIGHT_FWD_NT : 0;
}
int t_render_fit(const EvalArgs& e) { return is_lin(e) ? 0 : e.n_cta_r; }
int t_render_lin(const EvalArgs& e) { return is_lin(e) ? e.n_cta_r : 0; }
int t_adj_fit(const EvalArgs& e) { return is_lin(e) ? 0 : e.n_cta_adj; }
int t_adj_lin(const EvalArgs& e) { return is_lin(e) ? e.n_cta_adj : 0; }
int t_near_fit(const EvalArgs& e) { return is_lin(e) ? 0 : e.n_near; }
int t_near_lin(const EvalArgs& e) { return is_lin(e) ? e.n_near : 0; }
int t_gp_lines(const EvalArgs& e) { return (e.n_src + GP_LINES - 1) / GP_LINES; }
// the GP adjoint's cluster kernel where it fits (per storage type), else the line passes
int t_gp_cl_f(const EvalArgs& e) { return gp_cluster_ok(e.n_src, 4) ? GP_CL : 0; }
int t_gp_cl_d(const EvalArgs& e) { return gp_cluster_ok(e.n_src, 8) ? GP_CL : 0; }
int t_gp_lines_f(const EvalArgs& e) { return gp_cluster_ok(e.n_src, 4) ? 0 : t_gp_lines(e); }
int t_gp_lines_d(const EvalArgs& e) { return gp_cluster_ok(e.n_src, 8) ? 0 : t_gp_lines(e); }
int t_zero(const EvalArgs&) { return ZERO_TILES; }
int t_centre(const EvalArgs& e) { return e.n_cta_c; }
int t_adj(const EvalArgs& e) { return e.n_cta_adj; }
int t_psf_gen(const EvalArgs& e) { return e.psf_uv ? 0 : e.n_cta_p; }
// rank-1 PSFs by tap count: 21 and 9 have compiled tap loops, others a runtime one
int t_psf_sep21(const EvalArgs& e) { return e.psf_uv && e.psf_k == 21 ? e.n_cta_p : 0; }
int t_psf_sep9(const EvalArgs& e) { return e.psf_uv && e.psf_k == 9 ? e.n_cta_p : 0; }
int t_psf_sep_k(const EvalArgs& e) { return e.psf_uv && e.psf_k != 21 && e.psf_k != 9 ? e.n_cta_p : 0; }
int t_edge(const EvalArgs& e) { return e.n_edge; }
int t_cull_lin(const EvalArgs& e) { return is_lin(e) ? (e.n_cta_r + CULL_NT - 1) / CULL_NT : 0; }
int t_units(const EvalArgs& e) { return std::min(CMP_CTAS, std::max(1, (e.n_cta_r * (CTA_R / 32) + 63) / 64)); }
int t_defer(const EvalArgs& e) { return e.n_edge + 1; }
int t_cells(const EvalArgs& e) {
    const int nc = (e.n_src - 1) * (e.n_src - 1);
    return (nc + GATHER_NT / 16 - 1) / (GATHER_NT / 16);
}

enum Phase { PH_GRID = 1, PH_FORWARD = 2, PH_ADJOINT = 4 };

// A side stream per (host thread, device), created at the highest stream priority,
// carries the step's critical branch where the step forks: the grid build (S1-S5)
// beside the GP source of the forward (then the selected-rank lens Jacobians beside
// the render), the adjoint's ray list beside the forward's PSF and likelihood, and the
// transform / centre-ray adjoint beside the cell gather and GP adjoint of the adjoint.  Fork and join are event waits, so a call still orders everything
// after the work already on the caller's stream and leaves nothing pending on the side
// streams when it returns (and the pattern is legal inside CUDA graph capture).
// Created at the first call on a device and kept for the life of the thread.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int MAX_DEV = 64;

rtu_status side_stream(SideStream*& out) {
    static thread_local SideStream tab[MAX_DEV];
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return fail(RTU_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= MAX_DEV) return fail(RTU_E_ARG, "device index too large");
    SideStream& ss = tab[dev];
    if (!ss.s) {
        int least = 0, greatest = 0;
        if ((ce = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess ||
            (ce = cudaStreamCreateWithPriority(&ss.s, cudaStreamNonBlocking, greatest)) != cudaSuccess ||
            (ce = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)) != cudaSuccess ||
            (ce = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)) != cudaSuccess)
            return fail(RTU_E_CUDA, std::string("side stream: ") + cudaGetErrorString(ce));
    }
    out = &ss;
    return RTU_OK;
}

// after: `to` runs behind everything enqueued so far on `from`
rtu_status stream_after(cudaStream_t to, cudaStream_t from, cudaEvent_t ev) {
    cudaError_t ce = cudaEventRecord(ev, from);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(to, ev, 0);
    return ce == cudaSuccess ? RTU_OK : fail(RTU_E_CUDA, std::string("stream order: ") + cudaGetErrorString(ce));
}

template <typename T>
rtu_status run_chunk(Batch& B, int phase, cudaStream_t st, const SideStream& ss) {
    rtu_status r;
    int max_s2 = 0, any_sub = 0, maxK = 0, maxPsf = 0, any_light = 0;
    size_t grid_bytes = 0;     // the largest source grid the render kernels stage in shared memory
    for (int i = 0; i < B.n; ++i) {
        grid_bytes = std::max(grid_bytes, grid_smem_bytes(B.e[i].n_src, (int)sizeof(T)));
        maxPsf = std::max(maxPsf, B.e[i].psf_k);
        any_light |= B.e[i].n_light > 0;
        max_s2 = std::max(max_s2, B.e[i].s * B.e[i].s);
        any_sub |= (B.e[i].sub_kind && B.e[i].n_sub > 0);
        maxK = std::max(maxK, B.e[i].n_nodes + 2);
    }
    if (phase & (PH_GRID | PH_FORWARD)) {
        // S1-S5 (the forward's critical branch: on the high-priority side stream, issued
        // first, when the GP source, which only needs the latents and spectrum
        // parameters, runs beside it on the caller's stream)
        const bool fork = (phase & PH_FORWARD) != 0;
        const cudaStream_t sg = fork ? ss.s : st;
        if (fork && (r = stream_after(ss.s, st, ss.fork))) return r;
        if ((r = launch("k_zero", k_zero, B, t_zero, 256, 0, sg, fork ? 1 : 0))) return r;
        if ((r = launch("k_trace_centres", k_trace_centres, B, t_centre, CTA_C, 0, sg))) return r;
        if ((r = launch("k_centre_hist", k_centre_hist, B, t_centre, CTA_C, 0, sg))) return r;
        if ((r = launch("k_select_fit", k_select_fit, B, t_two_fit, SEL_NT, SEL_SMEM, sg))) return r;
        if ((r = launch("k_lin_sort", k_lin_sort, B, t_two_lin, LIN_NT, 0, sg))) return r;
        if ((phase & PH_FORWARD) && (r = launch("k_cull_tiles", k_cull_tiles, B, t_cull_lin, CULL_NT, 0, sg)))
            return r;
        if (fork)
            for (int pass = 0; pass < GP_PASSES; ++pass)
                if ((r = launch("k_gp_source", k_gp_lines<T>, B, t_gp_lines, GP_LINE_NT, 0, st, pass))) return r;
    }
    if (phase & PH_FORWARD) {
        if ((r = stream_after(st, ss.s, ss.join))) return r;
        // the selected-rank lens Jacobians (for the adjoint) beside the render
        if ((r = launch("k_sel_jac", k_sel_jac, B, t_one_fit, SEL_ADJ_NT, 0, ss.s))) return r;

        const size_t render_smem = grid_bytes + (size_t)CTA_R * max_s2 * 2;
        if (render_smem > MAX_DYN) return fail(RTU_E_ARG, "render shared memory exceeds the limit");
        if ((r = launch("k_render", k_render<T, false>, B, t_render_fit, CTA_R, render_smem, st))) return r;
        if ((r = launch("k_render", k_render<T, true>, B, t_render_lin, CTA_R, render_smem, st))) return r;
        // the adjoint's ray list (the adjoint follows the forward on the same slots) on
        // the side stream: the render warps' offsets and the compaction of the rays the
        // render decided beside the near-edge pass, then the rays that pass decides and
        // S11's cell offsets beside the lens light, the PSF and the likelihood
        if ((r = stream_after(ss.s, st, ss.fork))) return r;
        if ((r = launch("k_scan_warps", k_scan_warps, B, t_one, SCAN_NT, 0, ss.s))) return r;
        if ((r = launch("k_compact", k_compact, B, t_units, CMP_NT, 0, ss.s))) return r;
        if (sizeof(T) == 4 && (r = launch("k_render_edge", k_render_edge, B, t_edge, EDGE_NT, 0, st))) return r;
        if ((r = stream_after(ss.s, st, ss.fork))) return r;
        if ((r = launch("k_compact_deferred", k_compact_deferred, B, t_defer, CMPD_NT, 0, ss.s))) return r;
        if (any_light && (r = launch("k_light_fwd", k_light_fwd<T>, B, t_light_fwd, LIGHT_FWD_NT, 0, st))) return r;
        if ((r = launch("k_psf_like", k_psf_like_sep<T, 21>, B, t_psf_sep21, PSFS_NT, 0, st))) return r;
        if ((r = launch("k_psf_like", k_psf_like_sep<T, 9>, B, t_psf_sep9, PSFS_NT, 0, st))) return r;
        if ((r = launch("k_psf_like", k_psf_like_sep<T, 0>, B, t_psf_sep_k, PSFS_NT, 0, st))) return r;
        if (sizeof(T) == 4 && maxPsf <= 9) r = launch("k_psf_like", k_psf_like_t<9>, B, t_psf_gen, PSFT_NT, 0, st);
        else if (sizeof(T) == 4 && maxPsf <= 21) r = launch("k_psf_like", k_psf_like_t<21>, B, t_psf_gen, PSFT_NT, 0, st);
        else r = launch("k_psf_like", k_psf_like<T>, B, t_psf_gen, PSF_NT, 0, st);
        if (r) return r;
        if ((r = stream_after(st, ss.s, ss.join))) return r;
    }
    if (phase & PH_ADJOINT) {
        const size_t adj = grid_bytes + (size_t)(CTA_R / 32) * 4 * maxK * 2 * sizeof(T);
        if (adj > MAX_DYN) return fail(RTU_E_ARG, "adjoint shared memory exceeds the limit");
        if ((r = launch("k_psf_adj", k_psf_adj_sep<T, 21>, B, t_psf_sep21, PSFS_NT, 0, st))) return r;
        if ((r = launch("k_psf_adj", k_psf_adj_sep<T, 9>, B, t_psf_sep9, PSFS_NT, 0, st))) return r;
        if ((r = launch("k_psf_adj", k_psf_adj_sep<T, 0>, B, t_psf_sep_k, PSFS_NT, 0, st))) return r;
        if (sizeof(T) == 4 && maxPsf <= 9) r = launch("k_psf_adj", k_psf_adj_t<9>, B, t_psf_gen, PSFT_NT, 0, st);
        else if (sizeof(T) == 4 && maxPsf <= 21) r = launch("k_psf_adj", k_psf_adj_t<21>, B, t_psf_gen, PSFT_NT, 0, st);
        else r = launch("k_psf_adj", k_psf_adj<T>, B, t_psf_gen, PSF_NT, 0, st);
        if (r) return r;
        if (any_light && (r = launch("k_light_adj", k_light_adj<T>, B, t_light, CTA_R, 0, st))) return r;
        if (sizeof(T) == 4) {
            // the near-core rays' double-precision pass on the side stream, beside the
            // float pass (disjoint partial rows, records and subhalo entries)
            if ((r = stream_after(ss.s, st, ss.fork))) return r;
            if ((r = launch("k_render_adj_near", k_render_adj<float, false, true>, B, t_near_fit, CTA_R, adj, ss.s)))
                return r;
            if ((r = launch("k_render_adj_near", k_render_adj<float, true, true>, B, t_near_lin, CTA_R, adj, ss.s)))
                return r;
        }
        if ((r = launch("k_render_adj", k_render_adj<T, false, false>, B, t_adj_fit, CTA_R, adj, st))) return r;
        if ((r = launch("k_render_adj", k_render_adj<T, true, false>, B, t_adj_lin, CTA_R, adj, st))) return r;
        if (sizeof(T) == 4 && (r = stream_after(st, ss.s, ss.join))) return r;
        if (any_sub && (r = launch("k_sub_adj", k_sub_adj<T>, B, t_adj, CTA_R, 0, st))) return r;
        // transform and centre-ray adjoint (the critical branch, side stream) beside
        // the cell gather and GP adjoint (main)
        if ((r = stream_after(ss.s, st, ss.fork))) return r;
        if ((r = launch("k_cdf_adj", k_cdf_adj, B, t_two_fit, CDF_NT, 0, ss.s))) return r;
        if ((r = launch("k_centre_adj", k_centre_adj<T>, B, t_centre_fit, CTA_C, 0, ss.s))) return r;
        if ((r = launch("k_lin_centre_adj", k_lin_centre_adj, B, t_centre_lin, CTA_C, 0, ss.s))) return r;
        if ((r = launch("k_cell_gather", k_cell_gather<T>, B, t_cells, GATHER_NT, 0, st))) return r;
        // the GP adjoint: one cluster per evaluation where its lines fit, else line passes
        size_t gp_cl = 0;
        for (int i = 0; i < B.n; ++i)
            if (gp_cluster_ok(B.e[i].n_src, (int)sizeof(T))) gp_cl = std::max(gp_cl, gp_cluster_bytes(B.e[i].n_src, (int)sizeof(T)));
        if ((r = launch("k_gp_adjoint", k_gp_adj_cluster<T>, B, sizeof(T) == 4 ? t_gp_cl_f : t_gp_cl_d, GP_CL_NT, gp_cl, st)))
            return r;
        for (int pass = 0; pass < GP_PASSES; ++pass)
            if ((r = launch("k_gp_adjoint", k_gp_adj_lines<T>, B, sizeof(T) == 4 ? t_gp_lines_f : t_gp_lines_d, GP_LINE_NT,
                            0, st, pass)))
                return r;
        if ((r = stream_after(st, ss.s, ss.join))) return r;
        if ((r = launch("k_grad_final", k_grad_final, B, t_one, GRAD_NT, 0, st))) return r;
    }
    return RTU_OK;
}

// ---- replay of recorded launch sequences
// Every kernel of a chunk takes the Batch by value (plus a pass index) and its grid
// and shared-memory sizes follow from the Batch, so a chunk's launches are a pure
// function of (phase, precision, the Batch's systems).  The second time a call
// repeats those bytes, its launches are recorded into a CUDA graph (captured on a
// stream of the library's) and replayed on the caller's stream from then on while
// the bytes repeat; a batch seen once (serving's changing batches) launches plainly.
// Device data is read when the graph runs: new contents behind the same pointers
// are seen.  Per host thread and device, the GRAPH_CACHE most recently used graphs
// and the GRAPH_SEEN most recent batches' hashes are kept.
std::atomic<bool> g_graphs_on{true};
constexpr int GRAPH_CACHE = 8;
constexpr int GRAPH_SEEN = 32;
struct GraphEntry {
    int phase = 0, prec = 0;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long used = 0;
};
struct GraphCache {
    cudaStream_t cs = nullptr;
    std::vector<GraphEntry> ent;
    unsigned long long tick = 0;
    unsigned long long seen[GRAPH_SEEN] = {};
    int seen_at = 0;
};
// 64-bit multiplicative hash of the key bytes (it only decides when to record; a
// replay needs the bytes equal)
unsigned long long key_hash(int phase, int prec, const void* p, size_t bytes) {
    unsigned long long h = 0x9e3779b97f4a7c15ull ^ (unsigned long long)(phase * 31 + prec);
    const unsigned char* c = static_cast<const unsigned char*>(p);
    size_t i = 0;
    for (; i + 8 <= bytes; i += 8) {
        unsigned long long w;
        std::memcpy(&w, c + i, 8);
        h = (h ^ w) * 0x100000001b3ull;
        h ^= h >> 29;
    }
    for (; i < bytes; ++i) h = (h ^ c[i]) * 0x100000001b3ull;
    return h ? h : 1ull;
}
GraphCache* graph_cache() {
    static thread_local GraphCache tab[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return nullptr;
    GraphCache& gc = tab[dev];
    if (!gc.cs && cudaStreamCreateWithFlags(&gc.cs, cudaStreamNonBlocking) != cudaSuccess) {
        gc.cs = nullptr;
        return nullptr;
    }
    return &gc;
}
void graph_cache_clear() {
    GraphCache* gc = graph_cache();
    if (!gc) return;
    for (GraphEntry& e : gc->ent) cudaGraphExecDestroy(e.exec);
    gc->ent.clear();
}

// the caller's stream is being captured (by the caller): launch plainly into it
bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

rtu_status run_chunk_any(Batch& B, int phase, int prec, cudaStream_t st, const SideStream& ss) {
    return prec == RTU_F64 ? run_chunk<double>(B, phase, st, ss) : run_chunk<float>(B, phase, st, ss);
}

rtu_status run_chunk_graph(Batch& B, int phase, int prec, cudaStream_t st, const SideStream& ss) {
    GraphCache* gc = graph_cache();
    if (!gc) return run_chunk_any(B, phase, prec, st, ss);
    const size_t kb = sizeof(int) + (size_t)B.n * sizeof(EvalArgs);
    const unsigned char* kp = reinterpret_cast<const unsigned char*>(B.e);
    GraphEntry* hit = nullptr;
    for (GraphEntry& e : gc->ent)
        if (e.phase == phase && e.prec == prec && e.key.size() == kb &&
            std::memcmp(e.key.data(), &B.n, sizeof(int)) == 0 &&
            std::memcmp(e.key.data() + sizeof(int), kp, kb - sizeof(int)) == 0) {
            hit = &e;
            break;
        }
    if (!hit) {
        // record only a batch seen before
        const unsigned long long h = key_hash(phase, prec, kp, kb - sizeof(int)) ^ (unsigned long long)B.n;
        bool seen = false;
        for (int i = 0; i < GRAPH_SEEN; ++i) seen |= gc->seen[i] == h;
        if (!seen) {
            gc->seen[gc->seen_at] = h;
            gc->seen_at = (gc->seen_at + 1) % GRAPH_SEEN;
            return run_chunk_any(B, phase, prec, st, ss);
        }
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(gc->cs, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return run_chunk_any(B, phase, prec, st, ss);
        }
        const rtu_status r = run_chunk_any(B, phase, prec, gc->cs, ss);
        ce = cudaStreamEndCapture(gc->cs, &g);
        cudaGraphExec_t exec = nullptr;
        if (r == RTU_OK && ce == cudaSuccess && g) ce = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (r != RTU_OK) return r;
        if (ce != cudaSuccess || !exec) {
            // not recordable here: run the chunk plainly
            cudaGetLastError();
            return run_chunk_any(B, phase, prec, st, ss);
        }
        if ((int)gc->ent.size() >= GRAPH_CACHE) {
            auto lru = std::min_element(gc->ent.begin(), gc->ent.end(),
                                        [](const GraphEntry& x, const GraphEntry& y) { return x.used < y.used; });
            cudaGraphExecDestroy(lru->exec);
            gc->ent.erase(lru);
        }
        GraphEntry e;
        e.phase = phase;
        e.prec = prec;
        e.key.resize(kb);
        std::memcpy(e.key.data(), &B.n, sizeof(int));
        std::memcpy(e.key.data() + sizeof(int), kp, kb - sizeof(int));
        e.exec = exec;
        gc->ent.push_back(std::move(e));
        hit = &gc->ent.back();
    }
    hit->used = ++gc->tick;
    const cudaError_t ce = cudaGraphLaunch(hit->exec, st);
    if (ce != cudaSuccess) return fail(RTU_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

rtu_status run(rtu_system* const* sys, const rtu_eval* ev, int n, int phase, void* stream) {
    if (n < 0 || (n > 0 && (!sys || !ev))) return fail(RTU_E_ARG, "bad system/eval arrays");
    if (n == 0) return RTU_OK;
    const int prec = sys[0] ? sys[0]->d.precision : 0;
    for (int i = 0; i < n; ++i) {
        if (!sys[i]) return fail(RTU_E_ARG, "null system in batch");
        if (sys[i]->d.precision != prec) return fail(RTU_E_ARG, "all systems of one call must share the precision");
        if ((phase & PH_ADJOINT) && (!ev[i].g_latents || !ev[i].g_lens || !ev[i].g_ps))
            return fail(RTU_E_ARG, "adjoint outputs g_latents, g_lens, g_ps must be set");
        if ((phase & PH_ADJOINT) && sys[i]->d.n_light > 0 && !ev[i].g_light)
            return fail(RTU_E_ARG, "adjoint output g_light must be set when n_light > 0");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SideStream* ss = nullptr;
    if (rtu_status r = side_stream(ss)) return r;
    if (g_prof_on) g_side_hint = ss->s;
    static thread_local Batch B;
    const bool replay = g_graphs_on.load(std::memory_order_relaxed) && !g_prof_on && !stream_capturing(st);
    for (int c0 = 0; c0 < n; c0 += MAXB) {
        B.n = std::min(MAXB, n - c0);
        for (int i = 0; i < B.n; ++i) {
            rtu_status r = fill_args(sys[c0 + i], ev[c0 + i], B.e[i]);
            if (r) return r;
        }
        rtu_status r = replay ? run_chunk_graph(B, phase, prec, st, *ss) : run_chunk_any(B, phase, prec, st, *ss);
        if (r) return r;
    }
    return RTU_OK;
}

}  // namespace

extern "C" {

rtu_status rtu_build_grid(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream) {
    return run(sys, ev, n, PH_GRID, stream);
}

rtu_status rtu_forward(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream) {
    return run(sys, ev, n, PH_FORWARD, stream);
}

rtu_status rtu_adjoint(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream) {
    return run(sys, ev, n, PH_ADJOINT, stream);
}

rtu_status rtu_graph_replay(int32_t on) {
    g_graphs_on.store(on != 0, std::memory_order_relaxed);
    if (!on) graph_cache_clear();
    return RTU_OK;
}

rtu_status rtu_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = on != 0;
    return RTU_OK;
}

rtu_status rtu_profile_timeline(char* buf, size_t bytes) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    rtu_status rc = RTU_OK;
    std::string out;
    cudaEvent_t t0 = g_prof_pending.empty() ? nullptr : g_prof_pending.front().a;
    for (ProfRec& p : g_prof_pending) {
        float a = 0.f, b = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&a, t0, p.a) != cudaSuccess ||
            cudaEventElapsedTime(&b, t0, p.b) != cudaSuccess)
            rc = fail(RTU_E_CUDA, "profile event failed");
        char line[160];
        snprintf(line, sizeof(line), "%s %d %.6f %.6f\n", p.name, p.side, a, b);
        out += line;
    }
    for (ProfRec& p : g_prof_pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_prof_pending.clear();
    g_prof_acc.clear();
    if (buf && bytes) {
        size_t n = std::min(bytes - 1, out.size());
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return rc;
}

rtu_status rtu_profile_report(char* buf, size_t bytes) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    rtu_status rc = RTU_OK;
    for (ProfRec& p : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess)
            rc = fail(RTU_E_CUDA, "profile event failed");
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        bool found = false;
        for (auto& e : g_prof_acc)
            if (e.first == p.name) { e.second.first += 1; e.second.second += ms; found = true; break; }
        if (!found) g_prof_acc.push_back({p.name, {1L, (double)ms}});
    }
    g_prof_pending.clear();
    std::string out;
    for (auto& e : g_prof_acc) {
        char line[160];
        snprintf(line, sizeof(line), "%s %ld %.6f\n", e.first.c_str(), e.second.first, e.second.second);
        out += line;
    }
    g_prof_acc.clear();
    if (buf && bytes) {
        size_t n = std::min(bytes - 1, out.size());
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return rc;
}

}  // extern "C"

// ------------------------------------------------- double-float self-test
// y[i] = f(x) of the double-float type that the FP32 path's FP64-class islands use,
// from double inputs converted to double-float (hi = rounded x, lo = rounded rest):
// op 0 exp, 1 log, 2 sqrt (x[i]); 3 quotient, 4 product, 5 sum (x[2i], x[2i+1]);
// the near-edge pass's cell decision helpers: 6 floor, 7 distance to the nearest
// integer (x[i]); the cell gather's integer sums as float pairs: 8 the pair of the
// integer x[2i] (|x| < 2^48) scaled by 2^-x[2i+1], as hi + lo.
__global__ void __launch_bounds__(256) k_selftest_df(int op, const double* x, double* y, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DF r(0.0f, 0.0f);
    if (op == 6 || op == 7) {
        const DF a(x[i]);
        y[i] = op == 6 ? (double)df_floor(a) : (double)df_edge_dist(a);
        return;
    }
    if (op == 8) {
        const float2 p = fix_to_pair((long long)x[2 * i], (int)x[2 * i + 1], 0.0f);
        y[i] = (double)p.x + (double)p.y;
        return;
    }
    if (op <= 2) {
        const DF a(x[i]);
        r = op == 0 ? r_exp(a) : (op == 1 ? r_log(a) : r_sqrt(a));
    } else {
        const DF a(x[2 * i]), b(x[2 * i + 1]);
        r = op == 3 ? a / b : (op == 4 ? a * b : a + b);
    }
    y[i] = r.to_double();
}

extern "C" rtu_status rtu_selftest_df(int32_t op, const double* x, double* y, int32_t n, void* stream) {
    if (op < 0 || op > 8) return fail(RTU_E_ARG, "rtu_selftest_df: op must be in [0, 8]");
    if (n < 0 || (n > 0 && (!x || !y))) return fail(RTU_E_ARG, "rtu_selftest_df: bad buffers");
    if (n == 0) return RTU_OK;
    k_selftest_df<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(op, x, y, n);
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? RTU_OK : fail(RTU_E_CUDA, std::string("launch k_selftest_df: ") + cudaGetErrorString(ce));
}

namespace {

int t_elbo_sample(const ElboArgs& a) { return a.n_samples * ((a.st.n_state + ELBO_NT - 1) / ELBO_NT); }
int t_elbo_update(const ElboArgs& a) { return a.n_cta_upd; }
int t_elbo_one(const ElboArgs&) { return 1; }

template <typename Kern>
rtu_status launch_elbo(const char* name, Kern kern, ElboBatch& B, int (*tiles)(const ElboArgs&), int threads,
                       cudaStream_t st) {
    int tot = 0;
    for (int i = 0; i < B.n; ++i) { B.tile0[i] = tot; tot += tiles(B.e[i]); }
    B.tile0[B.n] = tot;
    if (tot == 0) return RTU_OK;
    kern<<<tot, threads, 0, st>>>(B);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(RTU_E_CUDA, std::string("launch ") + name + ": " + cudaGetErrorString(ce));
    return RTU_OK;
}

}  // namespace

extern "C" {

int32_t rtu_n_sites(const rtu_system_desc* d) {
    if (check_desc(d)) return 0;
    return sizes_of(*d).n_sites;
}

rtu_status rtu_elbo_init(rtu_system* s, const rtu_prior* priors, const double* fixed, const double* loc,
                         const double* rho, uint32_t tag) {
    const rtu_status r = rtu_elbo_init_on(s, priors, fixed, loc, rho, tag, nullptr);
    if (r != RTU_OK) return r;
    const cudaError_t ce = cudaStreamSynchronize(nullptr);     // synchronous, as documented
    return ce == cudaSuccess ? RTU_OK : fail(RTU_E_CUDA, std::string("rtu_elbo_init: ") + cudaGetErrorString(ce));
}

rtu_status rtu_elbo_init_on(rtu_system* s, const rtu_prior* priors, const double* fixed, const double* loc,
                            const double* rho, uint32_t tag, void* stream) {
    if (!s || !priors || !fixed || !loc || !rho) return fail(RTU_E_ARG, "rtu_elbo_init: null argument");
    const Sizes& z = s->z;
    for (int i = 0; i < z.n_sites; ++i) {
        const rtu_prior& p = priors[i];
        if (p.kind < 0 || p.kind > 3 || p.space < 0 || p.space > 1) return fail(RTU_E_ARG, "bad prior kind/space");
        if ((p.kind == RTU_PRIOR_NORMAL || p.kind == RTU_PRIOR_TRUNC_NORMAL) && !(p.b > 0))
            return fail(RTU_E_ARG, "normal prior needs sd > 0");
        if (p.kind == RTU_PRIOR_UNIFORM && !(p.b > p.a)) return fail(RTU_E_ARG, "uniform prior needs b > a");
        if ((p.kind == RTU_PRIOR_TRUNC_NORMAL || p.kind == RTU_PRIOR_LINEAR) && !(p.d > p.c))
            return fail(RTU_E_ARG, "bounded prior needs d > c");
        if (p.kind == RTU_PRIOR_LINEAR && !(p.a >= -1.0)) return fail(RTU_E_ARG, "linear prior needs a >= -1");
    }
    // the state region: loc and rho from the caller's arrays, Adam's m and v zeroed, the
    // priors, fixed values and step from one small host image, the partials and the last
    // gradient zeroed (two copies of the guide, one of the small image, two fills)
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    char* const sp = reinterpret_cast<char*>(s->st.prior);
    char* const send = reinterpret_cast<char*>(s->st.part);
    std::vector<char> img((size_t)(send - sp), 0);
    memcpy(img.data(), priors, (size_t)z.n_sites * sizeof(rtu_prior));
    memcpy(img.data() + (reinterpret_cast<char*>(s->st.fixed) - sp), fixed, (size_t)z.n_fixed * 8);
    const size_t nb = (size_t)z.n_state * 8;
    cudaError_t ce;
    if ((ce = cudaMemcpyAsync(s->st.loc, loc, nb, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(s->st.rho, rho, nb, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
        (ce = cudaMemsetAsync(s->st.m, 0, (size_t)(sp - reinterpret_cast<char*>(s->st.m)), cs)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(sp, img.data(), img.size(), cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
        (ce = cudaMemsetAsync(send, 0, (size_t)(reinterpret_cast<char*>(s->st.grad) + 2 * nb - send), cs)) !=
            cudaSuccess)
        return fail(RTU_E_CUDA, std::string("rtu_elbo_init: ") + cudaGetErrorString(ce));
    s->st.tag = tag;
    s->elbo_ready = true;
    return RTU_OK;
}

rtu_status rtu_elbo_step(rtu_system* const* sys, int32_t n, int32_t n_samples, uint64_t seed, double lr,
                         double* elbo_out, void* stream) {
    if (n < 0 || (n > 0 && !sys)) return fail(RTU_E_ARG, "bad system array");
    if (n_samples < 1 || n_samples > MAXS) return fail(RTU_E_ARG, "n_samples must be in [1, 8]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < n; ++i) {
        if (!sys[i]) return fail(RTU_E_ARG, "null system");
        if (!sys[i]->elbo_ready) return fail(RTU_E_ARG, "rtu_elbo_init was not called for a system");
        if (sys[i]->d.n_slots < n_samples) return fail(RTU_E_ARG, "n_samples exceeds the system's n_slots");
        for (int j = 0; j < i; ++j)
            if (sys[j] == sys[i]) return fail(RTU_E_ARG, "a system appears twice in one ELBO step");
    }
    static thread_local ElboBatch B;
    std::vector<rtu_system*> es;
    std::vector<rtu_eval> ev;
    for (int c0 = 0; c0 < n; c0 += ELBO_MAXB) {
        B.n = std::min(ELBO_MAXB, n - c0);
        es.clear();
        ev.clear();
        for (int i = 0; i < B.n; ++i) {
            rtu_system* s = sys[c0 + i];
            ElboArgs& a = B.e[i];
            memset(&a, 0, sizeof(a));
            a.st = s->st;
            a.profile = s->d.profile;
            a.nsub = s->d.sub_kind ? s->d.n_sub : 0;
            a.nl = s->z.nl;
            a.n_src = s->d.n_src;
            a.f64 = s->d.precision == RTU_F64;
            a.n_samples = n_samples;
            a.seed = seed;
            a.lr = lr;
            a.n_cta_upd = s->z.n_cta_upd;
            a.elbo_out = elbo_out ? elbo_out + c0 + i : nullptr;
            for (int k = 0; k < n_samples; ++k) {
                const SampleBufs& b = s->sbuf[k];
                a.lens[k] = b.lens; a.ps[k] = b.ps; a.lat[k] = b.lat; a.stats[k] = b.stats;
                a.glens[k] = b.glens; a.gps[k] = b.gps; a.glat[k] = b.glat;
                rtu_eval e;
                memset(&e, 0, sizeof(e));
                e.slot = k;
                e.lens = b.lens; e.latents = b.lat; e.ps = b.ps; e.stats = b.stats;
                e.g_latents = b.glat; e.g_lens = b.glens; e.g_ps = b.gps;
                e.light = s->d.n_light > 0 ? s->st.fixed + s->z.n_phys : nullptr;   // held fixed
                e.g_light = s->d.n_light > 0 ? b.glight : nullptr;
                es.push_back(s);
                ev.push_back(e);
            }
        }
        rtu_status r;
        if ((r = launch_elbo("k_elbo_sample", k_elbo_sample, B, t_elbo_sample, ELBO_NT, st))) return r;
        if ((r = run(es.data(), ev.data(), (int)es.size(), PH_FORWARD | PH_ADJOINT, stream))) return r;
        if ((r = launch_elbo("k_elbo_update", k_elbo_update, B, t_elbo_update, ELBO_NT, st))) return r;
        if ((r = launch_elbo("k_elbo_final", k_elbo_final, B, t_elbo_one, 32, st))) return r;
    }
    return RTU_OK;
}

size_t rtu_elbo_state_bytes(const rtu_system* s) {
    if (!s) return 0;
    return (size_t)6 * s->z.n_state * 8 + 8;
}

rtu_status rtu_elbo_export(const rtu_system* s, void* host, size_t bytes) {
    if (!s || !host || bytes < rtu_elbo_state_bytes(s)) return fail(RTU_E_ARG, "rtu_elbo_export: bad buffer");
    const size_t n = (size_t)s->z.n_state * 8;
    char* h = static_cast<char*>(host);
    cudaError_t ce;
    if ((ce = cudaMemcpy(h, s->st.loc, n, cudaMemcpyDeviceToHost)) ||
        (ce = cudaMemcpy(h + n, s->st.rho, n, cudaMemcpyDeviceToHost)) ||
        (ce = cudaMemcpy(h + 2 * n, s->st.m, 2 * n, cudaMemcpyDeviceToHost)) ||
        (ce = cudaMemcpy(h + 4 * n, s->st.v, 2 * n, cudaMemcpyDeviceToHost)) ||
        (ce = cudaMemcpy(h + 6 * n, s->st.t, 8, cudaMemcpyDeviceToHost)))
        return fail(RTU_E_CUDA, std::string("rtu_elbo_export: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

rtu_status rtu_elbo_grad(const rtu_system* s, double* host, size_t bytes) {
    if (!s || !host) return fail(RTU_E_ARG, "rtu_elbo_grad: null argument");
    const size_t n = (size_t)s->z.n_state * 8;
    if (bytes < 2 * n) return fail(RTU_E_ARG, "rtu_elbo_grad: buffer smaller than 2 (n_sites + n_src^2) doubles");
    if (!s->elbo_ready) return fail(RTU_E_ARG, "rtu_elbo_grad: call rtu_elbo_init first");
    const cudaError_t ce = cudaMemcpy(host, s->st.grad, 2 * n, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return fail(RTU_E_CUDA, std::string("rtu_elbo_grad: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

rtu_status rtu_elbo_import(rtu_system* s, const void* host, size_t bytes) {
    if (!s || !host || bytes < rtu_elbo_state_bytes(s)) return fail(RTU_E_ARG, "rtu_elbo_import: bad buffer");
    if (!s->elbo_ready) return fail(RTU_E_ARG, "rtu_elbo_import: call rtu_elbo_init first (priors, fixed values)");
    const size_t n = (size_t)s->z.n_state * 8;
    const char* h = static_cast<const char*>(host);
    cudaError_t ce;
    if ((ce = cudaMemcpy(s->st.loc, h, n, cudaMemcpyHostToDevice)) ||
        (ce = cudaMemcpy(s->st.rho, h + n, n, cudaMemcpyHostToDevice)) ||
        (ce = cudaMemcpy(s->st.m, h + 2 * n, 2 * n, cudaMemcpyHostToDevice)) ||
        (ce = cudaMemcpy(s->st.v, h + 4 * n, 2 * n, cudaMemcpyHostToDevice)) ||
        (ce = cudaMemcpy(s->st.t, h + 6 * n, 8, cudaMemcpyHostToDevice)))
        return fail(RTU_E_CUDA, std::string("rtu_elbo_import: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

}  // extern "C"
