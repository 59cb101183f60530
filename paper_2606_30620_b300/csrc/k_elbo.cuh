// k_elbo.cuh -- S10: one stochastic-variational step (Sec. 4) for a batch of
// systems: reparametrised samples of the mean-field Normal guide drawn on the
// device with Philox4x32-10 (Salmon et al. 2011) and Box-Muller, then (after the
// batched forward + adjoint of every sample) the Monte-Carlo ELBO, its gradient
// w.r.t. the guide's location and softplus-scale, and an Adam ascent step.
#pragma once
#include "rtu_internal.cuh"

namespace rtu {

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// standard normal of element e of one guide sample (same definition as the oracle)
__device__ __forceinline__ double guide_normal(uint64_t seed, uint32_t tag, uint32_t step, uint32_t sample, int e) {
    uint32_t c[4] = {(uint32_t)(e >> 1), sample, step, tag};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const uint32_t a = (e & 1) ? c[2] : c[0], b = (e & 1) ? c[3] : c[1];
    const double u1 = ((double)a + 0.5) / 4294967296.0;
    const double u2 = ((double)b + 0.5) / 4294967296.0;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

struct PriorD { int kind, space; double a, b, c, d; };

__device__ __forceinline__ double sigm(double u) { return 1.0 / (1.0 + exp(-u)); }
__device__ __forceinline__ double log_sigm(double u) {       // -softplus(-u), overflow free
    return -(fmax(-u, 0.0) + log1p(exp(-fabs(u))));
}
__device__ __forceinline__ double softplus_d(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

// site value v(u), dv/du, log p(v) + log|dv/du| and its u-derivative
__device__ __forceinline__ void site_eval(const PriorD& p, double u, double& v, double& dv, double& lp, double& dlp) {
    const double L2PI = 1.8378770664093453;   // ln(2 pi)
    if (p.kind == 0) {            // normal(mu = a, sd = b)
        v = u; dv = 1.0;
        const double z = (v - p.a) / p.b;
        lp = -0.5 * z * z - log(p.b) - 0.5 * L2PI;
        dlp = -z / p.b;
        return;
    }
    const double lo = p.kind == 1 ? p.a : p.c, hi = p.kind == 1 ? p.b : p.d;
    const double sg = sigm(u);
    v = lo + (hi - lo) * sg;
    dv = (hi - lo) * sg * (1.0 - sg);
    lp = log_sigm(u) + log_sigm(-u);
    dlp = 1.0 - 2.0 * sg;
    if (p.kind == 2) {            // truncated normal(mu = a, sd = b) on [c, d]
        const double z = (v - p.a) / p.b;
        const double Z = 0.5 * (erf((p.d - p.a) / (p.b * 1.4142135623730951)) -
                                erf((p.c - p.a) / (p.b * 1.4142135623730951)));
        lp += -0.5 * z * z - log(p.b) - 0.5 * L2PI - log(Z) + log(hi - lo);
        dlp += -z / p.b * dv;
    } else if (p.kind == 3) {     // linear: density 1 + a (v - lo)/(hi - lo) on [c, d]
        lp += log(1.0 + p.a * sg) - log((hi - lo) * (1.0 + 0.5 * p.a)) + log(hi - lo);
        dlp += p.a * sg * (1.0 - sg) / (1.0 + p.a * sg);
    }
    // uniform: log p = -log(hi - lo) cancels log(hi - lo) of the Jacobian
}

// physical index of non-latent site i (gamma of an SIE and tau of each subhalo are fixed)
__device__ __forceinline__ int site_target(int i, int profile, int nsub, int nl) {
    const int nlens = profile == 1 ? 8 : 7;
    if (i < nlens) return (profile == 1 || i == 0) ? i : i + 1;
    i -= nlens;
    if (i < 4 * nsub) {
        const int h = i / 4, k = i - 4 * h;
        return 8 + 5 * h + (k < 2 ? k : k + 1);
    }
    i -= 4 * nsub;
    return nl + i;
}

struct ElboState {
    double* loc;      // [n_state]
    double* rho;      // [n_state]
    double* m;        // [2 n_state] Adam first moments (loc then rho)
    double* v;        // [2 n_state]
    PriorD* prior;    // [n_sites]
    double* fixed;    // [n_phys] physical values of the non-site entries
    long long* t;     // step counter (device)
    double* part;     // per-CTA partial ELBO terms
    double* grad;     // [2 n_state] the last step's ELBO gradient w.r.t. loc, then rho (before Adam)
    uint32_t tag;
    int n_sites, n_state, n_phys;
};

constexpr int MAXS = 8;           // guide samples per step
constexpr int ELBO_MAXB = 24;     // systems per ELBO launch

struct ElboArgs {
    ElboState st;
    int profile, nsub, nl, n_src, f64, n_samples;
    uint64_t seed;
    double lr;
    // per sample s (< MAXS): the sample's parameter and gradient buffers
    double* lens[MAXS];
    double* ps[MAXS];
    void* lat[MAXS];
    double* stats[MAXS];
    double* glens[MAXS];
    double* gps[MAXS];
    void* glat[MAXS];
    double* elbo_out;
    int n_cta_upd;
};

struct ElboBatch {
    int n;
    int tile0[ELBO_MAXB + 1];
    ElboArgs e[ELBO_MAXB];
};

constexpr int ELBO_NT = 256;

// draw sample s of every site and write the sample's physical parameters
__global__ void __launch_bounds__(ELBO_NT) k_elbo_sample(const __grid_constant__ ElboBatch B) {
    const int ev = find_eval(B, blockIdx.x);
    const ElboArgs& A = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int per = (A.st.n_state + ELBO_NT - 1) / ELBO_NT;
    const int s = tile / per, e = (tile - s * per) * ELBO_NT + threadIdx.x;
    const uint32_t step = (uint32_t)(*A.st.t);
    if (tile - s * per == 0 && threadIdx.x < A.st.n_phys) {
        // non-site entries (overwritten below for the site entries by other threads
        // of this CTA only after the barrier)
        const int i = threadIdx.x;
        if (i < A.nl) A.lens[s][i] = A.st.fixed[i]; else A.ps[s][i - A.nl] = A.st.fixed[i];
    }
    __syncthreads();
    if (e >= A.st.n_state) return;
    const double eps = guide_normal(A.seed, A.st.tag, step, (uint32_t)s, e);
    const double u = A.st.loc[e] + softplus_d(A.st.rho[e]) * eps;
    if (e < A.st.n_sites) {
        const PriorD p = A.st.prior[e];
        double v, dv, lp, dlp;
        site_eval(p, u, v, dv, lp, dlp);
        const double th = p.space == 1 ? pow(10.0, v) : v;
        const int ti = site_target(e, A.profile, A.nsub, A.nl);
        if (ti < A.nl) A.lens[s][ti] = th; else A.ps[s][ti - A.nl] = th;
    } else {
        const int k = e - A.st.n_sites;
        if (A.f64) reinterpret_cast<double*>(A.lat[s])[k] = u;
        else reinterpret_cast<float*>(A.lat[s])[k] = (float)u;
    }
}

// gradient of the Monte-Carlo ELBO per element, Adam ascent, partial ELBO sums
__global__ void __launch_bounds__(ELBO_NT) k_elbo_update(const __grid_constant__ ElboBatch B) {
    const int ev = find_eval(B, blockIdx.x);
    const ElboArgs& A = B.e[ev];
    const int tile = blockIdx.x - B.tile0[ev];
    const int e = tile * ELBO_NT + threadIdx.x;
    __shared__ double red[ELBO_NT / 32];
    const uint32_t step = (uint32_t)(*A.st.t);
    const int S = A.n_samples;
    double term = 0.0;
    if (e < A.st.n_state) {
        const double rho = A.st.rho[e], loc = A.st.loc[e];
        const double sc = softplus_d(rho), sgr = sigm(rho);
        double gl = 0.0, gr = 0.0;
        PriorD p;
        int ti = -1;
        if (e < A.st.n_sites) { p = A.st.prior[e]; ti = site_target(e, A.profile, A.nsub, A.nl); }
        for (int s = 0; s < S; ++s) {
            const double eps = guide_normal(A.seed, A.st.tag, step, (uint32_t)s, e);
            const double u = loc + sc * eps;
            double gu, lp;
            if (e < A.st.n_sites) {
                double v, dv, dlp;
                site_eval(p, u, v, dv, lp, dlp);
                const double gth = ti < A.nl ? A.glens[s][ti] : A.gps[s][ti - A.nl];
                const double dth = p.space == 1 ? pow(10.0, v) * 2.302585092994046 : 1.0;
                gu = gth * dth * dv + dlp;
            } else {
                const int k = e - A.st.n_sites;
                const double g = A.f64 ? reinterpret_cast<const double*>(A.glat[s])[k]
                                       : (double)reinterpret_cast<const float*>(A.glat[s])[k];
                gu = g - u;                                  // d/dw [log L + log N(w; 0, 1)]
                lp = -0.5 * u * u - 0.9189385332046727;
            }
            gl += gu;
            gr += gu * eps * sgr;
            term += lp + 0.5 * eps * eps + log(sc) + 0.9189385332046727;   // log p + log|J| - log q
        }
        gl /= S;
        gr = gr / S + sgr / sc;                              // + d/drho of the guide entropy
        A.st.grad[e] = gl;
        A.st.grad[A.st.n_state + e] = gr;
        // Adam (ascent), t = step + 1
        const double b1 = 0.9, b2 = 0.999, ea = 1e-8;
        const double t1 = (double)step + 1.0;
        const double c1 = 1.0 - pow(b1, t1), c2 = 1.0 - pow(b2, t1);
        const int n = A.st.n_state;
        double m0 = b1 * A.st.m[e] + (1.0 - b1) * gl, v0 = b2 * A.st.v[e] + (1.0 - b2) * gl * gl;
        double m1 = b1 * A.st.m[n + e] + (1.0 - b1) * gr, v1 = b2 * A.st.v[n + e] + (1.0 - b2) * gr * gr;
        A.st.m[e] = m0; A.st.v[e] = v0; A.st.m[n + e] = m1; A.st.v[n + e] = v1;
        A.st.loc[e] = loc + A.lr * (m0 / c1) / (sqrt(v0 / c2) + ea);
        A.st.rho[e] = rho + A.lr * (m1 / c1) / (sqrt(v1 / c2) + ea);
    }
    term = block_sum<ELBO_NT>(term, red);
    if (threadIdx.x == 0) A.st.part[tile] = term;
}

// ELBO = (1/S) sum_s [log L_s + sum_elements (log p + log|J| - log q)]; step += 1
__global__ void __launch_bounds__(32) k_elbo_final(const __grid_constant__ ElboBatch B) {
    const ElboArgs& A = B.e[blockIdx.x];
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int t = 0; t < A.n_cta_upd; ++t) s += A.st.part[t];
    double ll = 0.0;
    for (int k = 0; k < A.n_samples; ++k) ll += A.stats[k][0];
    if (A.elbo_out) *A.elbo_out = (ll + s) / A.n_samples;
    *A.st.t += 1;
}

}  // namespace rtu
