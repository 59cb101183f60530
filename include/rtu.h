/*
 * rtu.h -- C ABI of the B300 (sm_103a) hot path of the RTU-grid lensing method
 * (Enzi, Krawczyk, Li & Collett, "Gaussian processes on ray-guided transformed
 * uniform grids for ... adaptive source reconstruction in lens modelling").
 *
 * One evaluation = one lens system with one parameter set.  A call takes an
 * array of systems and an array of per-evaluation bindings (rtu_eval) and
 * launches each step once for the whole array, so a batch of many systems of
 * uneven sizes fills the GPU; an array of one is the plain per-system path.
 *
 * Conventions common to every entry point
 *  - Ownership: the caller owns every pointer.  Device pointers must stay valid
 *    until the stream reaches the call.  The library allocates no device
 *    memory: all scratch lives in the workspace the caller passes to
 *    rtu_system_create (size from rtu_workspace_size).
 *  - Asynchrony: compute calls are stream-ordered and return before the GPU
 *    finishes; outputs are valid once `stream` has reached the call.
 *  - Precision: desc.precision selects RTU_F64 (every buffer marked "real"
 *    is double) or RTU_F32 (real = float; the centre-ray trace, the CDF
 *    order statistics, the fit, all reductions and near-core deflections stay
 *    in double).  Lens, subhalo and power-spectrum parameters, their
 *    gradients and the scalar statistics are always double.
 *  - Errors: argument, shape and CUDA launch errors are returned
 *    synchronously as a negative rtu_status and described by rtu_last_error().
 *    Conditions found on the device (a repaired non-monotone CDF fit, an
 *    order-statistic selection that ran out of candidate space, a bounded wait
 *    that gave up) are written as bits into stats[RTU_STAT_FLAGS].  Nothing
 *    aborts, traps or exits.
 *  - Thread safety: calls on distinct systems may run from distinct host
 *    threads; a system (its workspace) must not be used by two calls at once.
 *
 * Layouts
 *  - Images are row-major [n_img][n_img]; pixel (i, j), i = column = x, sits at
 *    theta = ((i - (n_img-1)/2) pix, (j - (n_img-1)/2) pix) arcsec; its
 *    s x s sub-rays at offsets ((a + 1/2)/s - 1/2) pix (Sec. 2.3, Sec. 3.1).
 *  - Source grids are row-major [n_src][n_src] on the unit square of RTU
 *    coordinates, node (i, j) at (i/(n_src-1), j/(n_src-1)) (Sec. 2.1-2.2).
 *  - lens[8] = theta_E, gamma, e1, e2, x0, y0, Gamma1, Gamma2 (App. A.1), then
 *    n_sub x {kappa_s, r_s, tau, x_s, y_s} (App. A.2).  (e1, e2) =
 *    (1-q)/(1+q) (cos 2 phi, sin 2 phi).  For RTU_SIE gamma is ignored (= 2) and
 *    its gradient is 0.
 *  - ps = family parameters then alpha_src (Eq. 3-4):
 *      RTU_PS_POWER_LAW   (A, beta):      P = A k^-beta, P(0) = 0
 *      RTU_PS_MATERN_LIKE (A, k0):        P = A / (1 + (k/k0)^2)^2
 *      RTU_PS_MATERN      (sigma, n, zeta): Eq. 4
 *    with k = 2 pi |fftfreq| / src_pitch.
 */
#ifndef RTU_H
#define RTU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rtu_status;

/* return codes (negative = error, returned synchronously) */
#define RTU_OK              0
#define RTU_E_ARG          -1   /* bad argument or unsupported shape */
#define RTU_E_CUDA         -2   /* a CUDA runtime call or launch failed */
#define RTU_E_WORKSPACE    -3   /* workspace too small or misaligned */
#define RTU_E_UNSUPPORTED  -4   /* a mode this build does not implement */

/* device-side flag bits in stats[RTU_STAT_FLAGS] */
#define RTU_W_NONMONOTONE   1   /* the CDF fit needed its monotonicity repair */
#define RTU_W_SELECT        2   /* order-statistic selection unresolved (not raised: the
                                   radix refinement resolves every rank within 8 levels) */
#define RTU_W_TIMEOUT       4   /* a bounded wait on an async copy gave up */
#define RTU_W_RANGE         8   /* the unsmoothed transform's exact position-gradient sums met a
                                   term of magnitude >= 2^40 (left out; the gradient is wrong) */

enum { RTU_F32 = 0, RTU_F64 = 1 };
enum { RTU_SIE = 0, RTU_EPL = 1 };
enum { RTU_SUB_NONE = 0, RTU_SUB_NFW = 1, RTU_SUB_TNFW = 2 };
enum { RTU_PS_POWER_LAW = 0, RTU_PS_MATERN_LIKE = 1, RTU_PS_MATERN = 2 };
/* Source-grid coordinates: the ray-guided transformed uniform grid (smoothed
 * marginal CDFs, Sec. 2.2, App. C), the uniform grid over the smallest square
 * box containing the masked rays (Sec. 2.1), mapped affinely onto [0, 1]^2, or
 * the unsmoothed transform of App. C (first paragraph): per axis the k-th smallest
 * traced arc-mask centre (of n) maps to k/(n-1), linearly in between, and beyond
 * the smallest and largest with the slope of the end segment (a zero-width end
 * segment gives a constant); rays mapped outside [0, 1]^2 see a zero source.  The
 * unsmoothed transform takes no ray weights. */
enum { RTU_TRANSFORM_RTU = 0, RTU_TRANSFORM_UNIFORM = 1, RTU_TRANSFORM_LINEAR = 2 };

/* stats[] written by rtu_forward (double[RTU_N_STATS]); N_IN_GRID = supersampled
 * rays that land inside the RTU grid (the rays the adjoint differentiates) */
enum { RTU_STAT_LOGL = 0, RTU_STAT_CHI2_MASK = 1, RTU_STAT_N_MASK = 2, RTU_STAT_FLAGS = 3,
       RTU_STAT_N_IN_GRID = 4, RTU_N_STATS = 5 };

#define RTU_N_LENS 8
#define RTU_N_SUB_PARAMS 5
#define RTU_MAX_SUB 16
#define RTU_MAX_LIGHT 8     /* MGE lens-light components (App. A.3 uses 5) */
#define RTU_N_LIGHT_PARAMS 6
#define RTU_MAX_NODES 64

/* Static description of one lens system (Sec. 3.1 observation + model choices). */
typedef struct {
    int32_t n_img;       /* image side, pixels (>= 2) */
    int32_t s_super;     /* sub-rays per pixel side (1..8) */
    int32_t n_src;       /* source-grid side; 2^a 3^b, 4 <= n_src <= 256 */
    int32_t psf_k;       /* odd PSF side, 1 <= psf_k <= 31 */
    int32_t profile;     /* RTU_SIE | RTU_EPL */
    int32_t sub_kind;    /* RTU_SUB_* */
    int32_t n_sub;       /* 0..RTU_MAX_SUB subhaloes */
    int32_t ps_family;   /* RTU_PS_* */
    int32_t precision;   /* RTU_F32 | RTU_F64 */
    int32_t n_nodes;     /* Chebyshev nodes M (App. C iii); must equal degree+1 */
    int32_t degree;      /* polynomial degree D of the quantile fit (21 in the paper) */
    int32_t n_slots;     /* concurrent evaluations of this system (e.g. ELBO samples) */
    int32_t transform;   /* RTU_TRANSFORM_RTU (Sec. 2.2) | RTU_TRANSFORM_UNIFORM (Sec. 2.1 box)
                            | RTU_TRANSFORM_LINEAR (App. C, unsmoothed eCDF) */
    int32_t n_light;     /* MGE lens-light components 0..RTU_MAX_LIGHT (App. A.3); 0 = none */
    double pix;          /* arcsec per pixel */
    double src_pitch;    /* source-grid pitch entering k (arcsec) */
    double sigma;        /* Gaussian noise rms (Sec. 3.1) */
    const void* data;    /* device, real [n_img*n_img] observed image */
    const uint8_t* mask; /* device, u8 [n_img*n_img]; nonzero = in the arc mask (Sec. 2.2) */
    const void* psf;     /* device, real [psf_k*psf_k], centre at (psf_k-1)/2 */
    const uint32_t* weights; /* device, u32 [n_img*n_img] or NULL: ray weights of the arc-mask
                                pixels for a weighted RTU grid (Sec. 6.3 extension): each centre
                                ray counts w times in the eCDFs (type-7 quantiles of the
                                weight-expanded sample); w >= 1 on the mask, sum over the mask
                                < 2^31.  NULL = every ray once.  Read once at create. */
} rtu_system_desc;

typedef struct rtu_system rtu_system;

/* Per-evaluation bindings; every pointer is a device pointer. */
typedef struct {
    int32_t slot;              /* workspace slot 0..n_slots-1 */
    int32_t pad_;
    const double* lens;        /* [8 + 5 n_sub] */
    const void* latents;       /* real [n_src*n_src] white-noise latents (Eq. 1) */
    const double* ps;          /* [n_family + 1] power spectrum params, alpha_src last */
    const double* dlogL;       /* adjoint: upstream scale on d log L (nullable => 1) */
    double* stats;             /* forward out: [RTU_N_STATS] (nullable) */
    void* model;               /* forward out: real [n_img^2] PSF-convolved model (nullable) */
    void* image;               /* forward out: real [n_img^2] unconvolved image (nullable) */
    void* source;              /* forward out: real [n_src^2] source brightness s* (nullable) */
    double* cdf;               /* build out: [3 + 4 (M+2)] mu_x, mu_y, sigma_min,
                                  knots_x[M+2], knots_y[M+2], slopes_x[M+2], slopes_y[M+2]
                                  (nullable); RTU_TRANSFORM_LINEAR writes mu_x, mu_y,
                                  sigma_min and zeros */
    int32_t* ray_hist;         /* forward out: [(n_src-1)^2] supersampled rays per RTU cell
                                  (nullable) */
    void* g_latents;           /* adjoint out: real [n_src^2] */
    double* g_lens;            /* adjoint out: [8 + 5 n_sub] */
    double* g_ps;              /* adjoint out: [n_family + 1] */
    const double* light;       /* [6 n_light] lens light (App. A.3), per component A, sigma
                                  (arcsec), q, phi (rad, from +x counter-clockwise), x_n, y_n;
                                  the image adds sum_n A/(2 pi) exp(-rho^2/(2 sigma^2)),
                                  rho^2 = q x'^2 + y'^2/q about (x_n, y_n) rotated by phi, at
                                  every sub-ray before the PSF.  Required when n_light > 0. */
    double* g_light;           /* adjoint out: [6 n_light]; required when n_light > 0 */
    int32_t* sel_hist;         /* build out (nullable): [2][65536] the integer histograms behind
                                  the order statistics (App. C ii), per axis the count (or, for a
                                  weighted grid, the weight) of arc-mask centre rays in each of
                                  65536 bins over [min, max] of that axis's traced positions:
                                  bin = floor((beta - min) * (65536 / (max - min))), clamped to
                                  [0, 65535] (all in bin 0 when max = min) */
    double* centres;           /* build out (nullable): [2][n_mask] the traced arc-mask centre
                                  positions beta_x then beta_y (App. C i), in row-major pixel order
                                  of the mask */
} rtu_eval;

/* Bytes of device workspace one system needs (256-byte aligned base). 0 on bad desc. */
size_t rtu_workspace_size(const rtu_system_desc* desc);

/* Create a system over caller-owned workspace.  Synchronous: copies the mask to
 * the host once to list the arc-mask pixels (Sec. 2.2 footnote: the CDF uses
 * only observed-pixel centres inside the mask) and uploads small tables
 * (FFT twiddles, digit reversal, Chebyshev nodes) into the workspace. */
rtu_status rtu_system_create(const rtu_system_desc* desc, void* workspace, size_t ws_bytes,
                             rtu_system** out);
/* Host copies of a system's observation inputs (each nullable): the arc mask
 * [n_img*n_img] u8, the PSF [psf_k*psf_k] real, the ray weights [n_img*n_img] u32 --
 * the same contents as the desc's device buffers.  upload_bytes > 0: the library first
 * copies upload_bytes from upload_src (host, pinned for an asynchronous copy) to
 * upload_dst (device) on the creation stream -- one block holding the desc's device
 * buffers, so that a caller need not order that copy itself; both pointers must then be
 * non-null (RTU_E_ARG otherwise), and upload_src must stay unchanged until the stream
 * has passed the copy. */
typedef struct {
    const uint8_t* mask;
    const void* psf;
    const uint32_t* weights;
    const void* upload_src;
    void* upload_dst;
    uint64_t upload_bytes;
} rtu_host_inputs;

/* rtu_system_create for a caller that holds the inputs on the host as well (e.g. a
 * server admitting systems while others run): the mask, PSF and weights are read from
 * `host` where given instead of being copied back from the device (a device-to-host
 * copy waits for the device), and the system's tables are uploaded with copies ordered
 * on `stream` (nullable = the legacy stream), which return once the driver has staged
 * the bytes.  The system may be used by calls ordered after `stream`'s copies; the
 * desc's device buffers must hold their contents by the time those calls run. */
rtu_status rtu_system_create_on(const rtu_system_desc* desc, const rtu_host_inputs* host, void* workspace,
                                size_t ws_bytes, void* stream, rtu_system** out);
/* Launch shapes of a system's kernels that may be tuned per problem size (they
 * change the work split only: results agree to the rounding of the partial sums, and
 * a given tuning gives the same bits from run to run):
 *   adj_div    render adjoint CTAs per evaluation = ceil(rays / (adj_div x 2048))
 *              (default 4: one chunk per CTA when a quarter of the rays are in the grid)
 *   near_ctas  CTAs per evaluation of the FP32 path's near-core adjoint pass (default 4)
 *   edge_ctas  CTAs per evaluation of the FP32 path's near-edge double pass (default 16)
 * rtu_system_tune sets them for later calls (ranges [1, 64], [1, 16], [1, 256];
 * RTU_E_ARG otherwise); the workspace holds any value in range. */
typedef struct {
    int32_t adj_div;
    int32_t near_ctas;
    int32_t edge_ctas;
} rtu_tuning;
rtu_status rtu_system_tune(rtu_system* sys, const rtu_tuning* tuning);
rtu_status rtu_system_destroy(rtu_system* sys);

/* S1-S5 (App. C steps i-iv, Sec. 2.2): trace the arc-mask pixel centres through
 * the lens (lens equation, App. A), standardise them, take the exact order
 * statistics at the Chebyshev nodes with integer histograms and prefix scans,
 * fit the degree-D quantile polynomial and build the Hermite CDF knots.
 * Writes ev.cdf when non-null; the transform stays in the slot for rtu_forward. */
rtu_status rtu_build_grid(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream);

/* S1-S8 + S11: rtu_build_grid, then the GP source (Eq. 1-4: FFT filter of the
 * latents by sqrt(P), softplus and alpha_src), the supersampled ray trace
 * through the RTU map (Eq. 5) with bilinear interpolation (zero outside the
 * grid), the supersample average, the PSF convolution and the Gaussian
 * log-likelihood / chi^2 in the mask (Sec. 3.1, Sec. 4). */
rtu_status rtu_forward(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream);

/* S9: gradient of dlogL * log L with respect to latents, lens (and subhalo)
 * parameters and power-spectrum parameters, through the PSF, the bilinear
 * interpolation (atomic-free: rays counting-sorted by source cell, gathered per
 * node), the Hermite CDF, the polynomial fit and the order statistics, the
 * standardisation and the ray trace.  Ray positions are recomputed, not stored.
 * Must follow rtu_forward on the same stream with the same bindings/slot. */
rtu_status rtu_adjoint(rtu_system* const* sys, const rtu_eval* ev, int32_t n, void* stream);

/* ---------------------------------------------------------------------------
 * S10: stochastic variational inference (Sec. 4).  A mean-field Normal guide
 * over unconstrained sites: the non-latent sites (n_sites of them: theta_E,
 * gamma (RTU_EPL only), e1, e2, x0, y0, Gamma1, Gamma2; per subhalo kappa_s,
 * r_s, x_s, y_s (tau held fixed); the power-spectrum parameters and alpha_src)
 * then the n_src^2 latents (prior N(0, 1), Eq. 1).  Site i has prior priors[i]
 * (Table A1 families) on its value v = support-map(u); its physical parameter is
 * v (RTU_SPACE_LINEAR) or 10^v (RTU_SPACE_LOG10).  The guide is
 * u = loc + softplus(rho) eps with eps drawn on the device by Philox4x32-10
 * (Salmon et al. 2011; counter (e/2, sample, step, tag), key = seed) and
 * Box-Muller.  All state lives in the system's workspace.
 * ------------------------------------------------------------------------- */
enum { RTU_PRIOR_NORMAL = 0,        /* a = mean, b = sd                       */
       RTU_PRIOR_UNIFORM = 1,       /* on [a, b]                              */
       RTU_PRIOR_TRUNC_NORMAL = 2,  /* mean a, sd b, truncated to [c, d]      */
       RTU_PRIOR_LINEAR = 3 };      /* density prop. to 1 + a (v-c)/(d-c) on [c, d] */
enum { RTU_SPACE_LINEAR = 0, RTU_SPACE_LOG10 = 1 };
typedef struct {
    int32_t kind;
    int32_t space;
    double a, b, c, d;
} rtu_prior;

/* Number of non-latent sites of a system (0 on a bad desc). */
int32_t rtu_n_sites(const rtu_system_desc* desc);

/* Set the guide of one system (synchronous host copies into the workspace):
 * priors[n_sites]; fixed[8 + 5 n_sub + n_ps + 6 n_light] physical values that supply
 * the non-site entries (gamma of an SIE, tau of each subhalo) followed by the lens
 * light, which the ELBO step holds fixed (no lens-light sites); loc and rho
 * [n_sites + n_src^2] unconstrained locations and softplus-scale parameters;
 * tag = the system's random stream.  Resets Adam's moments and the step. */
rtu_status rtu_elbo_init(rtu_system* sys, const rtu_prior* priors, const double* fixed,
                         const double* loc, const double* rho, uint32_t tag);
/* The same with the state's upload ordered on `stream` (returns once the driver has
 * staged the bytes); ELBO steps ordered after it see the new guide. */
rtu_status rtu_elbo_init_on(rtu_system* sys, const rtu_prior* priors, const double* fixed,
                            const double* loc, const double* rho, uint32_t tag, void* stream);

/* One optimiser step for each of n systems: n_samples (1..8, <= desc.n_slots)
 * reparametrised guide samples, the batched rtu_forward + rtu_adjoint of every
 * sample, the Monte-Carlo ELBO
 *   (1/S) sum_s [log L(theta_s) + sum_sites (log p + log|dv/du|) + sum_latents log N(w)
 *                - log q(u_s)],
 * its gradient w.r.t. loc and rho, and an Adam ascent step (beta1 0.9, beta2
 * 0.999, eps 1e-8, learning rate lr).  elbo_out (device double[n], nullable)
 * receives each system's ELBO.  Stream-ordered. */
rtu_status rtu_elbo_step(rtu_system* const* sys, int32_t n, int32_t n_samples, uint64_t seed,
                         double lr, double* elbo_out, void* stream);

/* Checkpoint / resume of the guide and optimiser state: bytes of the blob,
 * export into / import from caller host memory (synchronous). */
size_t rtu_elbo_state_bytes(const rtu_system* sys);
/* The Monte-Carlo ELBO gradient of the system's last rtu_elbo_step (Sec. 4), before
 * the Adam update: d ELBO / d loc [n_sites + n_src^2] then d ELBO / d rho [same], as
 * doubles into caller host memory of at least 2 (n_sites + n_src^2) doubles
 * (synchronous; zeros before the first step). */
rtu_status rtu_elbo_grad(const rtu_system* sys, double* host, size_t bytes);
rtu_status rtu_elbo_export(const rtu_system* sys, void* host, size_t bytes);
rtu_status rtu_elbo_import(rtu_system* sys, const void* host, size_t bytes);

/* Replay of recorded launch sequences (on by default).  rtu_build_grid,
 * rtu_forward and rtu_adjoint record the kernel launches of a call into a CUDA
 * graph the second time they see its systems and evaluation arguments (every
 * pointer and size of the batch, the step, the precision) and replay that graph
 * on the caller's stream whenever a later call repeats them; the data behind the
 * pointers is read when the graph runs.  Calls made while per-kernel timing is
 * on, or on a stream the caller is capturing, launch plainly.  Per host thread
 * and device the 8 most recently used graphs are kept.  on = 0 switches replay
 * off and frees the calling thread's graphs on the current device.  Process-wide
 * switch; always returns RTU_OK. */
rtu_status rtu_graph_replay(int32_t on);

/* Per-kernel timing (tracing aid, off by default).  While enabled, every kernel
 * launch of every call is bracketed by two CUDA events recorded on the call's
 * stream.  rtu_profile_report waits for those events, then writes one line
 * "<kernel> <launches> <total_ms>" per kernel into buf (truncated to bytes,
 * always NUL-terminated) and clears the record.  Returns RTU_E_CUDA if an event
 * call fails.  Process-wide; guarded by a mutex. */
rtu_status rtu_profile_enable(int32_t on);
rtu_status rtu_profile_report(char* buf, size_t bytes);
/* The same records as a timeline: waits for the events, then writes one line
 * "<kernel> <stream> <start_ms> <end_ms>" per launch, in launch order, with times
 * relative to the start of the first recorded launch and <stream> 0 for the
 * call's stream, 1 for the library's side stream; clears the record like
 * rtu_profile_report (so call one or the other).  Returns RTU_E_CUDA if an event
 * call fails. */
rtu_status rtu_profile_timeline(char* buf, size_t bytes);

/* Self-test of the double-float arithmetic (pairs of floats, about 48 significant
 * bits) in which the FP32 path evaluates its FP64-class islands -- the centre
 * rays that build the CDF, the near-edge and near-core rays, the GP source -- on
 * the FP32 pipes (the paper fixes no precision; this checks the islands' own
 * arithmetic).  Device buffers: x of n (op 0-2) or 2n (op 3-5) doubles, each
 * converted to a double-float (hi = x rounded to float, lo = the rest rounded);
 * y of n doubles receives hi + lo of the result: op 0 exp(x[i]), 1 log(x[i]),
 * 2 sqrt(x[i]), 3 x[2i] / x[2i+1], 4 x[2i] x[2i+1], 5 x[2i] + x[2i+1]; and the
 * helpers of the near-edge pass's cell decision, 6 floor(x[i]) and 7 the distance of
 * x[i] from the nearest integer (in float), and of the cell gather, 8 the float pair
 * of the integer x[2i] (|x[2i]| < 2^48) scaled by 2^-x[2i+1] (0 <= x[2i+1] <= 122).
 * op 8 takes 2n doubles like ops 3-5.
 * Stream-ordered; RTU_E_ARG on a bad op or null buffers. */
rtu_status rtu_selftest_df(int32_t op, const double* x, double* y, int32_t n, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free variant of the GP source step (the paper has no counterpart).
 * For callers that cannot allocate device memory: an application that hands
 * this library no workspace because its device memory is planned up front, or
 * a process that must not call cudaMalloc after start-up.  It computes the same
 * source brightness as rtu_forward's GP source step: the latents (white noise)
 * filtered by the square root of the power spectrum through a forward and an
 * inverse FFT, then the softplus map and the alpha_src power; the transforms and
 * the map run in double and the result is rounded to float, like the workspace
 * path.  Device pointers: latents [n_src*n_src] floats, ps [n_family + 1]
 * doubles (alpha_src last) -> source [n_src*n_src] floats;
 * k = 2 pi |fftfreq| / src_pitch.  The caller owns all three buffers.
 * Its FFT scratch is one static device array of RTU_STATIC_MAX_NSRC^2 complex
 * doubles (256 KiB) that every GPU loading the library holds until exit; n_src
 * above RTU_STATIC_MAX_NSRC (or not 2^a 3^b, or below 4) returns RTU_E_ARG.
 * The call looks up that array's device address (with the current device) at
 * its first call on a device and again at every call not being captured into a
 * CUDA graph; a call made while the stream is captured uses the address of the
 * device's last uncaptured call, so make a first call before any capture (a
 * captured first call returns RTU_E_ARG).  The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  All calls share the
 * array and it keeps the last call's contents (each call overwrites all it
 * reads), so calls that overlap on the GPU -- e.g. on two streams at once --
 * race; serialise them. */
#define RTU_STATIC_MAX_NSRC 128
rtu_status rtu_gp_source_static(int32_t n_src, double src_pitch, int32_t ps_family, const float* latents,
                                const double* ps, float* source, void* stream);

/* Human-readable description of the last error on this host thread. */
const char* rtu_last_error(void);

/* Library version string. */
const char* rtu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RTU_H */
