"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 3.1).

This module only draws inputs; it contains none of the method's arithmetic
(no ray tracing, no transform, no source model).  Both the CUDA path's tests
and the oracle's tests take their inputs from here.

The paper's mocks use HST images of NGC galaxies as sources and the
SDSS J0946+1006 data; neither is available, so each input stands in for
them with the same shapes and structure:
  * data: an analytic Einstein-ring arc image (a Gaussian ring at the Einstein
    radius with a cos-modulated azimuthal brightness, two bright knots) plus
    Gaussian noise of rms sigma = peak/SNR;
  * arc mask: the pixels within a band around the ring (the arcs), like the
    paper's thresholded smoothed-SNR masks;
  * PSF: a K x K sampled Gaussian of the stated FWHM, normalised to sum 1;
  * latents: white noise N(0, 1) on the N_src x N_src grid (Eq. 1);
  * lens / power-spectrum parameters drawn from the stated ranges.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PROFILE_SIE, PROFILE_EPL = 0, 1
SUB_NONE, SUB_NFW, SUB_TNFW = 0, 1, 2
PS_POWER_LAW, PS_MATERN_LIKE, PS_MATERN = 0, 1, 2


@dataclass
class Mock:
    name: str
    n_img: int
    pix: float
    s_super: int
    n_src: int
    src_pitch: float
    profile: int
    ps_family: int
    sub_kind: int
    data: np.ndarray        # [n_img, n_img] float64
    mask: np.ndarray        # [n_img, n_img] uint8
    psf: np.ndarray         # [K, K] float64
    sigma: float
    lens: np.ndarray        # [8]  theta_E, gamma, e1, e2, x0, y0, G1, G2
    latents: np.ndarray     # [n_src, n_src]
    ps: np.ndarray          # [n_family_params + 1]  (..., alpha_src)
    subs: np.ndarray | None = None   # [n_sub, 5] kappa_s, r_s, tau, x_s, y_s
    light: np.ndarray | None = None  # [n_light, 6] MGE lens light: A, sigma, q, phi, x_n, y_n
    weights: np.ndarray | None = None  # [n_img, n_img] uint32 ray weights (weighted RTU grid)
    extra: dict = field(default_factory=dict)

    @property
    def n_rays(self):
        return self.n_img * self.n_img * self.s_super * self.s_super

    @property
    def n_mask(self):
        return int(self.mask.sum())


def gaussian_psf(k: int, fwhm_arcsec: float, pix: float) -> np.ndarray:
    """K x K Gaussian sampled at integer offsets, sigma = FWHM/(2 sqrt(2 ln 2)) pixels, sum 1."""
    sig = fwhm_arcsec / pix / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    c = (k - 1) / 2.0
    a = np.arange(k) - c
    g = np.exp(-0.5 * (a[:, None] ** 2 + a[None, :] ** 2) / sig ** 2)
    return g / g.sum()


def ellipticity(q: float, phi: float):
    c = (1.0 - q) / (1.0 + q)
    return c * math.cos(2.0 * phi), c * math.sin(2.0 * phi)


def _ring(n_img, pix, theta_E, width, x0, y0, rng):
    c = (np.arange(n_img) - (n_img - 1) / 2.0) * pix
    yy, xx = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(xx - x0, yy - y0)
    ang = np.arctan2(yy - y0, xx - x0)
    a1, a2 = rng.uniform(0, 2 * np.pi, size=2)
    arc = np.exp(-0.5 * ((r - theta_E) / width) ** 2)
    mod = 0.35 + 0.65 * (0.5 + 0.5 * np.cos(ang - a1)) + 0.8 * np.exp(-0.5 * ((ang - a2 + np.pi) % (2 * np.pi) - np.pi) ** 2 / 0.05)
    img = arc * mod
    mask = (np.abs(r - theta_E) < 3.0 * width).astype(np.uint8)
    return img / img.max(), mask


def _finish(name, n_img, pix, s, n_src, profile, family, lens, ps, rng, *, psf_k, fwhm, snr,
            width, sub_kind=SUB_NONE, subs=None, pitch=None):
    clean, mask = _ring(n_img, pix, lens[0], width, lens[4], lens[5], rng)
    sigma = 1.0 / snr
    data = clean + sigma * rng.standard_normal(clean.shape)
    latents = rng.standard_normal((n_src, n_src))
    if pitch is None:
        pitch = 3.0 * lens[0] / n_src
    return Mock(name=name, n_img=n_img, pix=pix, s_super=s, n_src=n_src, src_pitch=pitch,
                profile=profile, ps_family=family, sub_kind=sub_kind, data=data, mask=mask,
                psf=gaussian_psf(psf_k, fwhm, pix), sigma=sigma, lens=np.asarray(lens, np.float64),
                latents=latents, ps=np.asarray(ps, np.float64),
                subs=None if subs is None else np.asarray(subs, np.float64))


def mge_components(rng, n: int, x0: float, y0: float, amp: float = 1.0) -> np.ndarray:
    """Lens-light parameters of n Gaussian components (App. A.3): sigma log-uniform in
    [0.1, 1.0] arcsec and sorted, axis ratio U[0.6, 1], position angle U[0, pi), centres
    within 0.02" of the lens centre, amplitudes U[0.5, 1.5] x amp."""
    sig = np.sort(10 ** rng.uniform(-1.0, 0.0, size=n))
    rows = [[amp * rng.uniform(0.5, 1.5), sig[k], rng.uniform(0.6, 1.0), rng.uniform(0.0, math.pi),
             x0 + 0.02 * rng.standard_normal(), y0 + 0.02 * rng.standard_normal()] for k in range(n)]
    return np.asarray(rows, np.float64).reshape(n, 6)


def with_light(m: Mock, n: int = 5, seed: int = 0, amp: float = 0.3) -> Mock:
    """The mock with an n-component MGE lens light (its data are unchanged: the
    parity tests need identical inputs on both sides, not a realistic fit)."""
    rng = np.random.default_rng(seed)
    m.light = mge_components(rng, n, float(m.lens[4]), float(m.lens[5]), amp)
    return m


def with_snr_weights(m: Mock, cap: int = 100) -> Mock:
    """Integer ray weights from the pixel SNR (data / sigma, rounded, clipped to
    [1, cap]) -- one of the weightings Sec. 6.3 names for a weighted RTU grid."""
    m.weights = np.clip(np.rint(m.data / m.sigma), 1, cap).astype(np.uint32)
    return m


def _matern_like_amp(k0, pitch, rms=0.3):
    # continuum estimate of the field variance of A/(1+(k/k0)^2)^2 on a grid of this pitch
    return rms * rms * 4.0 * math.pi / (k0 * k0 * pitch * pitch)


def config_c1(seed: int = 0) -> Mock:
    """64^2 at 0.05"/pix, 2x2 rays, SIE theta_E=1.2 q=0.8 phi=30deg at (0,0) + shear
    (0.03, -0.02), 32^2 grid, P = k^-3 (A=1), 9x9 PSF FWHM 0.1", sigma = 0.02 (FP64 case)."""
    rng = np.random.default_rng(seed)
    e1, e2 = ellipticity(0.8, math.radians(30.0))
    lens = [1.2, 2.0, e1, e2, 0.0, 0.0, 0.03, -0.02]
    return _finish("c1", 64, 0.05, 2, 32, PROFILE_SIE, PS_POWER_LAW, lens, [1.0, 3.0, 1.0], rng,
                   psf_k=9, fwhm=0.1, snr=50.0, width=0.15)


def _epl_lens(rng, theta_lo=1.0, theta_hi=1.8):
    gamma = rng.uniform(1.8, 2.2)
    q = rng.uniform(0.6, 0.95)
    phi = rng.uniform(0.0, math.pi)
    thE = rng.uniform(theta_lo, theta_hi)
    x0, y0 = rng.normal(0.0, 0.05, size=2)
    g = 0.05 * math.sqrt(rng.uniform())
    ga = rng.uniform(0, 2 * math.pi)
    e1, e2 = ellipticity(q, phi)
    return [thE, gamma, e1, e2, x0, y0, g * math.cos(ga), g * math.sin(ga)]


def config_c2(seed: int = 1000, n_img: int = 200, s: int = 4, n_src: int = 64) -> Mock:
    """200^2 at 0.05"/pix, 4x4 rays, EPL (gamma U[1.8,2.2], q U[0.6,0.95]) + |shear| <= 0.05,
    64^2 grid, Matern-like P = A/(1+(k/k0)^2)^2 with k0 U[0.5,4]/arcsec, 21x21 PSF, SNR 50."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    k0 = rng.uniform(0.5, 4.0)
    pitch = 3.0 * lens[0] / n_src
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    return _finish(f"c2-{seed}", n_img, 0.05, s, n_src, PROFILE_EPL, PS_MATERN_LIKE, lens, ps, rng,
                   psf_k=21, fwhm=0.1, snr=50.0, width=0.25, pitch=pitch)


def config_c3(seed: int = 2000, n_img: int = 256, s: int = 3, n_src: int = 128) -> Mock:
    """256^2 at 0.05"/pix, 3x3 rays, SIE + shear (7 lens parameters), 128^2 latents,
    power-law P = A k^-beta (amplitude and slope), 9x9 PSF."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    lens[1] = 2.0
    ps = [rng.uniform(0.5, 2.0), rng.uniform(2.5, 3.5), rng.uniform(1.0, 2.0)]
    return _finish(f"c3-{seed}", n_img, 0.05, s, n_src, PROFILE_SIE, PS_POWER_LAW, lens, ps, rng,
                   psf_k=9, fwhm=0.1, snr=50.0, width=0.25)


def tnfw_from_mass(m_sun: float, tau: float = 10.0):
    """Simplified subhalo scaling anchored on the paper's Mock 1 truth (kappa_s = 10^0.3,
    r_s = 10^-1.42 arcsec, taken as a 1e10 Msun halo): r_s and kappa_s both scale as M^(1/3)."""
    f = (m_sun / 1e10) ** (1.0 / 3.0)
    return 10 ** 0.3 * f, 10 ** -1.42 * f, tau


def config_core(seed: int = 4000, n_img: int = 40, s: int = 2, n_src: int = 24) -> Mock:
    """The field of view on the lens core: n_img^2 pixels spanning 2.4 x 0.01 theta_E
    around the lens centre, so that about half of the rays lie within 0.01 theta_E of it
    (where the FP32 path traces rays in FP64); EPL + shear, Matern-like spectrum, a smooth
    blob as data and the whole field masked (a ring mask would hold no pixel here)."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    lens[4] = lens[5] = 0.0
    pix = 2.4 * 0.01 * lens[0] / n_img
    pitch = 3.0 * lens[0] / n_src
    k0 = rng.uniform(0.5, 4.0)
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    c = (np.arange(n_img) - (n_img - 1) / 2.0) / n_img
    yy, xx = np.meshgrid(c, c, indexing="ij")
    clean = np.exp(-0.5 * ((xx - 0.1) ** 2 + (yy + 0.05) ** 2) / 0.3 ** 2)
    sigma = 1.0 / 30.0
    data = clean + sigma * rng.standard_normal(clean.shape)
    latents = rng.standard_normal((n_src, n_src))
    return Mock(name=f"core-{seed}", n_img=n_img, pix=pix, s_super=s, n_src=n_src, src_pitch=pitch,
                profile=PROFILE_EPL, ps_family=PS_MATERN_LIKE, sub_kind=SUB_NONE, data=data,
                mask=np.ones((n_img, n_img), np.uint8), psf=gaussian_psf(5, 2.0 * pix, pix), sigma=sigma,
                lens=np.asarray(lens, np.float64), latents=latents, ps=np.asarray(ps, np.float64))


def config_bimodal(seed: int = 4500, n_img: int = 120, s: int = 2, n_src: int = 32, profile=PROFILE_EPL) -> Mock:
    """An arc mask of two disks of unequal size outside the Einstein ring on opposite
    sides of the lens (centred at +-2 theta_E on a line through the lens centre): their
    centre rays land near +-theta_E in the source plane, so each marginal along that
    line is bimodal, its quantile function jumps between the two clusters, and the
    degree-21 interpolant of App. C overshoots and falls between nodes -- the input that
    exercises the fit's monotonicity guard.  EPL + shear, Matern-like spectrum."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    if profile == PROFILE_SIE:
        lens[1] = 2.0
    pix = 6.0 * lens[0] / n_img
    pitch = 3.0 * lens[0] / n_src
    k0 = rng.uniform(0.5, 4.0)
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    m = _finish(f"bimodal-{seed}", n_img, pix, s, n_src, profile, PS_MATERN_LIKE, lens, ps, rng,
                psf_k=5, fwhm=2 * pix, snr=50.0, width=0.25, pitch=pitch)
    c = (np.arange(n_img) - (n_img - 1) / 2.0) * pix
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ang = rng.uniform(0.0, math.pi)
    cx, cy = 2.0 * lens[0] * math.cos(ang), 2.0 * lens[0] * math.sin(ang)
    r1, r2 = 0.30 * lens[0], 0.18 * lens[0]
    m.mask = ((np.hypot(xx - lens[4] - cx, yy - lens[5] - cy) < r1)
              | (np.hypot(xx - lens[4] + cx, yy - lens[5] + cy) < r2)).astype(np.uint8)
    return m


def config_outlier(seed: int = 4600, n_img: int = 201, s: int = 2, n_src: int = 48) -> Mock:
    """A c2-like system whose arc mask also holds the 3 x 3 pixels around the lens
    centre, with a steep power law (gamma = 2.6: alpha grows as |theta|^-0.6 towards the
    centre) centred ~1e-4 pixel off the central pixel's centre: that pixel's centre ray
    lands ~1000" away, its neighbours ~10", the ring's within ~1" -- a few far outliers
    that squeeze the ring's rays into a small fraction of the order statistics'
    histogram bins over [min, max] (tens of rays per bin at the node ranks)."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    lens[1] = 2.6
    pix = 0.05
    lens[4], lens[5] = 1.6e-4 * pix, -0.9e-4 * pix
    pitch = 3.0 * lens[0] / n_src
    k0 = rng.uniform(0.5, 4.0)
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    m = _finish(f"outlier-{seed}", n_img, pix, s, n_src, PROFILE_EPL, PS_MATERN_LIKE, lens, ps, rng,
                psf_k=9, fwhm=0.1, snr=50.0, width=0.25, pitch=pitch)
    c = (n_img - 1) // 2
    m.mask[c - 1:c + 2, c - 1:c + 2] = 1
    return m


def config_ties(seed: int = 4700, n_img: int = 301, s: int = 2, n_src: int = 48) -> Mock:
    """Many exactly tied centre-ray positions: an odd image whose central column sits at
    theta_x = 0, a lens centred on that column with position angle 0 (e2 = 0) and shear
    Gamma2 = 0, so every pixel of the column traces to beta_x = 0 exactly.  The arc mask
    is the half annulus x > 0, 1.3 theta_E < |theta| < 2.5 theta_E (outside the critical
    curve: beta_x > 0 there) plus 121 pixels of the column: a block of 121 tied rays at
    the bottom of the x marginal, ~0.7% of the sample, covering the first Chebyshev
    node's ranks and no other."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng)
    q = rng.uniform(0.75, 0.95)
    lens[2], lens[3] = ellipticity(q, 0.0)
    lens[4] = 0.0
    lens[7] = 0.0
    pix = 0.025
    pitch = 3.0 * lens[0] / n_src
    k0 = rng.uniform(0.5, 4.0)
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    m = _finish(f"ties-{seed}", n_img, pix, s, n_src, PROFILE_EPL, PS_MATERN_LIKE, lens, ps, rng,
                psf_k=9, fwhm=0.05, snr=50.0, width=0.12, pitch=pitch)
    c = (np.arange(n_img) - (n_img - 1) / 2.0) * pix
    yy, xx = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(xx, yy - lens[5])
    m.mask = ((xx > 0.5 * pix) & (r > 1.3 * lens[0]) & (r < 2.5 * lens[0])).astype(np.uint8)
    mid = (n_img - 1) // 2
    m.mask[mid - 60:mid + 61, mid] = 1
    return m


def config_c4(seed: int = 3000, with_subs: bool = True, n_img: int = 400, s: int = 3,
              n_src: int = 128) -> Mock:
    """400^2 at 0.03"/pix, 3x3 rays, EPL + shear + 1-10 truncated NFW subhaloes
    (log10 M U[8,10], on the ring), 128^2 grid, 21x21 PSF FWHM 0.06"."""
    rng = np.random.default_rng(seed)
    lens = _epl_lens(rng, 1.5, 2.5)
    k0 = rng.uniform(0.5, 4.0)
    pitch = 3.0 * lens[0] / n_src
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    subs = None
    kind = SUB_NONE
    nsub = int(rng.integers(1, 11))
    rows = []
    for _ in range(nsub):
        m = 10 ** rng.uniform(8.0, 10.0)
        ks, rs, tau = tnfw_from_mass(m)
        ang = rng.uniform(0, 2 * math.pi)
        rad = lens[0] * (1.0 + rng.normal(0.0, 0.05))
        rows.append([ks, rs, tau, lens[4] + rad * math.cos(ang), lens[5] + rad * math.sin(ang)])
    if with_subs:
        subs = np.array(rows)
        kind = SUB_TNFW
    return _finish(f"c4-{seed}{'' if with_subs else '-smooth'}", n_img, 0.03, s, n_src,
                   PROFILE_EPL, PS_MATERN_LIKE, lens, ps, rng, psf_k=21, fwhm=0.06, snr=50.0,
                   width=0.25, sub_kind=kind, subs=subs, pitch=pitch)


def config_tiny(seed: int = 7, n_img: int = 12, s: int = 2, n_src: int = 8, profile=PROFILE_EPL,
                family=PS_MATERN_LIKE, psf_k=3, sub_kind=SUB_NONE, n_sub=0) -> Mock:
    """A tiny system for brute-force checks (finite differences, naive DFT)."""
    rng = np.random.default_rng(seed)
    pix = 3.6 / n_img
    lens = _epl_lens(rng, 1.0, 1.3)
    if profile == PROFILE_SIE:
        lens[1] = 2.0
    pitch = 3.0 * lens[0] / n_src
    if family == PS_MATERN_LIKE:
        k0 = rng.uniform(0.5, 4.0)
        ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    elif family == PS_POWER_LAW:
        ps = [rng.uniform(0.5, 2.0), rng.uniform(2.5, 3.5), rng.uniform(1.0, 2.0)]
    else:
        ps = [rng.uniform(0.1, 0.3), rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0), rng.uniform(1.0, 2.0)]
    subs = None
    if sub_kind != SUB_NONE:
        rows = []
        for _ in range(n_sub):
            ks, rs, tau = tnfw_from_mass(10 ** rng.uniform(9.0, 10.0))
            ang = rng.uniform(0, 2 * math.pi)
            rows.append([ks, rs * 5.0, tau, lens[0] * math.cos(ang), lens[0] * math.sin(ang)])
        subs = np.array(rows)
    m = _finish(f"tiny-{seed}", n_img, pix, s, n_src, profile, family, lens, ps, rng,
                psf_k=psf_k, fwhm=2 * pix, snr=20.0, width=0.35, sub_kind=sub_kind, subs=subs,
                pitch=pitch)
    # an asymmetric PSF catches a flipped kernel
    m.psf = m.psf * (1.0 + 0.3 * rng.uniform(size=m.psf.shape))
    m.psf /= m.psf.sum()
    return m


SERVE_IMG = (64, 96, 128, 192, 256)
SERVE_SRC = (32, 48, 64, 96, 128)
SERVE_S = (2, 3, 4)


def config_serving_system(seed: int, n_img: int | None = None, n_src: int | None = None,
                          s: int | None = None) -> Mock:
    """One request of the serving stream: image size U{64..256}, grid U{32..128},
    supersampling U{2,3,4}, SIE or EPL + shear with equal odds (a size given fixes it)."""
    rng = np.random.default_rng(seed)
    n_img_d = int(rng.choice(SERVE_IMG))
    n_src_d = int(rng.choice(SERVE_SRC))
    s_d = int(rng.choice(SERVE_S))
    n_img = n_img_d if n_img is None else int(n_img)
    n_src = n_src_d if n_src is None else int(n_src)
    s = s_d if s is None else int(s)
    profile = PROFILE_SIE if rng.uniform() < 0.5 else PROFILE_EPL
    lens = _epl_lens(rng, 0.8, 1.3)
    if profile == PROFILE_SIE:
        lens[1] = 2.0
    pix = 4.0 / n_img
    pitch = 3.0 * lens[0] / n_src
    k0 = rng.uniform(0.5, 4.0)
    ps = [_matern_like_amp(k0, pitch), k0, rng.uniform(1.0, 2.0)]
    return _finish(f"serve-{seed}", n_img, pix, s, n_src, profile, PS_MATERN_LIKE, lens, ps, rng,
                   psf_k=9, fwhm=2 * pix, snr=50.0, width=0.2, pitch=pitch)


def poisson_arrivals(n: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


# ---------------------------------------------------------------------------
# priors of the variational fit (Table A1) -- inputs to both sides
# ---------------------------------------------------------------------------
PRIOR_NORMAL, PRIOR_UNIFORM, PRIOR_TRUNC_NORMAL, PRIOR_LINEAR = 0, 1, 2, 3
SPACE_LINEAR, SPACE_LOG10 = 0, 1


def default_priors(profile, sub_kind, n_sub, family, subs=None):
    """Prior (kind, space, a, b, c, d) of each non-latent site, in the site order
    theta_E, [gamma], e1, e2, x0, y0, Gamma1, Gamma2, per subhalo (log10 kappa_s,
    log10 r_s, x_s, y_s), power-spectrum parameters, log10 alpha_src.

    Table A1: theta_E U(-10,15); gamma G(2, 0.2) on [1, 3]; e G(0, 0.1); centre
    G(0, 0.5); shear U(-0.2, 0.2); log10 kappa_s U(-10, 4); log10 r_s U(-4, 4);
    subhalo position G(guess, 0.05); n_src T(-1, 0.1, 10); zeta 10^G(2.1, 1.1);
    sigma_src 10^U(-5, 2); alpha_src 10^U(-1, 1).  The power-law and Matern-like
    spectra are not in the paper: A 10^U(-6, 6), beta U(1, 5), k0 10^G(0.3, 1)."""
    U, G, TG, T = PRIOR_UNIFORM, PRIOR_NORMAL, PRIOR_TRUNC_NORMAL, PRIOR_LINEAR
    L, LG = SPACE_LINEAR, SPACE_LOG10
    p = [(U, L, -10.0, 15.0, 0.0, 0.0)]
    if profile == PROFILE_EPL:
        p.append((TG, L, 2.0, 0.2, 1.0, 3.0))
    p += [(G, L, 0.0, 0.1, 0, 0), (G, L, 0.0, 0.1, 0, 0), (G, L, 0.0, 0.5, 0, 0), (G, L, 0.0, 0.5, 0, 0),
          (U, L, -0.2, 0.2, 0, 0), (U, L, -0.2, 0.2, 0, 0)]
    for h in range(n_sub if sub_kind else 0):
        gx, gy = (0.0, 0.0) if subs is None else (float(subs[h][3]), float(subs[h][4]))
        p += [(U, LG, -10.0, 4.0, 0, 0), (U, LG, -4.0, 4.0, 0, 0), (G, L, gx, 0.05, 0, 0), (G, L, gy, 0.05, 0, 0)]
    if family == PS_POWER_LAW:
        p += [(U, LG, -6.0, 6.0, 0, 0), (U, L, 1.0, 5.0, 0, 0)]
    elif family == PS_MATERN_LIKE:
        p += [(U, LG, -6.0, 6.0, 0, 0), (G, LG, 0.3, 1.0, 0, 0)]
    else:
        p += [(U, LG, -5.0, 2.0, 0, 0), (T, L, -1.0, 0.0, 0.1, 10.0), (G, LG, 2.1, 1.1, 0, 0)]
    p.append((U, LG, -1.0, 1.0, 0, 0))
    return p


def unconstrain(v, prior):
    """Unconstrained start value u of a site whose constrained value is v (the
    inverse of the site's support map): identity for normal priors, the logit of
    the position inside the interval otherwise."""
    kind, _space, a, b, c, d = prior
    if kind == PRIOR_NORMAL:
        return float(v)
    lo, hi = (a, b) if kind == PRIOR_UNIFORM else (c, d)
    t = (v - lo) / (hi - lo)
    t = min(max(t, 1e-12), 1 - 1e-12)
    return math.log(t / (1.0 - t))
