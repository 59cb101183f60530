"""FP64 CPU oracle for the RTU-grid lensing hot path (Enzi et al., "Gaussian
processes on ray-guided transformed uniform grids").

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may call this module; the product path (the
CUDA library and its Python binding) never imports it and shares no code with
it.

Plain, slow, obviously correct: every step is written out in float64 with
plain PyTorch CPU tensor ops in the paper's order and notation.  Library
primitives used as steps: ``torch.sort`` (order statistics), ``torch.fft``
(the FFT of Eq. 1), ``torch.linalg.solve`` (the polynomial fit) and
``torch.autograd`` (the gradient of log L / ELBO is by definition the
derivative of the forward model; autograd evaluates it exactly up to
rounding).

Passages followed (paper sections / equations):
  * pixel grid and supersampling ............ Sec. 2.3, Sec. 3.1
  * EPL convergence (Eq. A1) ................ App. A.1; deflection by the
    Tessore & Metcalf (2015) hypergeometric series (the paper gives kappa only)
  * external shear .......................... App. A.1
  * NFW (Eq. A2-A3), truncated NFW .......... App. A.2; truncation after
    Baltz, Marshall & Oguri (2009)
  * arc-mask centre rays, standardisation ... App. C step i, Sec. 2.2 footnote
  * marginal eCDFs / quantile function ...... Sec. 2.2, App. C step ii
  * weighted eCDFs (weighted RTU grid) ...... Sec. 6.3 (extension)
  * Chebyshev-node polynomial fit of the QF . App. C step iii (order 21)
  * cubic Hermite spline inverse (the CDF) .. App. C step iv
  * unsmoothed linear-interpolated eCDF ..... App. C (first paragraph)
  * copula map y = g(x) (Eq. 5) ............. Sec. 2.2
  * GP source f = F^-1(sqrt(P) xi) (Eq. 1) .. Sec. 2.1; Matern P(k) (Eq. 4)
  * softplus positivity (Eq. 2-3) ........... Sec. 2.1
  * bilinear interpolation, zero outside .... Sec. 2.1
  * supersample average, PSF, Gaussian noise  Sec. 2.3, Sec. 3.1
  * multi-Gaussian lens light ............... App. A.3
  * likelihood / chi^2 in the mask .......... Sec. 4
  * SVI ELBO with a Normal guide ............ Sec. 4 (location and scale)

Where the paper is silent or ambiguous, the function that takes a reading
says which one.  Parity unpinned (no independent pin exists):
the linear prior T(a, lo, hi) of Table A1, whose definition lives in a cited
paper that is not reproduced here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

DT = torch.float64
S0 = 0.01  # softplus transition scale s_0 (Eq. 3)

# lens-profile and family codes (shared *numbering* with the C ABI header;
# the numbers are an interface, not code)
PROFILE_SIE = 0
PROFILE_EPL = 1
SUB_NONE = 0
SUB_NFW = 1
SUB_TNFW = 2
PS_POWER_LAW = 0    # P = A k^-beta, P(0) = 0             params (A, beta)
PS_MATERN_LIKE = 1  # P = A / (1 + (k/k0)^2)^2             params (A, k0)
PS_MATERN = 2       # Eq. 4                                 params (sigma, n, zeta)
N_PS_PARAMS = {PS_POWER_LAW: 2, PS_MATERN_LIKE: 2, PS_MATERN: 3}
N_LENS = 8          # theta_E, gamma, e1, e2, x0, y0, Gamma1, Gamma2
N_SUB_PARAMS = 5    # kappa_s, r_s, tau, x_s, y_s

FLAG_NONMONOTONE = 1
TRANSFORM_RTU = 0       # the ray-guided transformed uniform grid (Sec. 2.2)
TRANSFORM_UNIFORM = 1   # the uniform grid over the masked rays' square box (Sec. 2.1)
TRANSFORM_LINEAR = 2    # the unsmoothed eCDF, linearly interpolated (App. C, first paragraph)


# ---------------------------------------------------------------------------
# image-plane rays (Sec. 2.3: s_super x s_super sub-rays per pixel)
# ---------------------------------------------------------------------------
def pixel_centres(n_img: int, pix: float):
    """Pixel (i, j) -> theta = ((i-(N-1)/2) pix, (j-(N-1)/2) pix); row-major [j][i]."""
    c = (torch.arange(n_img, dtype=DT) - (n_img - 1) / 2.0) * pix
    yy, xx = torch.meshgrid(c, c, indexing="ij")
    return xx.reshape(-1), yy.reshape(-1)


def subray_positions(n_img: int, pix: float, s: int):
    """Sub-ray (a, b) of a pixel sits at ((a+1/2)/s - 1/2) pix from its centre.

    Returns x, y of shape [n_img*n_img, s*s]; sub-ray index b*s + a."""
    xc, yc = pixel_centres(n_img, pix)
    off = ((torch.arange(s, dtype=DT) + 0.5) / s - 0.5) * pix
    oy, ox = torch.meshgrid(off, off, indexing="ij")
    return xc[:, None] + ox.reshape(1, -1), yc[:, None] + oy.reshape(1, -1)


# ---------------------------------------------------------------------------
# deflections (App. A)
# ---------------------------------------------------------------------------
def ellipticity_to_q_phi(e1, e2):
    """(e1, e2) = (1-q)/(1+q) (cos 2phi, sin 2phi); phi from +x, counter-clockwise."""
    c = torch.sqrt(e1 * e1 + e2 * e2)
    q = (1.0 - c) / (1.0 + c)
    phi = 0.5 * torch.atan2(e2, e1)
    return q, phi


def deflection_epl(x, y, theta_E, gamma, e1, e2, x0, y0, rel_tol=1e-17, max_terms=4000):
    """Deflection of kappa = (3-gamma)/2 (theta_E/rho)^(gamma-1), Eq. A1, with
    rho^2 = q x'^2 + y'^2/q in the frame centred on (x0, y0) and rotated by phi.

    Tessore & Metcalf (2015): with R^2 = q^2 x'^2 + y'^2 (= q rho^2),
    b = theta_E sqrt(q), t = gamma - 1, f = (1-q)/(1+q) and e^{i vphi} =
    (q x' + i y')/R, the complex deflection in the rotated frame is
        alpha' = 2b/(1+q) (b/R)^(t-1) sum_n Omega_n,
        Omega_0 = e^{i vphi},
        Omega_n = -f (2n-(2-t))/(2n+(2-t)) e^{2 i vphi} Omega_{n-1},
    the series of 2F1(1, t/2; 2-t/2; -f e^{2 i vphi}).  Summed until the term is
    below rel_tol.  R is clamped at 1e-10 arcsec (the singular centre)."""
    q, phi = ellipticity_to_q_phi(e1, e2)
    cp, sp = torch.cos(phi), torch.sin(phi)
    dx, dy = x - x0, y - y0
    xr = cp * dx + sp * dy
    yr = -sp * dx + cp * dy
    t = gamma - 1.0
    b = theta_E * torch.sqrt(q)
    R = torch.sqrt(q * q * xr * xr + yr * yr).clamp_min(1e-10)
    eiv = torch.complex(q * xr / R, yr / R)
    e2iv = eiv * eiv
    f = (1.0 - q) / (1.0 + q)
    term = eiv
    total = term
    for n in range(1, max_terms):
        term = term * e2iv * (-f * (2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t)))
        total = total + term
        if float(term.detach().abs().max()) <= rel_tol:
            break
    pref = 2.0 * b / (1.0 + q) * torch.pow(b / R, t - 1.0)
    axr = pref * total.real
    ayr = pref * total.imag
    return cp * axr - sp * ayr, sp * axr + cp * ayr


def deflection_shear(x, y, g1, g2):
    """External shear about the origin: potential psi = g1 (x^2-y^2)/2 + g2 x y."""
    return g1 * x + g2 * y, g2 * x - g1 * y


def _safe_F(x):
    """F(x) of Eq. A3: atan(sqrt(x^2-1))/sqrt(x^2-1) (x>1), atanh(sqrt(1-x^2))/sqrt(1-x^2) (x<1).

    Near x = 1 both branches equal the series sum_k w^k/(2k+1), w = 1-x^2."""
    w = 1.0 - x * x
    near = w.abs() < 1e-2
    ws = torch.where(near, w, torch.zeros_like(w))
    ser = torch.zeros_like(x)
    p = torch.ones_like(x)
    for k in range(0, 14):
        ser = ser + p / (2 * k + 1)
        p = p * ws
    lo = (w > 0) & ~near
    hi = (w < 0) & ~near
    sl = torch.sqrt(torch.where(lo, w, torch.full_like(w, 0.5)))
    sh = torch.sqrt(torch.where(hi, -w, torch.full_like(w, 0.5)))
    f_lo = torch.atanh(sl) / sl
    f_hi = torch.atan(sh) / sh
    return torch.where(near, ser, torch.where(lo, f_lo, f_hi))


def nfw_convergence(r, kappa_s, r_s):
    """Eq. A3: kappa = 2 kappa_s (1 - F(x)) / (x^2 - 1), x = r / r_s."""
    x = r / r_s
    w = 1.0 - x * x
    near = w.abs() < 1e-2
    # (1-F)/(x^2-1) = (F-1)/w = sum_{k>=1} w^(k-1)/(2k+1) near x = 1
    ws = torch.where(near, w, torch.zeros_like(w))
    ser = torch.zeros_like(x)
    p = torch.ones_like(x)
    for k in range(1, 15):
        ser = ser + p / (2 * k + 1)
        p = p * ws
    wsafe = torch.where(near, torch.ones_like(w), w)
    far = (_safe_F(x) - 1.0) / wsafe
    return 2.0 * kappa_s * torch.where(near, ser, far)


def _nfw_mass_fn(x):
    """h(x) = ln(x/2) + F(x): alpha(r) = 4 kappa_s r_s h(x)/x for Eq. A3."""
    return torch.log(x / 2.0) + _safe_F(x)


def _tnfw_mass_fn(x, tau):
    """Projected-mass function of the tau-truncated NFW (Baltz, Marshall & Oguri
    2009, rho = rho_NFW tau^2/(tau^2 + x^2)); tends to h(x) as tau -> infinity."""
    t2 = tau * tau
    sq = torch.sqrt(t2 + x * x)
    L = torch.log(x / (sq + tau))
    return t2 / (t2 + 1.0) ** 2 * (
        (t2 + 1.0 + 2.0 * (x * x - 1.0)) * _safe_F(x)
        + tau * math.pi
        + (t2 - 1.0) * torch.log(tau)
        + sq * (-math.pi + L * (t2 - 1.0) / tau)
    )


def deflection_nfw(x, y, kappa_s, r_s, tau, xs, ys, kind):
    """Radial deflection of an (optionally truncated) NFW subhalo centred at (xs, ys)."""
    dx, dy = x - xs, y - ys
    r = torch.sqrt(dx * dx + dy * dy).clamp_min(1e-10)
    xx = r / r_s
    g = _nfw_mass_fn(xx) if kind == SUB_NFW else _tnfw_mass_fn(xx, tau)
    a = 4.0 * kappa_s * r_s * g / xx / r
    return a * dx, a * dy


def trace(x, y, lens, profile, subs=None, sub_kind=SUB_NONE):
    """Lens equation beta = theta - sum alpha (App. A); lens = [thE, gamma, e1, e2, x0, y0, G1, G2]."""
    gamma = lens[1] if profile == PROFILE_EPL else torch.tensor(2.0, dtype=DT)
    ax, ay = deflection_epl(x, y, lens[0], gamma, lens[2], lens[3], lens[4], lens[5])
    sx, sy = deflection_shear(x, y, lens[6], lens[7])
    ax, ay = ax + sx, ay + sy
    if subs is not None and sub_kind != SUB_NONE:
        for h in range(subs.shape[0]):
            p = subs[h]
            nx, ny = deflection_nfw(x, y, p[0], p[1], p[2], p[3], p[4], sub_kind)
            ax, ay = ax + nx, ay + ny
    return x - ax, y - ay


# ---------------------------------------------------------------------------
# the RTU transform (Sec. 2.2, App. C)
# ---------------------------------------------------------------------------
def chebyshev_nodes(m: int):
    """u_j = (1 - cos((2j-1) pi / (2m)))/2, j = 1..m (ascending, inside (0, 1))."""
    j = torch.arange(1, m + 1, dtype=DT)
    return (1.0 - torch.cos((2.0 * j - 1.0) * math.pi / (2.0 * m))) / 2.0


def chebyshev_T(t, degree):
    """[len(t), degree+1] matrix of T_k(t) by the three-term recurrence."""
    cols = [torch.ones_like(t), t]
    for _ in range(2, degree + 1):
        cols.append(2.0 * t * cols[-1] - cols[-2])
    return torch.stack(cols[: degree + 1], dim=-1)


def chebyshev_dT(t, degree):
    """[len(t), degree+1] matrix of dT_k/dt = k U_{k-1}(t)."""
    U = [torch.ones_like(t), 2.0 * t]
    for _ in range(2, degree + 1):
        U.append(2.0 * t * U[-1] - U[-2])
    cols = [torch.zeros_like(t)] + [k * U[k - 1] for k in range(1, degree + 1)]
    return torch.stack(cols, dim=-1)


def quantile_type7(sorted_vals, u):
    """Empirical quantile (linear interpolation of order statistics, h = u (N-1))."""
    n = sorted_vals.shape[0]
    h = u * (n - 1)
    k = torch.floor(h).long().clamp(0, n - 1)
    k1 = (k + 1).clamp(max=n - 1)
    frac = h - k.to(DT)
    return sorted_vals[k] + frac * (sorted_vals[k1] - sorted_vals[k])


def quantile_weighted(sorted_vals, sorted_w, u):
    """Weighted empirical quantile: the type-7 quantile of the sample in which
    value i appears w_i times (w positive integers; weighted RTU grid, Sec. 6.3):
    h = u (W - 1) with W = sum w, and the expanded element of rank r is the value
    whose cumulative weight first exceeds r."""
    cw = torch.cumsum(sorted_w.to(torch.int64), 0)
    W = int(cw[-1])
    h = u * (W - 1)
    r = torch.floor(h).long().clamp(0, W - 1)
    r1 = (r + 1).clamp(max=W - 1)
    k = torch.searchsorted(cw, r, right=True)
    k1 = torch.searchsorted(cw, r1, right=True)
    frac = h - r.to(DT)
    return sorted_vals[k] + frac * (sorted_vals[k1] - sorted_vals[k])


@dataclass
class RTUTransform:
    """Per-axis smoothed CDF: mu, sigma_min and the Hermite knots (z-space)."""
    mu: torch.Tensor            # [2]
    sigma: torch.Tensor         # scalar sigma_min
    knots: torch.Tensor         # [2, M+2]  X_0 = p(0), X_j = p(u_j), X_{M+1} = p(1)
    values: torch.Tensor        # [M+2]     0, u_1..u_M, 1
    slopes: torch.Tensor        # [2, M+2]  dC/dz = 1 / p'(u)
    coeffs: torch.Tensor        # [2, D+1]  Chebyshev coefficients of the QF
    q_nodes: torch.Tensor       # [2, M]    empirical QF at the nodes
    flags: int = 0
    n_centre: int = 0
    extra: dict = field(default_factory=dict)


def standardise(bx, by):
    """App. C step i: mean per axis and sigma_min = min(std_x, std_y) (ddof 0, tie -> x)."""
    mu = torch.stack([bx.mean(), by.mean()])
    sx = torch.sqrt(((bx - mu[0]) ** 2).mean())
    sy = torch.sqrt(((by - mu[1]) ** 2).mean())
    sigma = sx if float(sx.detach()) <= float(sy.detach()) else sy
    return mu, sigma


SEL_BINS = 65536


def selection_histogram(values, weights=None, nbins=SEL_BINS):
    """The integer histogram behind the exact order statistics of one axis (App. C
    step ii: the eCDF's counts): nbins equal bins over [min, max] of the traced centre
    positions, value v in bin floor((v - min) * (nbins / (max - min))) clamped to
    [0, nbins - 1] (every value in bin 0 when max = min); each ray adds its integer
    weight (1 when unweighted).  Bit-exact for identical positions: one subtraction,
    one division and one product, each correctly rounded in float64."""
    v = values.detach().to(DT)
    lo, hi = float(v.min()), float(v.max())
    scale = nbins / (hi - lo) if hi > lo else 0.0
    b = torch.floor((v - lo) * scale).clamp(0, nbins - 1).long()
    w = torch.ones_like(b) if weights is None else weights.to(torch.int64)
    h = torch.zeros(nbins, dtype=torch.int64)
    return h.index_add_(0, b, w)


def fit_qf_polynomial(zs, u, degree, ws=None):
    """App. C step iii: Chebyshev coefficients c of p(u) = sum_k c_k T_k(2u-1) fitted to
    the empirical QF at the nodes u.  The paper takes as many Chebyshev nodes as the
    order of the fit; with M = degree+1 nodes the fit is the interpolant (the node
    weights -- the eCDF slopes -- drop out of a square solve), which is the reading
    taken here; other node counts are rejected.  ws: ray weights in the order of zs
    (weighted RTU grid), else every ray counts once."""
    m = u.shape[0]
    if m != degree + 1:
        raise ValueError("the quantile fit takes M = degree + 1 Chebyshev nodes")
    V = chebyshev_T(2.0 * u - 1.0, degree)
    Q = quantile_type7(zs, u) if ws is None else quantile_weighted(zs, ws, u)
    return torch.linalg.solve(V, Q), Q


def hermite_knots(c, u, degree, guard_eps=1e-6):
    """App. C step iv: knots X = p(0), p(u_1..u_M), p(1) and CDF slopes 1/p'(u) there.

    Monotonicity guard: p' >= eps*span, X_{j+1} >= X_j + eps*span with
    span = p(1) - p(0); returns (X, slopes, repaired?)."""
    t = torch.cat([torch.tensor([-1.0], dtype=DT), 2.0 * u - 1.0, torch.tensor([1.0], dtype=DT)])
    X = chebyshev_T(t, degree) @ c
    dp = (chebyshev_dT(t, degree) * 2.0) @ c
    repaired = False
    span = X[-1] - X[0]
    if float(span.detach()) <= 0.0:
        repaired = True
        span = span.abs() + 1e-300
    floor_d = guard_eps * span
    if bool((dp.detach() < floor_d.detach()).any()):
        repaired = True
    dp = torch.maximum(dp, floor_d)
    Xr = [X[0]]
    for j in range(1, X.shape[0]):
        lim = Xr[-1] + floor_d
        if float(X[j].detach()) < float(lim.detach()):
            repaired = True
        Xr.append(torch.maximum(X[j], lim))
    return torch.stack(Xr), 1.0 / dp, repaired


def fit_transform(bx, by, n_nodes=22, degree=21, guard_eps=1e-6, weights=None):
    """App. C steps i-iv from the traced centre rays (bx, by): standardise, sort each
    marginal (the eCDF, weighted by the rays' integer weights when given -- the
    weighted RTU grid of Sec. 6.3), fit the QF polynomial at the Chebyshev nodes, and
    build the Hermite CDF (values u_j at knots p(u_j), slopes 1/p'(u_j), linear beyond
    the ends).  The standardisation (step i) is unweighted."""
    mu, sigma = standardise(bx, by)
    u = chebyshev_nodes(n_nodes)
    flags = 0
    knots, slopes, coeffs, qn = [], [], [], []
    for a, b in enumerate((bx, by)):
        zs, order = torch.sort((b - mu[a]) / sigma, stable=True)
        c, Q = fit_qf_polynomial(zs, u, degree, None if weights is None else weights[order])
        X, d, rep = hermite_knots(c, u, degree, guard_eps)
        if rep:
            flags |= FLAG_NONMONOTONE
        knots.append(X)
        slopes.append(d)
        coeffs.append(c)
        qn.append(Q)
    values = torch.cat([torch.zeros(1, dtype=DT), u, torch.ones(1, dtype=DT)])
    return RTUTransform(mu=mu, sigma=sigma, knots=torch.stack(knots), values=values,
                        slopes=torch.stack(slopes), coeffs=torch.stack(coeffs),
                        q_nodes=torch.stack(qn), flags=flags, n_centre=bx.shape[0])


def hermite_cdf(z, X, U, d):
    """Cubic Hermite spline through (X_j, U_j) with slopes d_j; linear extrapolation
    beyond the end knots (so C can leave [0, 1])."""
    m = X.shape[0]
    j = (torch.searchsorted(X.detach(), z.detach(), right=True) - 1).clamp(0, m - 2)
    x0, x1 = X[j], X[j + 1]
    h = x1 - x0
    t = (z - x0) / h
    t2, t3 = t * t, t * t * t
    h00 = 2 * t3 - 3 * t2 + 1
    h10 = t3 - 2 * t2 + t
    h01 = -2 * t3 + 3 * t2
    h11 = t3 - t2
    inner = h00 * U[j] + h10 * h * d[j] + h01 * U[j + 1] + h11 * h * d[j + 1]
    left = U[0] + d[0] * (z - X[0])
    right = U[-1] + d[-1] * (z - X[-1])
    return torch.where(z < X[0], left, torch.where(z >= X[-1], right, inner))


@dataclass
class BoxTransform:
    """The old approach's uniform grid (Sec. 2.1): the smallest square box that
    contains every masked ray, mapped affinely onto the unit square."""
    lo: torch.Tensor        # [2] lower corner
    side: torch.Tensor      # box side
    flags: int = 0


def uniform_box(bx, by):
    """Square box around the masked centre rays: centred on each axis's range, side =
    the larger range (tie -> x)."""
    mins = torch.stack([bx.min(), by.min()])
    maxs = torch.stack([bx.max(), by.max()])
    rng = maxs - mins
    side = rng[0] if float(rng[0].detach()) >= float(rng[1].detach()) else rng[1]
    centre = 0.5 * (mins + maxs)
    return BoxTransform(lo=centre - 0.5 * side, side=side)


@dataclass
class LinearTransform:
    """The first-order transform of App. C: the marginal eCDFs of the standardised
    centre rays, linearly interpolated between the observations."""
    mu: torch.Tensor        # [2] standardisation (App. C step i)
    sigma: torch.Tensor
    knots: torch.Tensor     # [2, n] sorted standardised centre positions per axis
    flags: int = 0


def linear_ecdf_transform(bx, by):
    """App. C step i (standardise) and step ii (sort each marginal: the eCDF's
    observations).  No fit: the map interpolates the eCDF directly."""
    mu, sigma = standardise(bx, by)
    knots = [torch.sort((b - mu[a]) / sigma).values for a, b in enumerate((bx, by))]
    return LinearTransform(mu=mu, sigma=sigma, knots=torch.stack(knots))


def linear_ecdf(z, X):
    """The eCDF of the sorted observations X (n >= 2) interpolated linearly: the
    k-th observation (0-based) maps to k/(n-1) -- the inverse of the type-7 quantile
    function -- and between observations the map is linear.

    Readings (the paper gives the interpolation only): beyond the end observations
    the map continues with the slope of the end segment, as the smoothed CDF
    continues linearly beyond its end knots, so rays there leave [0, 1] and see a
    zero source; with k the last observation <= z (clamped to [0, n-2]) a segment of
    zero width (tied observations at an end) contributes a constant k/(n-1)."""
    n = X.shape[0]
    k = (torch.searchsorted(X.detach(), z.detach(), right=True) - 1).clamp(0, n - 2)
    x0, x1 = X[k], X[k + 1]
    h = x1 - x0
    ok = h.detach() > 0
    t = torch.where(ok, (z - x0) / torch.where(ok, h, torch.ones_like(h)), torch.zeros_like(z))
    return (k.to(DT) + t) / (n - 1)


def rtu_map(bx, by, T):
    """Source-grid coordinates of source-plane positions: for the RTU grid Eq. 5,
    y = g(x) = (C_1(z_1), C_2(z_2)) with z = (beta - mu)/sigma_min; for the uniform
    grid the affine box map y = (beta - lo)/side; for the unsmoothed transform the
    interpolated eCDFs of z."""
    if isinstance(T, BoxTransform):
        return (bx - T.lo[0]) / T.side, (by - T.lo[1]) / T.side
    if isinstance(T, LinearTransform):
        zx = (bx - T.mu[0]) / T.sigma
        zy = (by - T.mu[1]) / T.sigma
        return linear_ecdf(zx, T.knots[0]), linear_ecdf(zy, T.knots[1])
    zx = (bx - T.mu[0]) / T.sigma
    zy = (by - T.mu[1]) / T.sigma
    return (hermite_cdf(zx, T.knots[0], T.values, T.slopes[0]),
            hermite_cdf(zy, T.knots[1], T.values, T.slopes[1]))


# ---------------------------------------------------------------------------
# the GP source (Sec. 2.1, Eq. 1-4)
# ---------------------------------------------------------------------------
def wavenumbers(n_src: int, pitch: float):
    """k = 2 pi |(fx, fy)| / pitch with f = fftfreq(n_src) per axis (cycles per pixel)."""
    f = torch.fft.fftfreq(n_src, dtype=DT)
    fy, fx = torch.meshgrid(f, f, indexing="ij")
    return 2.0 * math.pi * torch.sqrt(fx * fx + fy * fy) / pitch


def power_spectrum(family: int, ps, k):
    """P(k) of the chosen family; ps holds the family's parameters."""
    if family == PS_POWER_LAW:
        A, beta = ps[0], ps[1]
        zero = k == 0
        ks = torch.where(zero, torch.ones_like(k), k)
        return torch.where(zero, torch.zeros_like(k), A * torch.pow(ks, -beta))
    if family == PS_MATERN_LIKE:
        A, k0 = ps[0], ps[1]
        return A / (1.0 + (k / k0) ** 2) ** 2
    if family == PS_MATERN:  # Eq. 4
        sig, n, zeta = ps[0], ps[1], ps[2]
        a = 2.0 * n / (zeta * zeta)
        return sig * sig * 4.0 * math.pi * n * torch.pow(a, n) * torch.pow(a + k * k, -(n + 1.0))
    raise ValueError(family)


def gp_field(w, sqrtP):
    """Eq. 1: f = F^-1(sqrt(P) . F(w)), unnormalised forward FFT, 1/N^2 inverse."""
    return torch.fft.ifft2(sqrtP * torch.fft.fft2(w)).real


def softplus(x):
    """Eq. 2, phi_sp(x) = log(1 + exp(x)), in the overflow-free form max(x,0) + log1p(exp(-|x|))."""
    return torch.clamp_min(x, 0.0) + torch.log1p(torch.exp(-x.abs()))


def source_brightness(f, alpha_src):
    """Eq. 3: s = (phi_sp(f/s0) s0)^alpha_src."""
    return torch.pow(softplus(f / S0) * S0, alpha_src)


def bilinear(grid, yx, yy):
    """Bilinear interpolation of a vertex-centred grid on [0,1]^2 (node (i, j) at
    (i/(N-1), j/(N-1)), grid[j][i]); zero outside the unit square (Sec. 2.1)."""
    n = grid.shape[0]
    inside = (yx >= 0) & (yx <= 1) & (yy >= 0) & (yy <= 1)
    gx = yx.clamp(0.0, 1.0) * (n - 1)
    gy = yy.clamp(0.0, 1.0) * (n - 1)
    i0 = torch.floor(gx.detach()).long().clamp(0, n - 2)
    j0 = torch.floor(gy.detach()).long().clamp(0, n - 2)
    fx = gx - i0.to(DT)
    fy = gy - j0.to(DT)
    v = ((1 - fx) * (1 - fy) * grid[j0, i0] + fx * (1 - fy) * grid[j0, i0 + 1]
         + (1 - fx) * fy * grid[j0 + 1, i0] + fx * fy * grid[j0 + 1, i0 + 1])
    return torch.where(inside, v, torch.zeros_like(v))


# ---------------------------------------------------------------------------
# image formation and likelihood (Sec. 3.1, Sec. 4)
# ---------------------------------------------------------------------------
def psf_convolve(img, psf):
    """'same' 2-D convolution with zero padding: m[j,i] = sum_{b,a} psf[b,a] img[j-(b-c), i-(a-c)]."""
    n = img.shape[0]
    K = psf.shape[0]
    c = (K - 1) // 2
    pad = torch.zeros((n + 2 * c, n + 2 * c), dtype=DT)
    pad = pad.index_put((torch.arange(c, c + n)[:, None], torch.arange(c, c + n)[None, :]), img)
    out = torch.zeros((n, n), dtype=DT)
    for b in range(K):
        for a in range(K):
            # img[j - (b - c)] = pad[j - b + 2c]
            out = out + psf[b, a] * pad[2 * c - b: 2 * c - b + n, 2 * c - a: 2 * c - a + n]
    return out


def log_likelihood(model, data, sigma, mask):
    """Gaussian noise over all pixels (Sec. 2.2: light outside the mask is kept):
    log L = -1/2 sum ((d-m)/sigma)^2 - N log(sigma sqrt(2 pi)); chi^2_img in the mask."""
    r = (data - model) / sigma
    r2 = r * r
    n = data.numel()
    logL = -0.5 * r2.sum() - n * math.log(sigma * math.sqrt(2.0 * math.pi))
    nm = int(mask.sum())
    chi2 = (r2 * mask.to(DT)).sum() / max(nm, 1)
    return logL, chi2


@dataclass
class System:
    """One lens system: observation (Sec. 3.1) plus the model's fixed choices."""
    data: torch.Tensor          # [n_img, n_img] float64
    mask: torch.Tensor          # [n_img, n_img] bool (arc mask)
    psf: torch.Tensor           # [K, K]
    sigma: float                # Gaussian noise rms
    pix: float                  # arcsec per pixel
    s_super: int
    n_src: int
    src_pitch: float            # source-grid pitch for k (arcsec)
    profile: int = PROFILE_SIE
    ps_family: int = PS_POWER_LAW
    sub_kind: int = SUB_NONE
    n_nodes: int = 22
    degree: int = 21
    transform: int = TRANSFORM_RTU
    weights: torch.Tensor | None = None   # [n_img, n_img] positive integer ray weights

    @property
    def n_img(self):
        return self.data.shape[0]


def build_grid(sys: System, lens, subs=None):
    """rtu_build_grid: trace the masked pixel centres and fit the transform."""
    xc, yc = pixel_centres(sys.n_img, sys.pix)
    sel = sys.mask.reshape(-1)
    bx, by = trace(xc[sel], yc[sel], lens, sys.profile, subs, sys.sub_kind)
    if sys.transform == TRANSFORM_UNIFORM:
        return uniform_box(bx, by)
    if sys.transform == TRANSFORM_LINEAR:
        if sys.weights is not None:
            raise ValueError("the unsmoothed eCDF transform takes unweighted rays")
        if bx.shape[0] < 2:
            raise ValueError("the unsmoothed eCDF transform needs at least two masked pixels")
        return linear_ecdf_transform(bx, by)
    w = None if sys.weights is None else sys.weights.reshape(-1)[sel]
    return fit_transform(bx, by, sys.n_nodes, sys.degree, weights=w)


def gp_source(sys: System, latents, ps):
    """Source grid s*(y) on the RTU grid; ps = [family params..., alpha_src]."""
    k = wavenumbers(sys.n_src, sys.src_pitch)
    npar = N_PS_PARAMS[sys.ps_family]
    P = power_spectrum(sys.ps_family, ps[:npar], k)
    f = gp_field(latents, torch.sqrt(P))
    return source_brightness(f, ps[npar]), f


def ray_hist(sys: System, lens, subs=None, T=None):
    """Integer count of supersampled rays per RTU cell (cells (N-1)^2, row-major);
    rays outside the unit square are not counted."""
    if T is None:
        T = build_grid(sys, lens, subs)
    x, y = subray_positions(sys.n_img, sys.pix, sys.s_super)
    bx, by = trace(x.reshape(-1), y.reshape(-1), lens, sys.profile, subs, sys.sub_kind)
    yx, yy = rtu_map(bx, by, T)
    n = sys.n_src
    inside = (yx >= 0) & (yx <= 1) & (yy >= 0) & (yy <= 1)
    i0 = torch.floor(yx.clamp(0, 1) * (n - 1)).long().clamp(0, n - 2)
    j0 = torch.floor(yy.clamp(0, 1) * (n - 1)).long().clamp(0, n - 2)
    cell = (j0 * (n - 1) + i0)[inside]
    return torch.bincount(cell, minlength=(n - 1) * (n - 1)).to(torch.int64)


def mge_light(x, y, light):
    """Multi-Gaussian lens light (App. A.3): sum over components n of
    A_n/(2 pi) exp(-rho_n^2 / (2 sigma_n^2)), rho_n^2 = q_n x'^2 + y'^2/q_n, where
    (x', y') is the position relative to the component's centre (x_n, y_n) in the frame
    rotated by its position angle phi_n (from +x, counter-clockwise; x' is the major axis
    for q_n < 1, as for the lens profile).  light: [n, 6] rows (A, sigma, q, phi, x_n, y_n)."""
    out = torch.zeros_like(x)
    for n in range(light.shape[0]):
        A, sg, q, phi, xn, yn = light[n]
        dx, dy = x - xn, y - yn
        c, s = torch.cos(phi), torch.sin(phi)
        xp = c * dx + s * dy
        yp = -s * dx + c * dy
        rho2 = q * xp * xp + yp * yp / q
        out = out + A / (2.0 * math.pi) * torch.exp(-0.5 * rho2 / (sg * sg))
    return out


def forward(sys: System, lens, latents, ps, subs=None, light=None):
    """rtu_forward: RTU grid -> GP source -> ray-traced supersampled image (+ the MGE
    lens light at the same sub-ray positions, when given) -> PSF -> log L."""
    T = build_grid(sys, lens, subs)
    src, f = gp_source(sys, latents, ps)
    x, y = subray_positions(sys.n_img, sys.pix, sys.s_super)
    bx, by = trace(x.reshape(-1), y.reshape(-1), lens, sys.profile, subs, sys.sub_kind)
    yx, yy = rtu_map(bx, by, T)
    vals = bilinear(src, yx, yy)
    if light is not None and light.shape[0] > 0:
        vals = vals + mge_light(x.reshape(-1), y.reshape(-1), light)
    vals = vals.reshape(sys.n_img * sys.n_img, sys.s_super ** 2)
    image = vals.mean(dim=1).reshape(sys.n_img, sys.n_img)
    model = psf_convolve(image, sys.psf)
    logL, chi2 = log_likelihood(model, sys.data, sys.sigma, sys.mask)
    return dict(logL=logL, chi2=chi2, model=model, image=image, source=src, field=f, T=T)


def forward_adjoint(sys: System, lens, latents, ps, subs=None, light=None):
    """rtu_adjoint reference: log L and its gradient w.r.t. lens, latents, ps (and
    subhaloes, lens light)."""
    lens = lens.detach().clone().requires_grad_(True)
    latents = latents.detach().clone().requires_grad_(True)
    ps = ps.detach().clone().requires_grad_(True)
    inputs = [lens, latents, ps]
    if subs is not None:
        subs = subs.detach().clone().requires_grad_(True)
        inputs.append(subs)
    if light is not None:
        light = light.detach().clone().requires_grad_(True)
        inputs.append(light)
    out = forward(sys, lens, latents, ps, subs, light)
    grads = torch.autograd.grad(out["logL"], inputs, allow_unused=True)
    grads = [torch.zeros_like(v) if g is None else g for g, v in zip(grads, inputs)]
    res = dict(logL=out["logL"].detach(), chi2=out["chi2"].detach(), model=out["model"].detach(),
               image=out["image"].detach(), g_lens=grads[0], g_latents=grads[1], g_ps=grads[2],
               flags=out["T"].flags)
    if subs is not None:
        res["g_subs"] = grads[3]
    if light is not None:
        res["g_light"] = grads[-1]
    if sys.profile == PROFILE_SIE:
        res["g_lens"][1] = 0.0
    return res


# ---------------------------------------------------------------------------
# Stochastic variational inference (Sec. 4): Normal guide in unconstrained space
# ---------------------------------------------------------------------------
# Counter-based generator for the guide's noise: Philox4x32-10 (Salmon, Moraes,
# Dror & Shaw 2011), written from its published definition, and Box-Muller.
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Ten rounds of the Philox 4x32 bijection of counter `ctr` (4 words) under
    `key` (2 words); the key is bumped by the Weyl constants between rounds."""
    c0, c1, c2, c3 = [int(v) & MASK32 for v in ctr]
    k0, k1 = [int(v) & MASK32 for v in key]
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def guide_noise(seed: int, tag: int, step: int, sample: int, n: int):
    """Standard normals e_0..e_{n-1} of one guide sample.  Element e takes the Philox
    block with counter (e // 2, sample, step, tag) and key (seed lo, seed hi); words
    (0, 1) for even e and (2, 3) for odd e give u1 = (w + 1/2)/2^32, u2 likewise, and
    e = sqrt(-2 ln u1) cos(2 pi u2)."""
    out = torch.empty(n, dtype=DT)
    key = (seed & MASK32, (seed >> 32) & MASK32)
    for e in range(n):
        w = philox4x32_10((e >> 1, sample, step, tag), key)
        a, b = (w[0], w[1]) if e % 2 == 0 else (w[2], w[3])
        u1 = (a + 0.5) / 4294967296.0
        u2 = (b + 0.5) / 4294967296.0
        out[e] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    return out


PRIOR_NORMAL, PRIOR_UNIFORM, PRIOR_TRUNC_NORMAL, PRIOR_LINEAR = 0, 1, 2, 3
SPACE_LINEAR, SPACE_LOG10 = 0, 1


def site_targets(profile: int, sub_kind: int, n_sub: int, family: int):
    """Physical-parameter index of every non-latent site, in order: the lens
    vector [8 + 5 n_sub] (gamma skipped for the SIE, tau of each subhalo held
    fixed), then the power-spectrum vector [n_family + 1] offset by the lens size."""
    nl = 8 + 5 * (n_sub if sub_kind else 0)
    idx = [0] + ([1] if profile == PROFILE_EPL else []) + [2, 3, 4, 5, 6, 7]
    for h in range(n_sub if sub_kind else 0):
        idx += [8 + 5 * h + 0, 8 + 5 * h + 1, 8 + 5 * h + 3, 8 + 5 * h + 4]
    idx += [nl + k for k in range(N_PS_PARAMS[family] + 1)]
    return idx


def _sigmoid(u):
    return 1.0 / (1.0 + torch.exp(-u))


def _log_sigmoid(u):
    return -softplus(-u)


def site_value_and_logdensity(u, prior):
    """Support transform v(u) of one site and log p(v) + log |dv/du| under its prior
    (Table A1 families: G normal, U uniform, truncated normal, T linear)."""
    kind, _space, a, b, c, d = prior
    if kind == PRIOR_NORMAL:
        v = u
        return v, -0.5 * ((v - a) / b) ** 2 - math.log(b) - 0.5 * math.log(2 * math.pi)
    if kind == PRIOR_UNIFORM:
        v = a + (b - a) * _sigmoid(u)
        return v, _log_sigmoid(u) + _log_sigmoid(-u)
    if kind == PRIOR_TRUNC_NORMAL:
        lo, hi = c, d
        v = lo + (hi - lo) * _sigmoid(u)
        Z = 0.5 * (math.erf((hi - a) / (b * math.sqrt(2))) - math.erf((lo - a) / (b * math.sqrt(2))))
        lp = -0.5 * ((v - a) / b) ** 2 - math.log(b) - 0.5 * math.log(2 * math.pi) - math.log(Z)
        return v, lp + math.log(hi - lo) + _log_sigmoid(u) + _log_sigmoid(-u)
    if kind == PRIOR_LINEAR:
        # p(v) proportional to 1 + a (v - lo)/(hi - lo) on [lo, hi]  (parity unpinned reading)
        lo, hi = c, d
        sg = _sigmoid(u)
        v = lo + (hi - lo) * sg
        lp = torch.log(1.0 + a * sg) - math.log((hi - lo) * (1.0 + 0.5 * a))
        return v, lp + math.log(hi - lo) + _log_sigmoid(u) + _log_sigmoid(-u)
    raise ValueError(kind)


@dataclass
class GuideState:
    """Mean-field Normal guide: location and softplus-parametrised scale per site,
    for the n_sites physical sites and the n_src^2 latents, plus Adam moments."""
    loc: torch.Tensor
    rho: torch.Tensor
    m: torch.Tensor
    v: torch.Tensor
    t: int = 0


def elbo_estimate(sys: System, state: GuideState, priors, fixed_phys, n_samples: int, seed: int, tag: int,
                  step: int, subs_kind_n=(SUB_NONE, 0)):
    """Monte-Carlo ELBO of the Normal guide (reparametrised samples; Sec. 4):
    ELBO = (1/S) sum_s [log L(theta_s) + sum_sites (log p + log|J|)
                        + sum_latents log N(w; 0, 1) - log q(u_s)],
    u_s = loc + softplus(rho) e_s.  `fixed_phys` is the physical vector
    [lens (8 + 5 n_sub) | ps | lens light (6 n_light, optional)] that supplies the
    values of non-site entries (gamma of an SIE, tau of each subhalo) and the lens
    light, which is held fixed (the paper's Table A1 gives it no prior).  Returns the
    ELBO (with autograd graph)."""
    sub_kind, n_sub = subs_kind_n
    targets = site_targets(sys.profile, sub_kind, n_sub, sys.ps_family)
    ns = len(targets)
    nl = 8 + 5 * (n_sub if sub_kind else 0)
    n_lat = sys.n_src * sys.n_src
    scale = softplus(state.rho)
    total = 0.0
    for s in range(n_samples):
        eps = guide_noise(seed, tag, step, s, ns + n_lat)
        u = state.loc + scale * eps
        phys = [torch.as_tensor(float(x), dtype=DT) for x in fixed_phys]
        lpj = 0.0
        for i, ti in enumerate(targets):
            v, lp = site_value_and_logdensity(u[i], priors[i])
            phys[ti] = torch.pow(10.0, v) if priors[i][1] == SPACE_LOG10 else v
            lpj = lpj + lp
        w = u[ns:].reshape(sys.n_src, sys.n_src)
        lpj = lpj + (-0.5 * w * w - 0.5 * math.log(2 * math.pi)).sum()
        lens = torch.stack(phys[:8])
        subs = torch.stack(phys[8:nl]).reshape(-1, 5) if nl > 8 else None
        nps = N_PS_PARAMS[sys.ps_family] + 1
        ps = torch.stack(phys[nl:nl + nps])
        light = torch.stack(phys[nl + nps:]).reshape(-1, 6) if len(phys) > nl + nps else None
        logL = forward(sys, lens, w, ps, subs, light)["logL"]
        logq = (-0.5 * eps * eps - torch.log(scale) - 0.5 * math.log(2 * math.pi)).sum()
        total = total + logL + lpj - logq
    return total / n_samples


def elbo_step(sys: System, state: GuideState, priors, fixed_phys, n_samples, seed, tag, lr=1e-3,
              b1=0.9, b2=0.999, eps=1e-8, subs_kind_n=(SUB_NONE, 0)):
    """One optimiser step: ELBO and its gradient w.r.t. (loc, rho) at the current
    step's noise, then Adam ascent; returns (elbo, grad_loc, grad_rho, new state)."""
    loc = state.loc.detach().clone().requires_grad_(True)
    rho = state.rho.detach().clone().requires_grad_(True)
    st = GuideState(loc=loc, rho=rho, m=state.m, v=state.v, t=state.t)
    elbo = elbo_estimate(sys, st, priors, fixed_phys, n_samples, seed, tag, state.t, subs_kind_n)
    gl, gr = torch.autograd.grad(elbo, [loc, rho])
    g = torch.cat([gl, gr])
    t = state.t + 1
    m = b1 * state.m + (1 - b1) * g
    v = b2 * state.v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p = torch.cat([state.loc, state.rho]) + lr * mh / (torch.sqrt(vh) + eps)
    n = state.loc.numel()
    new = GuideState(loc=p[:n].detach(), rho=p[n:].detach(), m=m.detach(), v=v.detach(), t=t)
    return float(elbo), gl.detach(), gr.detach(), new
