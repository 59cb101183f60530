"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here retypes an oracle formula: each check compares an oracle step
with an independent route to the same number (a closed form, a quadrature
of the paper's convergence, a brute-force sum, a library routine the oracle
does not call, or a derivative by central differences).
"""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, signal

from oracle import rtu_oracle as O
from paper_2606_30620_b300 import inputs as I
from tests import oracle_io

DT = torch.float64


def t(v):
    return torch.tensor(v, dtype=DT)


# ---------------------------------------------------------------- deflections
def _pts(n=40, seed=3, scale=2.0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-scale, scale, size=(n, 2))
    return t(p[:, 0]), t(p[:, 1])


def test_sis_deflection_has_magnitude_theta_E():
    # q = 1, gamma = 2: |alpha| = theta_E everywhere (singular isothermal sphere)
    x, y = _pts()
    ax, ay = O.deflection_epl(x, y, t(1.3), t(2.0), t(0.0), t(0.0), t(0.0), t(0.0))
    assert torch.allclose(torch.hypot(ax, ay), torch.full_like(x, 1.3), rtol=0, atol=1e-13)
    # and it points radially
    assert torch.allclose(ax * y - ay * x, torch.zeros_like(x), atol=1e-13)


@pytest.mark.parametrize("gamma", [1.6, 1.9, 2.2, 2.5])
def test_round_power_law_closed_form(gamma):
    # q = 1: alpha(r) = (2/r) int_0^r kappa r' dr' = theta_E^(gamma-1) r^(2-gamma)
    x, y = _pts(seed=5)
    thE = 1.1
    ax, ay = O.deflection_epl(x, y, t(thE), t(gamma), t(0.0), t(0.0), t(0.0), t(0.0))
    r = torch.hypot(x, y)
    ref = thE ** (gamma - 1.0) * r ** (2.0 - gamma)
    assert torch.allclose(torch.hypot(ax, ay), ref, rtol=1e-13)


def _keeton_alpha(xr, yr, kappa_of_xi, q):
    """Deflection of a homoeoidal kappa(xi), xi^2 = x^2 + y^2/q^2, by the 1-D
    integrals J_n = int_0^1 kappa(xi(u)) / (1-(1-q^2)u)^(n+1/2) du:
    alpha_x = q x J_0, alpha_y = q y J_1 (Schramm 1990; Keeton 2001)."""
    def xi(u):
        return math.sqrt(u * (xr * xr + yr * yr / (1.0 - (1.0 - q * q) * u)))

    def J(n):
        # u = v^2 removes the integrable u -> 0 singularity
        f = lambda v: 2 * v * kappa_of_xi(xi(v * v)) / (1.0 - (1.0 - q * q) * v * v) ** (n + 0.5)
        val, _ = integrate.quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=400)
        return val
    return q * xr * J(0), q * yr * J(1)


@pytest.mark.parametrize("gamma,q,phi", [(2.0, 0.8, 0.5236), (1.85, 0.65, 1.1), (2.15, 0.9, 2.6),
                                         (2.0, 0.5, 0.0)])
def test_epl_series_matches_quadrature_of_eq_A1(gamma, q, phi):
    thE, x0, y0 = 1.2, 0.07, -0.04
    e1, e2 = I.ellipticity(q, phi)
    x, y = _pts(n=12, seed=11)
    ax, ay = O.deflection_epl(x, y, t(thE), t(gamma), t(e1), t(e2), t(x0), t(y0))
    for k in range(x.shape[0]):
        dx, dy = float(x[k]) - x0, float(y[k]) - y0
        xr = math.cos(phi) * dx + math.sin(phi) * dy
        yr = -math.sin(phi) * dx + math.cos(phi) * dy
        # Eq. A1 with rho^2 = q x^2 + y^2/q = q xi^2
        kap = lambda xi: (3.0 - gamma) / 2.0 * (thE / (math.sqrt(q) * xi)) ** (gamma - 1.0)
        axr, ayr = _keeton_alpha(xr, yr, kap, q)
        rx = math.cos(phi) * axr - math.sin(phi) * ayr
        ry = math.sin(phi) * axr + math.cos(phi) * ayr
        assert abs(float(ax[k]) - rx) < 1e-9 and abs(float(ay[k]) - ry) < 1e-9


def _fd_jacobian(fn, x, y, h=1e-5):
    axp, ayp = fn(x + h, y)
    axm, aym = fn(x - h, y)
    bxp, byp = fn(x, y + h)
    bxm, bym = fn(x, y - h)
    return ((axp - axm) / (2 * h), (bxp - bxm) / (2 * h), (ayp - aym) / (2 * h), (byp - bym) / (2 * h))


def test_epl_divergence_is_twice_kappa_and_curl_free():
    thE, gamma, q, phi, x0, y0 = 1.3, 2.1, 0.7, 0.4, 0.05, 0.02
    e1, e2 = I.ellipticity(q, phi)
    fn = lambda X, Y: O.deflection_epl(X, Y, t(thE), t(gamma), t(e1), t(e2), t(x0), t(y0))
    x, y = _pts(n=30, seed=2, scale=2.5)
    dxx, dxy, dyx, dyy = _fd_jacobian(fn, x, y)
    dx, dy = x - x0, y - y0
    xr = math.cos(phi) * dx + math.sin(phi) * dy
    yr = -math.sin(phi) * dx + math.cos(phi) * dy
    rho = torch.sqrt(q * xr * xr + yr * yr / q)
    kappa = (3.0 - gamma) / 2.0 * (thE / rho) ** (gamma - 1.0)
    assert torch.allclose(dxx + dyy, 2 * kappa, rtol=2e-7, atol=1e-8)
    assert torch.allclose(dxy, dyx, atol=1e-7)


def test_shear_is_gradient_of_its_potential():
    g1, g2 = 0.03, -0.045
    psi = lambda X, Y: 0.5 * g1 * (X * X - Y * Y) + g2 * X * Y
    x, y = _pts(seed=9)
    ax, ay = O.deflection_shear(x, y, t(g1), t(g2))
    h = 1e-5
    assert torch.allclose(ax, (psi(x + h, y) - psi(x - h, y)) / (2 * h), atol=1e-10)
    assert torch.allclose(ay, (psi(x, y + h) - psi(x, y - h)) / (2 * h), atol=1e-10)


def _project(rho3d, R):
    """Sigma(R) = 2 int_0^inf rho(sqrt(R^2+z^2)) dz."""
    f = lambda z: rho3d(math.sqrt(R * R + z * z))
    a, _ = integrate.quad(f, 0.0, 50.0 * max(R, 1e-3), epsabs=1e-13, epsrel=1e-12, limit=400)
    b, _ = integrate.quad(f, 50.0 * max(R, 1e-3), np.inf, epsabs=1e-13, epsrel=1e-12, limit=400)
    return 2.0 * (a + b)


@pytest.mark.parametrize("xval", [0.05, 0.4, 0.999, 1.0, 1.004, 2.5, 9.0])
def test_nfw_convergence_is_projected_eq_A2(xval):
    ks, rs = 0.7, 0.3
    rho = lambda r: (ks / rs) / ((r / rs) * (1.0 + r / rs) ** 2)   # rho_s r_s = kappa_s (Sigma_cr = 1)
    ref = _project(rho, xval * rs)
    got = float(O.nfw_convergence(t([xval * rs]), t(ks), t(rs))[0])
    assert abs(got - ref) < 1e-8 * max(1.0, abs(ref))
    if xval == 1.0:
        assert abs(got - 2.0 * ks / 3.0) < 1e-14


@pytest.mark.parametrize("r", [0.02, 0.3, 0.2995, 0.7, 2.0])
def test_nfw_deflection_is_enclosed_convergence(r):
    ks, rs = 0.7, 0.3
    enc, _ = integrate.quad(lambda s: float(O.nfw_convergence(t([s]), t(ks), t(rs))[0]) * s, 0.0, r,
                            epsabs=1e-14, epsrel=1e-12, limit=400, points=[rs] if rs < r else None)
    ref = 2.0 * enc / r
    ax, ay = O.deflection_nfw(t([r]), t([0.0]), t(ks), t(rs), t(1.0), t(0.0), t(0.0), O.SUB_NFW)
    assert abs(float(ax[0]) - ref) < 1e-9 and abs(float(ay[0])) < 1e-15


@pytest.mark.parametrize("r,tau", [(0.05, 4.0), (0.3, 10.0), (0.9, 3.0), (2.5, 10.0)])
def test_tnfw_deflection_is_projected_truncated_density(r, tau):
    ks, rs = 0.5, 0.25
    rho = lambda R3: (ks / rs) / ((R3 / rs) * (1.0 + R3 / rs) ** 2) * tau * tau / (tau * tau + (R3 / rs) ** 2)
    enc, _ = integrate.quad(lambda s: _project(rho, s) * s, 0.0, r, epsabs=1e-12, epsrel=1e-10, limit=200)
    ref = 2.0 * enc / r
    ax, _ = O.deflection_nfw(t([r]), t([0.0]), t(ks), t(rs), t(tau), t(0.0), t(0.0), O.SUB_TNFW)
    assert abs(float(ax[0]) - ref) < 1e-7 * max(abs(ref), 1e-3)


def test_tnfw_tends_to_nfw_for_large_tau():
    r = t([0.1, 0.5, 1.3])
    z = torch.zeros_like(r)
    a_n, _ = O.deflection_nfw(r, z, t(0.6), t(0.4), t(1.0), t(0.0), t(0.0), O.SUB_NFW)
    a_t, _ = O.deflection_nfw(r, z, t(0.6), t(0.4), t(1e5), t(0.0), t(0.0), O.SUB_TNFW)
    assert torch.allclose(a_n, a_t, rtol=1e-4)


# ---------------------------------------------------------- the RTU transform
def test_subrays_tile_each_pixel():
    x, y = O.subray_positions(5, 0.1, 3)
    xc, yc = O.pixel_centres(5, 0.1)
    assert torch.allclose(x.mean(1), xc) and torch.allclose(y.mean(1), yc)
    d = torch.diff(x[0, :3])
    assert torch.allclose(d, torch.full_like(d, 0.1 / 3))


def test_quantile_matches_numpy_linear_method():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(101)
    u = np.linspace(0, 1, 37)
    got = O.quantile_type7(torch.sort(t(v))[0], t(u)).numpy()
    assert np.allclose(got, np.quantile(v, u, method="linear"), atol=1e-15)


def test_standardise_is_affine_invariant():
    rng = np.random.default_rng(1)
    bx, by = t(rng.standard_normal(500)), t(2.0 * rng.standard_normal(500))
    mu, s = O.standardise(bx, by)
    mu2, s2 = O.standardise(3.0 * bx + 1.0, 3.0 * by - 2.0)
    assert torch.allclose((bx - mu[0]) / s, (3 * bx + 1 - mu2[0]) / s2)
    # the smaller std is taken: here x (std ~1) over y (std ~2)
    assert abs(float(s) - float(bx.std(unbiased=False))) < 1e-14


def test_chebyshev_interpolation_equals_dct_sums():
    # M = D + 1 nodes: c_k = (2/M) sum_j Q_j T_k(t_j), c_0 halved (discrete orthogonality)
    M, D = 22, 21
    u = O.chebyshev_nodes(M)
    tj = 2 * u - 1
    rng = np.random.default_rng(4)
    zs = torch.sort(t(rng.standard_normal(3000)))[0]
    c, Q = O.fit_qf_polynomial(zs, u, D)
    theta = (2 * torch.arange(1, M + 1, dtype=DT) - 1) * math.pi / (2 * M)
    # t_j = -cos(theta_j) = cos(pi - theta_j)  ->  T_k(t_j) = cos(k (pi - theta_j))
    ref = torch.stack([(2.0 / M) * (Q * torch.cos(k * (math.pi - theta))).sum() for k in range(D + 1)])
    ref[0] /= 2
    assert torch.allclose(c, ref, atol=1e-12)
    assert torch.allclose(tj, -torch.cos(theta), atol=1e-15)


def test_polynomial_quantile_is_reproduced_exactly():
    # a QF that *is* a degree-5 polynomial is returned exactly, with exact p(0), p(1), p'
    M, D = 22, 21
    u = O.chebyshev_nodes(M)
    poly = lambda v: -1.0 + 2.0 * v + 0.3 * v ** 3 - 0.1 * v ** 5
    dpoly = lambda v: 2.0 + 0.9 * v ** 2 - 0.5 * v ** 4
    n = 200001
    zs = poly(torch.linspace(0, 1, n, dtype=DT))     # sorted sample whose type-7 QF is poly at grid u
    c, Q = O.fit_qf_polynomial(zs, u, D)
    X, d, rep = O.hermite_knots(c, u, D)
    uu = torch.cat([t([0.0]), u, t([1.0])])
    assert not rep
    # Q(u) is the linear interpolation of poly on a 1/(n-1) grid: error <= max|p''| h^2 / 8
    assert torch.allclose(X, poly(uu), atol=1e-10)
    assert torch.allclose(1.0 / d, dpoly(uu), atol=1e-6)


def test_hermite_cdf_interpolates_and_reproduces_cubics():
    X = t([-2.0, -1.0, -0.2, 0.5, 1.7, 3.0])
    cub = lambda z: 0.5 + 0.1 * z + 0.02 * z ** 2 + 0.003 * z ** 3
    dcub = lambda z: 0.1 + 0.04 * z + 0.009 * z ** 2
    U, d = cub(X), dcub(X)
    z = torch.linspace(-2.0, 2.999, 301, dtype=DT)
    assert torch.allclose(O.hermite_cdf(z, X, U, d), cub(z), atol=1e-13)
    assert torch.allclose(O.hermite_cdf(X[:-1], X, U, d), U[:-1], atol=1e-15)
    # linear extrapolation with the end slopes
    assert abs(float(O.hermite_cdf(t([4.0]), X, U, d)[0]) - float(U[-1] + d[-1])) < 1e-14


def test_uniform_ray_density_gives_identity_map():
    # Sec. 6.1: uniform marginals make the transform (affine in z) the identity up to
    # scaling; equally spaced rays land on equally spaced y = k/(N-1)
    n = 2001
    rng = np.random.default_rng(6)
    gx = np.linspace(-1.3, 0.9, n)
    gy = np.linspace(0.2, 2.7, n)
    bx, by = t(rng.permutation(gx)), t(rng.permutation(gy))
    T = O.fit_transform(bx, by)
    yx, yy = O.rtu_map(t(gx), t(gy), T)
    k = torch.arange(n, dtype=DT) / (n - 1)
    assert T.flags == 0
    assert torch.allclose(yx, k, atol=1e-12) and torch.allclose(yy, k, atol=1e-12)


def test_cdf_is_monotone_and_hits_node_values_on_a_lensed_mock():
    m = I.config_c1()
    s = oracle_io.system(m)
    lens, _, _, _ = oracle_io.params(m)
    T = O.build_grid(s, lens)
    assert T.flags == 0
    for a in range(2):
        z = torch.linspace(float(T.knots[a, 0]) - 1, float(T.knots[a, -1]) + 1, 20001, dtype=DT)
        C = O.hermite_cdf(z, T.knots[a], T.values, T.slopes[a])
        assert bool((torch.diff(C) > 0).all())
        assert torch.allclose(O.hermite_cdf(T.knots[a, 1:-1], T.knots[a], T.values, T.slopes[a]),
                              T.values[1:-1], atol=1e-14)
        # the smoothed CDF tracks the eCDF of the centre rays (Fig. C1): KS distance small
    xc, yc = O.pixel_centres(s.n_img, s.pix)
    sel = s.mask.reshape(-1)
    bx, by = O.trace(xc[sel], yc[sel], lens, s.profile)
    yx, yy = O.rtu_map(bx, by, T)
    for v in (yx, yy):
        vs = torch.sort(v)[0]
        ecdf = torch.arange(1, vs.numel() + 1, dtype=DT) / vs.numel()
        assert float((vs - ecdf).abs().max()) < 0.02


# ---------------------------------------------------------------- GP source
def test_unit_power_spectrum_reproduces_white_noise():
    rng = np.random.default_rng(2)
    w = t(rng.standard_normal((16, 16)))
    assert torch.allclose(O.gp_field(w, torch.ones(16, 16, dtype=DT)), w, atol=1e-14)
    assert torch.allclose(O.gp_field(w, torch.full((16, 16), 3.0, dtype=DT)), 3.0 * w, atol=1e-13)


def test_gp_filter_against_naive_dft():
    rng = np.random.default_rng(3)
    for n in (4, 6, 8):
        w = rng.standard_normal((n, n))
        sq = rng.uniform(0.1, 2.0, size=(n, n))
        sq = 0.5 * (sq + sq[(-np.arange(n)) % n][:, (-np.arange(n)) % n])   # real-even filter
        ref = np.zeros((n, n))
        for j in range(n):
            for i in range(n):
                acc = 0.0 + 0.0j
                for kj in range(n):
                    for ki in range(n):
                        W = 0.0 + 0.0j
                        for b in range(n):
                            for a in range(n):
                                W += w[b, a] * np.exp(-2j * np.pi * (ki * a + kj * b) / n)
                        acc += sq[kj, ki] * W * np.exp(2j * np.pi * (ki * i + kj * j) / n)
                ref[j, i] = (acc / (n * n)).real
        assert np.allclose(O.gp_field(t(w), t(sq)).numpy(), ref, atol=1e-12)


def test_field_variance_is_mean_power():
    # Var f_x = (1/N^2) sum_k P_k for unit white noise: empirical check over seeds
    n = 16
    k = O.wavenumbers(n, 0.1)
    P = O.power_spectrum(O.PS_MATERN_LIKE, t([2.0, 6.0]), k)
    rng = np.random.default_rng(7)
    acc = torch.zeros(n, n, dtype=DT)
    reps = 3000
    for _ in range(reps):
        f = O.gp_field(t(rng.standard_normal((n, n))), torch.sqrt(P))
        acc += f * f
    assert abs(float(acc.mean()) / reps - float(P.mean())) < 0.03 * float(P.mean())


def test_matern_with_n1_is_the_matern_like_form():
    # Eq. 4 with n = 1: P = 2 pi sigma^2 zeta^2 / (1 + (k/k0)^2)^2 with k0 = sqrt(2)/zeta
    k = O.wavenumbers(12, 0.07)
    sig, zeta = 0.3, 0.9
    a = O.power_spectrum(O.PS_MATERN, t([sig, 1.0, zeta]), k)
    b = O.power_spectrum(O.PS_MATERN_LIKE, t([2 * math.pi * sig ** 2 * zeta ** 2, math.sqrt(2) / zeta]), k)
    assert torch.allclose(a, b, rtol=1e-13)


def test_power_law_zero_mode_and_wavenumbers():
    k = O.wavenumbers(8, 0.5)
    assert float(k[0, 0]) == 0.0
    # fftfreq: index 1 is 1/8 cycles per pixel; index 4 is the Nyquist -1/2
    assert abs(float(k[0, 1]) - 2 * math.pi * (1 / 8) / 0.5) < 1e-14
    assert abs(float(k[4, 0]) - 2 * math.pi * 0.5 / 0.5) < 1e-14
    P = O.power_spectrum(O.PS_POWER_LAW, t([1.0, 3.0]), k)
    assert float(P[0, 0]) == 0.0 and abs(float(P[0, 1]) - float(k[0, 1]) ** -3) < 1e-12


def test_softplus_source_values():
    f = t([-0.2, -0.01, 0.0, 0.004, 0.05, 0.8])
    s = O.source_brightness(f, t(1.7)).numpy()
    ref = [(math.log1p(math.exp(v / 0.01)) * 0.01) ** 1.7 for v in f.tolist()]
    assert np.allclose(s, ref, rtol=1e-13)


# --------------------------------------------------------- image formation
def test_bilinear_exact_on_bilinear_functions_and_zero_outside():
    n = 9
    g = torch.linspace(0, 1, n, dtype=DT)
    Y, X = torch.meshgrid(g, g, indexing="ij")
    fn = lambda x, y: 0.3 + 1.2 * x - 0.7 * y + 2.1 * x * y
    grid = fn(X, Y)
    rng = np.random.default_rng(8)
    yx, yy = t(rng.uniform(0, 1, 500)), t(rng.uniform(0, 1, 500))
    assert torch.allclose(O.bilinear(grid, yx, yy), fn(yx, yy), atol=1e-14)
    out = O.bilinear(grid, t([-1e-9, 0.5, 1.0 + 1e-9, 0.5]), t([0.5, -0.2, 0.5, 1.5]))
    assert bool((out == 0).all())
    assert abs(float(O.bilinear(grid, t([1.0]), t([1.0]))[0]) - float(grid[-1, -1])) < 1e-15


def test_psf_convolution_matches_scipy_same_mode():
    rng = np.random.default_rng(9)
    img = rng.standard_normal((13, 13))
    for K in (1, 3, 5):
        psf = rng.uniform(size=(K, K))
        ref = signal.convolve2d(img, psf, mode="same", boundary="fill")
        assert np.allclose(O.psf_convolve(t(img), t(psf)).numpy(), ref, atol=1e-12)
    delta = np.zeros((5, 5))
    delta[2, 2] = 1.0
    assert np.allclose(O.psf_convolve(t(img), t(delta)).numpy(), img)


def test_likelihood_at_perfect_fit():
    d = t(np.ones((6, 6)))
    mask = torch.zeros(6, 6, dtype=torch.bool)
    mask[1:3, 2:5] = True
    L, chi2 = O.log_likelihood(d, d, 0.1, mask)
    assert abs(float(L) + 36 * math.log(0.1 * math.sqrt(2 * math.pi))) < 1e-12 and float(chi2) == 0.0
    m = d.clone()
    m[1, 2] += 0.2
    L, chi2 = O.log_likelihood(m, d, 0.1, mask)
    assert abs(float(chi2) - 4.0 / 6.0) < 1e-12


# ---------------------------------------------------------------- gradients
@pytest.mark.parametrize("seed,profile,family", [(7, I.PROFILE_EPL, I.PS_MATERN_LIKE),
                                                 (8, I.PROFILE_SIE, I.PS_POWER_LAW),
                                                 (9, I.PROFILE_EPL, I.PS_MATERN)])
def test_gradient_matches_central_differences(seed, profile, family):
    m = I.config_tiny(seed=seed, profile=profile, family=family)
    s = oracle_io.system(m)
    lens, lat, ps, _ = oracle_io.params(m)
    g = O.forward_adjoint(s, lens, lat, ps)
    rng = np.random.default_rng(seed)
    L = lambda a, b, c: float(O.forward(s, a, b, c)["logL"])
    for which in range(3):
        base = [lens, lat, ps]
        v = t(rng.standard_normal(base[which].shape))
        if which == 0 and profile == I.PROFILE_SIE:
            v[1] = 0.0
        # the tiny system is strongly non-linear (few rays per cell, an active
        # monotonicity guard): a small step keeps kinks outside +-h
        h = 1e-7
        p = [b.clone() for b in base]
        mm = [b.clone() for b in base]
        p[which] = p[which] + h * v
        mm[which] = mm[which] - h * v
        fd = (L(*p) - L(*mm)) / (2 * h)
        an = float((g[["g_lens", "g_latents", "g_ps"][which]] * v).sum())
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (which, fd, an)


def test_subhalo_gradient_matches_central_differences():
    m = I.config_tiny(seed=12, sub_kind=I.SUB_TNFW, n_sub=2)
    s = oracle_io.system(m)
    lens, lat, ps, subs = oracle_io.params(m)
    g = O.forward_adjoint(s, lens, lat, ps, subs)
    rng = np.random.default_rng(3)
    v = t(rng.standard_normal(subs.shape))
    h = 1e-7
    fd = (float(O.forward(s, lens, lat, ps, subs + h * v)["logL"])
          - float(O.forward(s, lens, lat, ps, subs - h * v)["logL"])) / (2 * h)
    an = float((g["g_subs"] * v).sum())
    assert abs(fd - an) < 1e-5 * max(1.0, abs(an))


# ------------------------------------------------------- uniform-grid baseline
def test_uniform_box_is_the_smallest_square_around_the_masked_rays():
    # Sec. 2.1: the grid spans the smallest square box containing every masked ray
    m = I.config_c2(1040, n_img=64, s=2, n_src=32)
    s = oracle_io.system(m)
    s.transform = O.TRANSFORM_UNIFORM
    lens, _, _, _ = oracle_io.params(m)
    T = O.build_grid(s, lens)
    xc, yc = O.pixel_centres(s.n_img, s.pix)
    sel = s.mask.reshape(-1)
    bx, by = O.trace(xc[sel], yc[sel], lens, s.profile)
    yx, yy = O.rtu_map(bx, by, T)
    lo = torch.stack([yx.min(), yy.min()])
    hi = torch.stack([yx.max(), yy.max()])
    assert float(lo.min()) >= -1e-12 and float(hi.max()) <= 1 + 1e-12
    wide = int(torch.argmax(hi - lo))
    assert abs(float(lo[wide])) < 1e-12 and abs(float(hi[wide]) - 1) < 1e-12     # tight on the wider axis
    assert abs(float(0.5 * (lo[1 - wide] + hi[1 - wide])) - 0.5) < 1e-12           # centred on the other


def test_uniform_grid_gradient_matches_central_differences():
    m = I.config_tiny(seed=17)
    s = oracle_io.system(m)
    s.transform = O.TRANSFORM_UNIFORM
    lens, lat, ps, _ = oracle_io.params(m)
    g = O.forward_adjoint(s, lens, lat, ps)
    rng = np.random.default_rng(17)
    for which, key in ((0, "g_lens"), (1, "g_latents"), (2, "g_ps")):
        base = [lens, lat, ps]
        v = t(rng.standard_normal(base[which].shape))
        h = 1e-7
        p = [b.clone() for b in base]
        q = [b.clone() for b in base]
        p[which] = p[which] + h * v
        q[which] = q[which] - h * v
        fd = (float(O.forward(s, *p)["logL"]) - float(O.forward(s, *q)["logL"])) / (2 * h)
        an = float((g[key] * v).sum())
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (key, fd, an)


# ------------------------------------------------------- MGE lens light (App. A.3)
def _light_grid(half=6.0, n=801):
    x = torch.linspace(-half, half, n, dtype=torch.float64)
    X, Y = torch.meshgrid(x, x, indexing="xy")
    return X.reshape(-1), Y.reshape(-1), float(x[1] - x[0]) ** 2


def test_mge_component_flux_is_amplitude_times_sigma_squared():
    # A/(2 pi) exp(-rho^2/(2 sigma^2)) with rho^2 = q x'^2 + y'^2/q (unit Jacobian)
    # integrates to A sigma^2 over the plane, for any axis ratio and angle
    X, Y, dA = _light_grid()
    for row in ([2.0, 0.4, 0.6, 0.7, 0.1, -0.2], [0.5, 0.8, 0.95, 2.9, -0.3, 0.2]):
        L = t([row])
        flux = float(O.mge_light(X, Y, L).sum()) * dA
        assert abs(flux - row[0] * row[1] ** 2) < 1e-9


def test_mge_axis_ratio_and_angle_equivalence():
    # (q, phi) and (1/q, phi + pi/2) describe the same ellipse
    X, Y, _ = _light_grid(3.0, 101)
    a = O.mge_light(X, Y, t([[1.3, 0.3, 0.7, 0.4, 0.05, 0.1]]))
    b = O.mge_light(X, Y, t([[1.3, 0.3, 1 / 0.7, 0.4 + math.pi / 2, 0.05, 0.1]]))
    assert float((a - b).abs().max()) < 1e-14


def test_round_mge_component_values():
    L = t([[3.0, 0.5, 1.0, 1.1, 0.2, -0.1]])
    x = t([0.2, 0.2 + 0.5, 0.2])
    y = t([-0.1, -0.1, -0.1 - 1.0])
    v = O.mge_light(x, y, L)
    assert abs(float(v[0]) - 3.0 / (2 * math.pi)) < 1e-15
    assert abs(float(v[1]) - 3.0 / (2 * math.pi) * math.exp(-0.5)) < 1e-15
    assert abs(float(v[2]) - 3.0 / (2 * math.pi) * math.exp(-2.0)) < 1e-15


def test_lens_light_gradient_matches_central_differences():
    m = I.with_light(I.config_tiny(seed=21), n=3, seed=4, amp=0.5)
    s = oracle_io.system(m)
    lens, lat, ps, _ = oracle_io.params(m)
    L = oracle_io.light(m)
    g = O.forward_adjoint(s, lens, lat, ps, light=L)
    rng = np.random.default_rng(5)
    v = t(rng.standard_normal(L.shape))
    h = 1e-6
    fd = (float(O.forward(s, lens, lat, ps, light=L + h * v)["logL"])
          - float(O.forward(s, lens, lat, ps, light=L - h * v)["logL"])) / (2 * h)
    an = float((g["g_light"] * v).sum())
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


# ------------------------------------------------------- weighted RTU grid (Sec. 6.3)
def test_weighted_quantile_is_type7_of_the_expanded_sample():
    rng = np.random.default_rng(8)
    for n in (1, 2, 7, 40):
        v = torch.sort(t(rng.standard_normal(n)))[0]
        w = torch.tensor(rng.integers(1, 6, size=n), dtype=torch.int64)
        u = t(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 30)]))
        brute = O.quantile_type7(torch.repeat_interleave(v, w), u)
        assert float((O.quantile_weighted(v, w, u) - brute).abs().max()) == 0.0


def test_unit_weights_give_the_unweighted_transform():
    m = I.config_c2(1050, n_img=48, s=2, n_src=16)
    s = oracle_io.system(m)
    lens, _, _, _ = oracle_io.params(m)
    T0 = O.build_grid(s, lens)
    s.weights = torch.ones(m.n_img, m.n_img, dtype=torch.int64)
    T1 = O.build_grid(s, lens)
    assert float((T0.knots - T1.knots).abs().max()) == 0.0
    assert float((T0.slopes - T1.slopes).abs().max()) == 0.0


def test_weights_move_the_knots_toward_heavy_rays():
    # weighting by the pixel SNR moves the nodes' quantiles (so the knots) toward the
    # rays of bright pixels
    m = I.with_snr_weights(I.config_c2(1051, n_img=48, s=2, n_src=16))
    s = oracle_io.system(m)
    lens, _, _, _ = oracle_io.params(m)
    Tw = O.build_grid(s, lens)
    s.weights = None
    Tu = O.build_grid(s, lens)
    assert float((Tw.knots - Tu.knots).abs().max()) > 1e-3


def test_weighted_grid_gradient_matches_central_differences():
    m = I.with_snr_weights(I.config_tiny(seed=19), cap=7)
    s = oracle_io.system(m)
    lens, lat, ps, _ = oracle_io.params(m)
    g = O.forward_adjoint(s, lens, lat, ps)
    rng = np.random.default_rng(19)
    v = t(rng.standard_normal(8))
    h = 1e-7
    fd = (float(O.forward(s, lens + h * v, lat, ps)["logL"])
          - float(O.forward(s, lens - h * v, lat, ps)["logL"])) / (2 * h)
    an = float((g["g_lens"] * v).sum())
    assert abs(fd - an) < 1e-5 * max(1.0, abs(an))


# ------------------------------------------- unsmoothed linear eCDF (App. C, first paragraph)
def test_linear_ecdf_is_numpy_interp_inside_and_maps_observations_to_ranks():
    rng = np.random.default_rng(31)
    for n in (2, 3, 17, 400):
        X = np.sort(rng.standard_normal(n))
        z = rng.uniform(X[0], X[-1], 200)
        ref = np.interp(z, X, np.linspace(0.0, 1.0, n))
        got = O.linear_ecdf(t(z), t(X)).numpy()
        assert np.abs(got - ref).max() < 1e-14, n
        # the k-th observation sits at the k-th rank, k/(n-1)
        at = O.linear_ecdf(t(X), t(X)).numpy()
        assert np.abs(at - np.arange(n) / (n - 1)).max() < 1e-15, n


def test_linear_ecdf_inverts_the_type7_quantile_function():
    rng = np.random.default_rng(32)
    X = np.sort(rng.standard_normal(250))
    u = np.concatenate([[0.0, 1.0], rng.uniform(0.0, 1.0, 300)])
    q = np.quantile(X, u, method="linear")
    back = O.linear_ecdf(t(q), t(X)).numpy()
    assert np.abs(back - u).max() < 1e-12


def test_linear_ecdf_extrapolates_with_the_end_segment_slopes():
    X = t([-1.0, -0.5, 0.25, 2.0])
    n = 4
    d = t([0.3, 1.7])
    left = O.linear_ecdf(X[0] - d, X)
    right = O.linear_ecdf(X[-1] + d, X)
    assert float((left - (-d / ((n - 1) * 0.5))).abs().max()) < 1e-15
    assert float((right - (1.0 + d / ((n - 1) * 1.75))).abs().max()) < 1e-15
    # tied end observations: a zero-width end segment gives a constant
    Xt = t([0.0, 0.0, 1.0, 2.0])
    v = O.linear_ecdf(t([-0.5, -3.0]), Xt)
    assert float(v.abs().max()) == 0.0


def _linear_mock_rays(seed):
    m = I.config_c2(seed, n_img=48, s=2, n_src=16)
    s = oracle_io.system(m)
    s.transform = O.TRANSFORM_LINEAR
    lens, _, _, _ = oracle_io.params(m)
    xc, yc = O.pixel_centres(s.n_img, s.pix)
    sel = s.mask.reshape(-1)
    bx, by = O.trace(xc[sel], yc[sel], lens, s.profile)
    return s, lens, bx, by


def test_linear_transform_gives_exactly_uniform_marginals_of_the_centre_rays():
    # App. C: the interpolated eCDF makes the marginals of the observations uniform
    # by construction: the centre rays land on the ranks k/(n-1)
    s, lens, bx, by = _linear_mock_rays(1060)
    T = O.build_grid(s, lens)
    yx, yy = O.rtu_map(bx, by, T)
    n = bx.shape[0]
    ranks = np.arange(n) / (n - 1)
    assert np.abs(np.sort(yx.numpy()) - ranks).max() < 1e-12
    assert np.abs(np.sort(yy.numpy()) - ranks).max() < 1e-12


def test_linear_transform_does_not_depend_on_the_standardisation():
    # the interpolated eCDF commutes with any increasing affine map applied to the
    # observations and the query alike, so step i drops out: it equals numpy's
    # interpolation of the raw source-plane positions
    s, lens, bx, by = _linear_mock_rays(1061)
    T = O.build_grid(s, lens)
    x, y = O.subray_positions(s.n_img, s.pix, s.s_super)
    rx, ry = O.trace(x.reshape(-1), y.reshape(-1), lens, s.profile)
    yx, yy = O.rtu_map(rx, ry, T)
    for got, b, r in ((yx, bx, rx), (yy, by, ry)):
        X = np.sort(b.numpy())
        inside = (r.numpy() >= X[0]) & (r.numpy() <= X[-1])
        ref = np.interp(r.numpy()[inside], X, np.linspace(0.0, 1.0, X.size))
        assert inside.sum() > 100
        assert np.abs(got.numpy()[inside] - ref).max() < 1e-12


def test_linear_grid_gradient_matches_central_differences():
    m = I.config_tiny(seed=23)
    s = oracle_io.system(m)
    s.transform = O.TRANSFORM_LINEAR
    lens, lat, ps, _ = oracle_io.params(m)
    g = O.forward_adjoint(s, lens, lat, ps)
    rng = np.random.default_rng(23)
    for which, key in ((0, "g_lens"), (1, "g_latents"), (2, "g_ps")):
        base = [lens, lat, ps]
        v = t(rng.standard_normal(base[which].shape))
        # the map has a kink at every observation: a small step keeps them outside +-h
        h = 1e-8
        p = [b.clone() for b in base]
        q = [b.clone() for b in base]
        p[which] = p[which] + h * v
        q[which] = q[which] - h * v
        fd = (float(O.forward(s, *p)["logL"]) - float(O.forward(s, *q)["logL"])) / (2 * h)
        an = float((g[key] * v).sum())
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (key, fd, an)


# ------------------------------------------------- monotonicity guard (App. C iv)
def test_hermite_guard_repairs_a_non_monotone_fit():
    # p(t) = T_3(t) = 4 t^3 - 3 t (t = 2u - 1) falls for |t| < 1/2.  With M = 4 nodes the
    # knot points are t = -1, -cos((2j-1) pi/8) (j = 1..4), +1 and p there is
    # -1, -cos(3 pi/8), -cos(9 pi/8), -cos(15 pi/8), -cos(21 pi/8), 1 (T_3(-cos a) =
    # -cos 3a); dp/du = 2 (12 t^2 - 3).  span = p(1) - p(0) = 2, floor = 1e-6 span.
    # Written out by hand: the two interior points with dp/du = 2 (12 t^2 - 3) < 0 get
    # the floor slope, and the knots after the fall are lifted to prev + floor.
    D = 3
    u = O.chebyshev_nodes(4)
    c = t([0.0, 0.0, 0.0, 1.0])
    X, d, rep = O.hermite_knots(c, u, D)
    c1, c3 = math.cos(math.pi / 8), math.cos(3 * math.pi / 8)   # cos(pi/8), cos(3pi/8)
    fl = 2e-6
    raw = [-1.0, -c3, c1, -c1, c3, 1.0]                          # -cos(9pi/8) = c1, ...
    want = [raw[0], raw[1], raw[2], raw[2] + fl, raw[2] + 2 * fl, 1.0]
    tk = [-1.0, -c1, -c3, c3, c1, 1.0]
    dp = [2 * (12 * v * v - 3) for v in tk]
    want_d = [1.0 / max(v, fl) for v in dp]
    assert rep
    assert np.allclose(X.numpy(), want, rtol=0, atol=1e-13)
    assert np.allclose(d.numpy(), want_d, rtol=1e-12)
    assert want_d[2] == want_d[3] == 1.0 / fl


def test_hermite_guard_repairs_a_falling_fit():
    # p(t) = -t: the span p(1) - p(0) = -2 is not positive -> repaired with |span|;
    # every slope gets the floor 2e-6 and every knot after the first is lifted.
    u = O.chebyshev_nodes(4)
    X, d, rep = O.hermite_knots(t([0.0, -1.0, 0.0, 0.0]), u, 3)
    assert rep
    fl = 1e-6 * 2.0
    assert np.allclose(X.numpy(), [1.0 + k * fl for k in range(6)], rtol=0, atol=1e-14)
    assert np.allclose(d.numpy(), np.full(6, 1.0 / fl), rtol=1e-12)


def test_quantile_fit_takes_degree_plus_one_nodes():
    zs = torch.sort(t(np.random.default_rng(1).standard_normal(100)))[0]
    with pytest.raises(ValueError):
        O.fit_qf_polynomial(zs, O.chebyshev_nodes(30), 21)


# ------------------------------------------- rays-per-cell histogram (Fig. 1, S11)
def test_ray_hist_of_a_closed_form_box_grid():
    # A lens of negligible deflection (theta_E = 1e-300) and the uniform box grid:
    # 4 x 4 pixels of 1", 2 x 2 sub-rays at +-0.25" -> sub-ray coordinates
    # -1.75 ... 1.75 in steps of 0.5 on each axis.  Mask rows j = 2, 3: the masked
    # centres span x in [-1.5, 1.5], y in [0.5, 1.5]; box side 3, lower corner
    # (-1.5, -0.5).  So y_x = (x + 1.5)/3 puts 2 sub-ray columns in each of the 3 cells
    # per axis (6 inside), and y_y = (y + 0.5)/3 puts 2, 2, 1 sub-ray rows in cells
    # 0, 1, 2 (5 inside).  Counts are x_count[i] y_count[j], row-major [j][i].
    n = 4
    mask = torch.zeros(n, n, dtype=torch.bool)
    mask[2:, :] = True
    s = O.System(data=torch.zeros(n, n, dtype=DT), mask=mask, psf=torch.ones(1, 1, dtype=DT), sigma=1.0,
                 pix=1.0, s_super=2, n_src=4, src_pitch=1.0, transform=O.TRANSFORM_UNIFORM)
    lens = t([1e-300, 2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    h = O.ray_hist(s, lens)
    assert h.tolist() == [4, 4, 4, 4, 4, 4, 2, 2, 2]


def test_ray_hist_equals_a_per_ray_count():
    # each supersampled ray counted by hand: its RTU position, then the cell (i, j)
    # with i <= y_x (n-1) < i + 1 (the last cell closed at y = 1), rays outside the
    # unit square skipped, cell index j (n-1) + i
    m = I.config_tiny(seed=5, n_img=12, s=2, n_src=7)
    s = oracle_io.system(m)
    lens, _, _, _ = oracle_io.params(m)
    T = O.build_grid(s, lens)
    x, y = O.subray_positions(s.n_img, s.pix, s.s_super)
    bx, by = O.trace(x.reshape(-1), y.reshape(-1), lens, s.profile)
    yx, yy = O.rtu_map(bx, by, T)
    n = s.n_src
    counts = [0] * ((n - 1) * (n - 1))
    inside = 0
    for px, py in zip(yx.tolist(), yy.tolist()):
        if not (0.0 <= px <= 1.0 and 0.0 <= py <= 1.0):
            continue
        inside += 1
        gx, gy = px * (n - 1), py * (n - 1)
        ci = next(i for i in range(n - 1) if i <= gx < i + 1 or (i == n - 2 and gx >= n - 2))
        cj = next(j for j in range(n - 1) if j <= gy < j + 1 or (j == n - 2 and gy >= n - 2))
        counts[cj * (n - 1) + ci] += 1
    h = O.ray_hist(s, lens, T=T)
    assert 0 < inside < len(yx)
    assert h.tolist() == counts


# ------------------------------- the order statistics' integer histograms (App. C ii)
def test_selection_histogram_counts_by_explicit_bin_edges():
    # 8 bins over [min, max]: each value counted in the bin whose edges
    # min + b (max - min)/8 <= v < min + (b + 1)(max - min)/8 contain it (the maximum in
    # the last bin); random values stay far from the edges at this size
    rng = np.random.default_rng(11)
    v = rng.uniform(-3.0, 5.0, 500)
    lo, hi = v.min(), v.max()
    want = [0] * 8
    for x in v:
        b = next((k for k in range(8) if lo + k * (hi - lo) / 8 <= x < lo + (k + 1) * (hi - lo) / 8), 7)
        want[b] += 1
    assert O.selection_histogram(t(v), nbins=8).tolist() == want


def test_selection_histogram_is_a_counting_sort_of_the_sorted_values():
    # the k-th smallest value lies in the bin whose cumulative count first exceeds k;
    # weights count as repeated values; min in bin 0, max in the last bin
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.normal(0.0, 1.0, 3000), [40.0, -25.0]])     # with far outliers
    w = rng.integers(1, 5, v.size)
    h = O.selection_histogram(t(v), torch.tensor(w)).numpy()
    assert h.sum() == w.sum() and h[0] >= 1 and h[-1] >= 1
    order = np.argsort(v, kind="stable")
    cum = np.cumsum(h)
    lo, hi = v.min(), v.max()
    r = 0
    for i in order:
        b = int(np.floor((v[i] - lo) * (65536 / (hi - lo))))
        b = min(max(b, 0), 65535)
        assert (cum[b - 1] if b else 0) <= r < cum[b]
        r += w[i]
    assert O.selection_histogram(t(np.full(5, 2.5))).tolist()[0] == 5
