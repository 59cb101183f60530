"""Pins of the oracle's variational-inference step (Sec. 4): the counter-based
generator against its published known answers, the prior densities against
their normalisation, the Monte-Carlo ELBO gradient against central differences
at fixed noise, and Adam's first step against its closed form."""
import math
import os

import numpy as np
import pytest
import torch
from scipy import integrate

from oracle import rtu_oracle as O
from paper_2606_30620_b300 import inputs as I
from tests import oracle_io

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert O.philox4x32_10(w[:4], w[4:6]) == tuple(w[6:])
        n += 1
    assert n == 3


def test_guide_noise_is_standard_normal():
    e = O.guide_noise(seed=12345, tag=3, step=7, sample=1, n=20000).numpy()
    assert abs(e.mean()) < 0.03 and abs(e.var() - 1.0) < 0.04
    assert abs(np.mean(e ** 4) - 3.0) < 0.25
    # distinct streams for distinct (tag, step, sample) and reproducible
    a = O.guide_noise(1, 2, 3, 0, 64)
    assert torch.equal(a, O.guide_noise(1, 2, 3, 0, 64))
    assert not torch.equal(a, O.guide_noise(1, 2, 3, 1, 64))
    assert not torch.equal(a, O.guide_noise(1, 2, 4, 0, 64))
    assert not torch.equal(a, O.guide_noise(1, 3, 3, 0, 64))


@pytest.mark.parametrize("prior", [(O.PRIOR_NORMAL, 0, 0.3, 0.7, 0, 0), (O.PRIOR_UNIFORM, 0, -10.0, 15.0, 0, 0),
                                   (O.PRIOR_TRUNC_NORMAL, 0, 2.0, 0.2, 1.0, 3.0),
                                   (O.PRIOR_LINEAR, 0, -1.0, 0.0, 0.1, 10.0),
                                   (O.PRIOR_LINEAR, 0, 0.6, 0.0, -2.0, 3.0)])
def test_prior_densities_integrate_to_one_over_the_unconstrained_axis(prior):
    # log p(v(u)) + log|dv/du| is a density in u: it integrates to one
    f = lambda u: math.exp(float(O.site_value_and_logdensity(torch.tensor(u, dtype=torch.float64), prior)[1]))
    val, _ = integrate.quad(f, -60, 60, limit=400, epsabs=1e-12)
    assert abs(val - 1.0) < 1e-8


def test_site_layout():
    assert O.site_targets(O.PROFILE_SIE, O.SUB_NONE, 0, O.PS_POWER_LAW) == [0, 2, 3, 4, 5, 6, 7, 8, 9, 10]
    t = O.site_targets(O.PROFILE_EPL, O.SUB_TNFW, 2, O.PS_MATERN)
    assert t[:8] == list(range(8)) and t[8:16] == [8, 9, 11, 12, 13, 14, 16, 17] and t[16:] == [18, 19, 20, 21]


def _tiny_state(m, sub_kind, n_sub, rng):
    targets = O.site_targets(m.profile, sub_kind, n_sub, m.ps_family)
    phys = list(m.lens) + ([] if m.subs is None else list(m.subs.ravel())) + list(m.ps)
    priors = I.default_priors(m.profile, sub_kind, n_sub, m.ps_family)
    loc = []
    for ti, pr in zip(targets, priors):
        v = math.log10(phys[ti]) if pr[1] == O.SPACE_LOG10 else phys[ti]
        loc.append(I.unconstrain(v, pr))
    ns = len(targets)
    loc = torch.tensor(loc + list(m.latents.ravel()), dtype=torch.float64)
    rho = torch.tensor(rng.uniform(-4.0, -2.0, size=loc.numel()), dtype=torch.float64)
    z = torch.zeros(2 * loc.numel(), dtype=torch.float64)
    return O.GuideState(loc=loc, rho=rho, m=z.clone(), v=z.clone(), t=0), priors, phys, ns


def test_elbo_gradient_matches_central_differences_at_fixed_noise():
    m = I.config_tiny(seed=31, n_img=10, n_src=6)
    s = oracle_io.system(m)
    rng = np.random.default_rng(0)
    st, priors, phys, ns = _tiny_state(m, O.SUB_NONE, 0, rng)
    elbo, gl, gr, _ = O.elbo_step(s, st, priors, phys, n_samples=2, seed=99, tag=5)
    f = lambda loc, rho: float(O.elbo_estimate(s, O.GuideState(loc, rho, st.m, st.v, 0), priors, phys, 2, 99, 5, 0))
    assert abs(f(st.loc, st.rho) - elbo) < 1e-9 * abs(elbo)
    for which in range(2):
        v = torch.tensor(rng.standard_normal(st.loc.numel()), dtype=torch.float64)
        h = 1e-7
        if which == 0:
            fd = (f(st.loc + h * v, st.rho) - f(st.loc - h * v, st.rho)) / (2 * h)
            an = float((gl * v).sum())
        else:
            fd = (f(st.loc, st.rho + h * v) - f(st.loc, st.rho - h * v)) / (2 * h)
            an = float((gr * v).sum())
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (which, fd, an)


def test_adam_first_step_closed_form():
    m = I.config_tiny(seed=32, n_img=10, n_src=6)
    s = oracle_io.system(m)
    st, priors, phys, ns = _tiny_state(m, O.SUB_NONE, 0, np.random.default_rng(1))
    lr = 1e-3
    _, gl, gr, new = O.elbo_step(s, st, priors, phys, 1, 7, 2, lr=lr)
    g = torch.cat([gl, gr])
    # step 1: m_hat = g, v_hat = g^2 -> delta = lr g / (|g| + eps)
    delta = torch.cat([new.loc - st.loc, new.rho - st.rho])
    assert torch.allclose(delta, lr * g / (g.abs() + 1e-8), rtol=1e-10, atol=1e-15)
    assert new.t == 1
