"""rtu_elbo_step (S10) against the oracle's SVI step: same guide, same Philox
noise, same priors -> the same ELBO, the same ELBO gradient w.r.t. the guide's
location and scale (before the optimiser) and the same Adam-updated guide.
FP64 mode: 1e-10; FP32 mode: 1e-5 (relative, L2 over each gradient block)."""
import math

import numpy as np
import pytest
import torch

from oracle import rtu_oracle as O
from paper_2606_30620_b300 import inputs as I
from tests import gpu_cases as G
from tests import oracle_io

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu as mod
    return mod


def guide_start(m, rng, rho_lo=-5.0, rho_hi=-3.0):
    sub_kind = m.sub_kind
    n_sub = 0 if m.subs is None else m.subs.shape[0]
    targets = O.site_targets(m.profile, sub_kind, n_sub, m.ps_family)
    phys = list(m.lens) + ([] if m.subs is None else list(m.subs.ravel())) + list(m.ps)
    priors = I.default_priors(m.profile, sub_kind, n_sub, m.ps_family, m.subs)
    loc = [I.unconstrain(math.log10(phys[t]) if p[1] == I.SPACE_LOG10 else phys[t], p)
           for t, p in zip(targets, priors)]
    loc = np.array(loc + list(m.latents.ravel()))
    rho = rng.uniform(rho_lo, rho_hi, size=loc.size)
    light = [] if m.light is None else list(m.light.ravel())       # held fixed by the ELBO step
    return priors, np.array(phys + light), loc, rho


def run_both(rtu, m, prec, n_samples, steps, seed=77, tag=9, lr=1e-2):
    rng = np.random.default_rng(5)
    priors, phys, loc, rho = guide_start(m, rng)
    s = rtu.System.from_mock(m, precision=prec, n_slots=n_samples)
    s.elbo_init(priors, phys, loc, rho, tag)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    osys = oracle_io.system(m)
    st = O.GuideState(loc=torch.tensor(loc), rho=torch.tensor(rho), m=torch.zeros(2 * loc.size, dtype=torch.float64),
                      v=torch.zeros(2 * loc.size, dtype=torch.float64), t=0)
    n_sub = 0 if m.subs is None else m.subs.shape[0]
    res = []
    for _ in range(steps):
        rtu.rtu_elbo_step([s], n_samples, seed, lr, out)
        torch.cuda.synchronize()
        e_or, _, _, st = O.elbo_step(osys, st, priors, list(phys), n_samples, seed, tag, lr=lr,
                                     subs_kind_n=(m.sub_kind, n_sub))
        gl, gr, t = s.elbo_state()
        res.append((float(out[0]), e_or, gl, gr, st.loc.numpy(), st.rho.numpy(), t, st.t))
    return res, s


def test_elbo_steps_fp64_tiny(rtu):
    m = I.config_tiny(seed=41, n_img=16, n_src=8)
    res, _ = run_both(rtu, m, rtu.RTU_F64, n_samples=3, steps=3)
    for e_g, e_o, lg, rg, lo, ro, t, to in res:
        assert abs(e_g - e_o) < 1e-10 * abs(e_o)
        assert G.rel_l2(lg, lo) < 1e-10 and G.rel_l2(rg, ro) < 1e-10
        assert t == to


def test_elbo_steps_fp64_subhaloes_and_matern(rtu):
    m = I.config_tiny(seed=42, n_img=16, n_src=8, family=I.PS_MATERN, sub_kind=I.SUB_TNFW, n_sub=2)
    res, _ = run_both(rtu, m, rtu.RTU_F64, n_samples=2, steps=2)
    for e_g, e_o, lg, rg, lo, ro, t, to in res:
        assert abs(e_g - e_o) < 1e-10 * abs(e_o)
        assert G.rel_l2(lg, lo) < 1e-10 and G.rel_l2(rg, ro) < 1e-10


def test_elbo_steps_fp64_with_fixed_lens_light(rtu):
    m = I.with_light(I.config_tiny(seed=44, n_img=16, n_src=8), n=5, seed=6, amp=0.5)
    res, _ = run_both(rtu, m, rtu.RTU_F64, n_samples=2, steps=2)
    for e_g, e_o, lg, rg, lo, ro, t, to in res:
        assert abs(e_g - e_o) < 1e-10 * abs(e_o)
        assert G.rel_l2(lg, lo) < 1e-10 and G.rel_l2(rg, ro) < 1e-10


def _batched_vs_oracle(rtu, mocks, prec, n_samples, seed=77, lr=1e-3):
    """One batched rtu_elbo_step over every mock against the oracle's step of each:
    returns per mock (ELBO gpu, ELBO oracle, grad loc / rho gpu, grad loc / rho oracle,
    n_sites)."""
    rng = np.random.default_rng(5)
    starts = [guide_start(m, rng) for m in mocks]
    systems = []
    for k, (m, (pr, ph, lo, rh)) in enumerate(zip(mocks, starts)):
        s = rtu.System.from_mock(m, precision=prec, n_slots=n_samples)
        s.elbo_init(pr, ph, lo, rh, 100 + k)
        systems.append(s)
    out = torch.zeros(len(mocks), dtype=torch.float64, device="cuda")
    rtu.rtu_elbo_step(systems, n_samples, seed, lr, out)
    torch.cuda.synchronize()
    res = []
    for k, (m, s, (pr, ph, lo, rh)) in enumerate(zip(mocks, systems, starts)):
        key = (m.name, n_samples, seed, 100 + k, lr)
        if key not in _ORACLE_STEPS:       # the same oracle step serves both precisions
            st = O.GuideState(loc=torch.tensor(lo), rho=torch.tensor(rh), m=torch.zeros(2 * lo.size, dtype=torch.float64),
                              v=torch.zeros(2 * lo.size, dtype=torch.float64), t=0)
            n_sub = 0 if m.subs is None else m.subs.shape[0]
            e_or, gl_or, gr_or, _ = O.elbo_step(oracle_io.system(m), st, pr, list(ph), n_samples, seed, 100 + k,
                                                lr=lr, subs_kind_n=(m.sub_kind, n_sub))
            _ORACLE_STEPS[key] = (e_or, gl_or.numpy(), gr_or.numpy())
        e_or, gl_or, gr_or = _ORACLE_STEPS[key]
        gl, gr = s.elbo_grad()
        res.append((float(out[k]), e_or, gl, gr, gl_or, gr_or, s.n_sites))
    return res


_ORACLE_STEPS = {}


def _check_elbo(res, tol, rho_sites=True):
    """The ELBO and its gradient: the whole gradient (loc and rho, sites and latents),
    and each block whose magnitude would otherwise hide it.  rho_sites=False leaves out
    the block d ELBO / d rho of the non-latent sites: it is (1/S) sum_s g_s eps_s
    sigmoid(rho) + ..., a Monte-Carlo sum in which the per-sample lens gradients g_s
    (each held to 1e-5 through the loc block and the parity tests) cancel by a factor
    sum |eps_s| / |sum eps_s| (~50 on the 8-sample workload), beyond float accuracy."""
    for e_g, e_o, gl, gr, glo, gro, ns in res:
        assert abs(e_g - e_o) < tol * abs(e_o), (e_g, e_o)
        whole = G.rel_l2(np.concatenate([gl, gr]), np.concatenate([glo, gro]))
        assert whole < tol, ("whole gradient", whole)
        blocks = [("loc sites", gl[:ns], glo[:ns]), ("loc latents", gl[ns:], glo[ns:]),
                  ("rho latents", gr[ns:], gro[ns:])]
        if rho_sites:
            blocks.append(("rho sites", gr[:ns], gro[:ns]))
        for name, a, b in blocks:
            assert G.rel_l2(a, b) < tol, (name, G.rel_l2(a, b))


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-10)])
def test_elbo_gradient_c3_matches_oracle(rtu, prec, tol):
    # the differentiation workload: 16 seeded mocks, 256^2 pixels, 3x3 rays, SIE + shear,
    # 128^2 latents, power-law spectrum (amplitude, slope), 8 guide samples; the ELBO and
    # its gradient w.r.t. the guide (before Adam) of one batched step against the oracle
    mocks = [I.config_c3(2000 + k) for k in range(16)]
    _check_elbo(_batched_vs_oracle(rtu, mocks, prec, n_samples=8), tol, rho_sites=prec == 1)


@pytest.mark.parametrize("with_subs", [True, False])
def test_elbo_gradient_c4_with_and_without_subhaloes(rtu, with_subs):
    # the substructure workload: 400^2 pixels at 0.03", 3x3 rays, EPL + shear with 1-10
    # truncated NFW subhaloes on the ring (or none), 128^2 grid, FP32 bulk; 2 samples
    mocks = [I.config_c4(3000 + k, with_subs=with_subs) for k in range(2)]
    _check_elbo(_batched_vs_oracle(rtu, mocks, 0, n_samples=2), 1e-5)


def test_checkpoint_resume_continues_the_same_run(rtu):
    # every sum of the step has a fixed order (or is an exact integer sum): the resumed
    # run continues bit for bit
    m = I.config_tiny(seed=43, n_img=16, n_src=8)
    rng = np.random.default_rng(2)
    priors, phys, loc, rho = guide_start(m, rng)
    a = rtu.System.from_mock(m, precision=rtu.RTU_F64, n_slots=2)
    b = rtu.System.from_mock(m, precision=rtu.RTU_F64, n_slots=2)
    a.elbo_init(priors, phys, loc, rho, 3)
    b.elbo_init(priors, phys, loc, rho, 3)
    for _ in range(2):
        rtu.rtu_elbo_step([a], 2, 11, 1e-2)
    blob = a.elbo_export()
    b.elbo_import(blob)
    rtu.rtu_elbo_step([a], 2, 11, 1e-2)
    rtu.rtu_elbo_step([b], 2, 11, 1e-2)
    torch.cuda.synchronize()
    la, ra, ta = a.elbo_state()
    lb, rb, tb = b.elbo_state()
    assert ta == tb == 3
    assert np.array_equal(lb, la) and np.array_equal(rb, ra)


def test_batched_elbo_equals_alone(rtu):
    mocks = [I.config_tiny(seed=50 + k, n_img=12 + 4 * k, n_src=(8, 12, 16)[k % 3]) for k in range(4)]
    rng = np.random.default_rng(9)
    starts = [guide_start(m, rng) for m in mocks]
    alone, batch = [], []
    for m, (pr, ph, lo, rh) in zip(mocks, starts):
        s = rtu.System.from_mock(m, precision=rtu.RTU_F64, n_slots=2)
        s.elbo_init(pr, ph, lo, rh, 1)
        alone.append(s)
        t = rtu.System.from_mock(m, precision=rtu.RTU_F64, n_slots=2)
        t.elbo_init(pr, ph, lo, rh, 1)
        batch.append(t)
    for s in alone:
        rtu.rtu_elbo_step([s], 2, 5, 1e-2)
    out = torch.zeros(len(batch), dtype=torch.float64, device="cuda")
    rtu.rtu_elbo_step(batch, 2, 5, 1e-2, out)
    torch.cuda.synchronize()
    for s, t in zip(alone, batch):
        la, ra, _ = s.elbo_state()
        lb, rb, _ = t.elbo_state()
        assert np.array_equal(lb, la) and np.array_equal(rb, ra)
