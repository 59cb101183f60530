"""rtu_elbo_step (S10) against the oracle's SVI step: same guide, same Philox
noise, same priors -> the same ELBO and the same Adam-updated guide.
FP64 mode: 1e-10; FP32 mode: 1e-5 (relative L2 of loc and rho updates)."""
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


def test_elbo_step_fp32_c3_shape(rtu):
    # 128^2 latents, power-law spectrum (amplitude and slope), SIE + shear, 8 samples
    m = I.config_c3(2001, n_img=128, s=3, n_src=128)
    res, _ = run_both(rtu, m, rtu.RTU_F32, n_samples=8, steps=1, lr=1e-3)
    e_g, e_o, lg, rg, lo, ro, t, to = res[0]
    assert abs(e_g - e_o) < 1e-5 * abs(e_o)
    loc0 = guide_start(m, np.random.default_rng(5))[2]
    # compare the Adam steps themselves (the update is lr-sized, the state O(1))
    assert G.rel_l2(lg - loc0, lo - loc0) < 1e-3


def test_checkpoint_resume_continues_the_same_run(rtu):
    # the per-cell source-gradient sums run over counting-sorted records whose order
    # inside a cell depends on integer-atomic timing, so two runs agree to rounding of
    # those FP64 sums, not always to the last bit
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
    assert G.rel_l2(lb, la) < 1e-12 and G.rel_l2(rb, ra) < 1e-12


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
        assert G.rel_l2(lb, la) < 1e-12 and G.rel_l2(rb, ra) < 1e-12
