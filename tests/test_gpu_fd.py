"""Central finite differences (h = 1e-4, FP64 path) of the GPU's own forward model
and ELBO against its hand-written adjoint, on the differentiation workload (16 seeded
mocks of 256^2 pixels, 3x3 rays, SIE + shear, 128^2 latents, power-law spectrum).

Smooth coordinates only.  log L is smooth in the latents and the spectrum parameters
(the rays do not move), so a central difference agrees to O(h^2).  In the lens
parameters log L is only piecewise smooth: every swap of two centre rays' ranks moves
the order statistics' slopes and every ray crossing a bilinear cell edge moves the
interpolation's slope, and on these mocks such kinks lie far closer together than h
(the oracle's own central differences along random lens directions miss its gradient
by 5% even at h = 1e-6, by several times the gradient at h = 1e-4).  The lens
coordinates are therefore excluded here; their gradient is checked against the
oracle's (test_gpu_parity, test_gpu_elbo).  The ELBO's gradient w.r.t. the guide
locations and scales of the latents and the spectrum sites is checked against central
differences of the ELBO itself (same Philox noise at the same step), by exporting the
guide state, shifting it and importing it again.  Tolerance: 1e-5 of the directional
derivative plus the central difference's own rounding, 1e-14 |f| / h (the relative
rounding of an FP64 sum of ~1e6 terms, over 2h)."""
import numpy as np
import pytest
import torch

from paper_2606_30620_b300 import inputs as I
from tests.test_gpu_elbo import guide_start

pytestmark = pytest.mark.gpu

H = 1e-4
TOL = 1e-5
MOCKS = 16
# FP64 evaluation of log L or the ELBO (sums over ~1e5-1e6 terms) carries a relative
# error of order 1e-14; divided by 2h that bounds the central difference's rounding.
# A direction is checked at |fd - an| <= TOL |an| + EVAL_REL |f| / h.
EVAL_REL = 1e-14


@pytest.fixture(scope="module")
def rtu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu as mod
    return mod


def _ok(fd, an, f):
    return abs(fd - an) <= TOL * abs(an) + EVAL_REL * abs(f) / H


def test_log_likelihood_central_differences(rtu):
    rng = np.random.default_rng(31)
    worst = 0.0
    for k in range(MOCKS):
        m = I.config_c3(2000 + k)
        s = rtu.System.from_mock(m, precision=rtu.RTU_F64)
        b = rtu.Binding(s, m.lens, m.latents, m.ps)
        batch = rtu.Batch([b])
        batch.forward()
        batch.adjoint()
        torch.cuda.synchronize()
        g_lat = b.g_latents.cpu().numpy().ravel().copy()
        g_ps = b.g_ps.cpu().numpy().copy()
        lat0, ps0 = b.latents.clone(), b.ps.clone()

        def logL():
            batch.forward()
            torch.cuda.synchronize()
            return float(b.stats[rtu.STAT_LOGL])

        dirs = []
        for _ in range(2):                                  # random latent directions
            v = rng.standard_normal(g_lat.size)
            dirs.append(("lat", v / np.linalg.norm(v)))
        for j in range(g_ps.size):                          # each spectrum parameter and alpha_src
            dirs.append(("ps", np.eye(g_ps.size)[j]))
        for kind, v in dirs:
            vt = torch.tensor(v, dtype=torch.float64, device="cuda")
            vals = []
            for sgn in (1.0, -1.0):
                if kind == "lat":
                    b.latents.copy_(lat0 + sgn * H * vt.view_as(lat0))
                else:
                    b.ps.copy_(ps0 + sgn * H * vt)
                vals.append(logL())
            b.latents.copy_(lat0)
            b.ps.copy_(ps0)
            fd = (vals[0] - vals[1]) / (2 * H)
            an = float(np.dot(g_lat if kind == "lat" else g_ps, v))
            worst = max(worst, abs(fd - an) / abs(an))
            assert _ok(fd, an, vals[0]), (m.name, kind, fd, an)
        s.close()
    print("worst relative error", worst)


def test_elbo_central_differences(rtu):
    rng = np.random.default_rng(32)
    S, seed, lr = 8, 77, 1e-3
    for k in range(MOCKS):
        m = I.config_c3(2000 + k)
        pr, ph, loc, rho = guide_start(m, np.random.default_rng(5))
        s = rtu.System.from_mock(m, precision=rtu.RTU_F64, n_slots=S)
        s.elbo_init(pr, ph, loc, rho, 100 + k)
        blob0 = bytearray(s.elbo_export())
        out = torch.zeros(1, dtype=torch.float64, device="cuda")

        def elbo(blob):
            s.elbo_import(bytes(blob))
            rtu.rtu_elbo_step([s], S, seed, lr, out)
            torch.cuda.synchronize()
            return float(out[0])

        e0 = elbo(blob0)
        gl, gr = s.elbo_grad()
        ns, n = s.n_sites, loc.size
        ps_sites = np.arange(ns - 3, ns)                    # the two spectrum sites and alpha_src
        dirs = []
        v = np.zeros(n); v[ns:] = rng.standard_normal(n - ns); dirs.append(("loc latents", v / np.linalg.norm(v), 0))
        for j in ps_sites:
            v = np.zeros(n); v[j] = 1.0; dirs.append((f"loc site {j}", v, 0))
        # the scales: along the gradient's latent and spectrum parts (a random latent
        # direction has a gradient too small to rise above the evaluation's rounding)
        v = np.zeros(n); v[ns:] = gr[ns:]; dirs.append(("rho latents", v / np.linalg.norm(v), 1))
        v = np.zeros(n); v[ps_sites] = gr[ps_sites]; dirs.append(("rho sites", v / np.linalg.norm(v), 1))
        for name, v, which in dirs:
            vals = []
            for sgn in (1.0, -1.0):
                blob = bytearray(blob0)
                f = np.frombuffer(blob, dtype=np.float64, count=2 * n)
                f[which * n:(which + 1) * n] += sgn * H * v
                vals.append(elbo(blob))
            fd = (vals[0] - vals[1]) / (2 * H)
            an = float(np.dot(gl if which == 0 else gr, v))
            assert _ok(fd, an, e0), (m.name, name, fd, an)
        s.close()
