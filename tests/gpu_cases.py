"""Run one seeded input through the CUDA path and through the oracle."""
import numpy as np
import torch

from oracle import rtu_oracle as O
from tests import oracle_io


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


F64_TOL = 1e-10
F32_TOL = 1e-5


def check(r, prec):
    """The parity bar on a compare() result: FP64 path 1e-10, FP32 path 1e-5 (relative
    L2) on log L, chi^2, source, image, model and every gradient; the CDF block (FP64 in
    both modes) 1e-10; the integer rays-per-cell histogram and the flags bit-exact."""
    tol = F64_TOL if prec == 1 else F32_TOL
    assert r["cdf"] < F64_TOL, r
    assert r["logL"] < tol and r["chi2"] < tol, r
    for k in ("source", "image", "model"):
        assert r[k] < tol, (k, r)
    if "g_latents" in r:
        assert r["g_latents"] < tol, r
        assert r["g_ps"] < tol, r
        assert r["g_lens"] < tol, r
    if "g_light" in r:
        assert r["g_light"] < tol, r
    assert r["hist_diff"] == 0, r
    assert r["flags"][0] == r["flags"][1], r


def run_gpu(m, precision, want_grads=True, n_slots=1, transform=0):
    from paper_2606_30620_b300 import rtu
    sysm = rtu.System.from_mock(m, precision=precision, n_slots=n_slots, transform=transform)
    lens = m.lens if m.subs is None else np.concatenate([m.lens, m.subs.ravel()])
    b = rtu.Binding(sysm, lens, m.latents, m.ps, want_model=True, want_image=True, want_source=True,
                    want_cdf=True, want_hist=True, grads=want_grads, light=m.light)
    batch = rtu.Batch([b])
    batch.forward()
    if want_grads:
        batch.adjoint()
    torch.cuda.synchronize()
    out = dict(stats=b.stats.cpu().numpy(), model=b.model.cpu().numpy(), image=b.image.cpu().numpy(),
               source=b.source.cpu().numpy(), cdf=b.cdf.cpu().numpy(), hist=b.ray_hist.cpu().numpy())
    if want_grads:
        out.update(g_latents=b.g_latents.cpu().numpy(), g_lens=b.g_lens.cpu().numpy(),
                   g_ps=b.g_ps.cpu().numpy())
        if b.g_light is not None:
            out["g_light"] = b.g_light.cpu().numpy()
    return out, sysm, b


def run_oracle(m, grads=True, transform=0):
    s = oracle_io.system(m)
    s.transform = transform
    lens, lat, ps, subs = oracle_io.params(m)
    light = oracle_io.light(m)
    if grads:
        r = O.forward_adjoint(s, lens, lat, ps, subs, light)
    else:
        f = O.forward(s, lens, lat, ps, subs, light)
        r = dict(logL=f["logL"], chi2=f["chi2"], model=f["model"], image=f["image"], flags=f["T"].flags)
    T = O.build_grid(s, lens, subs)
    src, _ = O.gp_source(s, lat, ps)
    hist = O.ray_hist(s, lens, subs, T)
    if isinstance(T, O.BoxTransform):
        cdf = None          # the box map has no knots of its own to compare
    elif isinstance(T, O.LinearTransform):
        # the unsmoothed eCDF: the standardisation, then zeros in the knot/slope slots
        cdf = np.concatenate([T.mu.detach().numpy(), [float(T.sigma)], np.zeros(4 * (s.n_nodes + 2))])
    else:
        cdf = np.concatenate([T.mu.detach().numpy(), [float(T.sigma)], T.knots.detach().numpy().ravel(),
                              T.slopes.detach().numpy().ravel()])
    out = dict(logL=float(r["logL"]), chi2=float(r["chi2"]), model=r["model"].detach().numpy(),
               image=r["image"].detach().numpy(), source=src.detach().numpy(), cdf=cdf,
               hist=hist.numpy(), flags=T.flags)
    if grads:
        g_lens = r["g_lens"].numpy()
        if subs is not None:
            g_lens = np.concatenate([g_lens, r["g_subs"].numpy().ravel()])
        out.update(g_latents=r["g_latents"].numpy(), g_lens=g_lens, g_ps=r["g_ps"].numpy())
        if light is not None:
            out["g_light"] = r["g_light"].numpy().ravel()
    return out


def compare(g, o):
    res = dict(
        logL=abs(g["stats"][0] - o["logL"]) / abs(o["logL"]),
        chi2=abs(g["stats"][1] - o["chi2"]) / abs(o["chi2"]),
        cdf=rel_l2(g["cdf"], o["cdf"]) if o["cdf"] is not None else 0.0,
        source=rel_l2(g["source"], o["source"]),
        image=rel_l2(g["image"], o["image"]),
        model=rel_l2(g["model"], o["model"]),
        hist_diff=int(np.abs(g["hist"].astype(np.int64) - o["hist"]).sum()),
        flags=(int(g["stats"][3]), o["flags"]),
    )
    if "g_latents" in g and "g_latents" in o:
        res.update(g_latents=rel_l2(g["g_latents"], o["g_latents"]), g_lens=rel_l2(g["g_lens"], o["g_lens"]),
                   g_ps=rel_l2(g["g_ps"], o["g_ps"]))
    if "g_light" in g and "g_light" in o:
        res["g_light"] = rel_l2(g["g_light"], o["g_light"])
    return res
