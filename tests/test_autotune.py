"""The autotuner of launch shapes: the cache's keys and format (CPU), and on the GPU
that a tuned shape changes the work split only (results agree to rounding, and each
shape is reproducible bit for bit), that a sweep returns shapes in range, and that a
system picks up its bucket's cached shape."""
import json

import numpy as np
import pytest
import torch

from paper_2606_30620_b300 import autotune as A
from paper_2606_30620_b300 import inputs as I


def test_bucket_keys_and_the_committed_cache():
    assert A.bucket_key(200, 64, 4, 0) == "200x64x4:f32"
    assert A.bucket_key(96, 48, 3, 1) == "96x48x3:f64"
    data = A.load()
    for gpu, buckets in data.items():
        for key, v in buckets.items():
            n_img, n_src, rest = key.split("x")
            assert rest.split(":")[1] in ("f32", "f64")
            t = v["tuning"]
            assert 1 <= t["adj_div"] <= 64 and 1 <= t["near_ctas"] <= 16 and 1 <= t["edge_ctas"] <= 256
            assert v["ms_tuned"] <= v["ms_default"] * 1.0001


def test_load_reads_a_given_file(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"GPU X": {"64x32x2:f32": {"tuning": {"adj_div": 1, "near_ctas": 2, "edge_ctas": 8},
                                                        "ms_default": 1.0, "ms_tuned": 0.5}}}))
    assert A.load(str(p))["GPU X"]["64x32x2:f32"]["tuning"]["near_ctas"] == 2
    A.load()          # back to the package cache


@pytest.mark.gpu
def test_tuned_shapes_change_only_the_work_split():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu
    from tests import gpu_cases as G
    m = I.config_c2(1007, n_img=96, s=3, n_src=48)
    runs = []
    for t in (A.DEFAULT, {"adj_div": 1, "near_ctas": 1, "edge_ctas": 4}, {"adj_div": 16, "near_ctas": 16,
                                                                          "edge_ctas": 64}):
        s = rtu.System.from_mock(m, precision=rtu.RTU_F64, tune=False)
        s.tune(t)
        b = rtu.Binding(s, m.lens, m.latents, m.ps, want_model=True)
        out = []
        for _ in range(2):
            rtu.Batch([b]).forward()
            rtu.Batch([b]).adjoint()
            torch.cuda.synchronize()
            out.append([b.model.cpu().numpy().copy(), b.g_lens.cpu().numpy().copy(), b.g_latents.cpu().numpy().copy()])
        for u, v in zip(out[0], out[1]):
            assert np.array_equal(u, v)
        runs.append(out[0])
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0])                  # the forward does not depend on the split
        assert G.rel_l2(r[1], runs[0][1]) < 1e-12 and G.rel_l2(r[2], runs[0][2]) < 1e-12


@pytest.mark.gpu
def test_sweep_and_cache_lookup(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu
    mocks = [I.config_serving_system(9100 + k, n_img=64, n_src=32, s=2) for k in range(4)]
    systems = [rtu.System.from_mock(m, tune=False) for m in mocks]
    batch = rtu.Batch([rtu.Binding(s, m.lens, m.latents, m.ps) for s, m in zip(systems, mocks)])
    flush = torch.empty(1 << 20, device="cuda")
    best, ms0, ms1, trials = A.tune_batch(systems, lambda: (batch.forward(), batch.adjoint()), flush, steps=3)
    assert ms1 <= ms0 and len(trials) >= 10
    assert 1 <= best["adj_div"] <= 64 and 1 <= best["near_ctas"] <= 16 and 1 <= best["edge_ctas"] <= 256
    p = tmp_path / "c.json"
    p.write_text(json.dumps({A.gpu_name(): {A.bucket_key(64, 32, 2, 0): {"tuning": best, "ms_default": ms0,
                                                                          "ms_tuned": ms1}}}))
    assert A.lookup(64, 32, 2, 0, path=str(p)) == best
    assert A.lookup(64, 32, 3, 0, path=str(p)) is None
    A.load()
