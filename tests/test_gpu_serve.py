"""Continuous-batching server: every request completes, each system's result is
the same alone and in the mix (bit for bit: every sum of a step is per system and
in a fixed order), admission respects the HBM budget, and multi-step requests keep
their state on the device."""
import numpy as np
import pytest
import torch

from paper_2606_30620_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import serve as mod
    return mod


def small_stream(serve, n, rate=400.0, seed=7000):
    times = I.poisson_arrivals(n, rate, seed)
    reqs = []
    for k in range(n):
        m = I.config_serving_system(seed + 1 + k)
        # keep the test quick: cap the image at 128^2 and 3x3 rays
        if m.n_img > 128 or m.s_super > 3:
            m = I.config_c2(seed + 1 + k, n_img=96, s=2, n_src=m.n_src)
        reqs.append(serve.Request(rid=k, system_id=k, mock=m, arrival=float(times[k])))
    return reqs


def test_results_alone_equal_results_in_the_mix(serve):
    reqs = small_stream(serve, 24)
    srv = serve.Server(budget_bytes=8 << 30, max_batch=8, n_samples=1, lr=1e-3)
    out = srv.run(reqs, realtime=True)
    assert out["systems"] == 24 and all(r.finish is not None for r in reqs)
    assert out["p99_ms"] >= out["p50_ms"] > 0
    alone = small_stream(serve, 24)
    serve.serve_plain(alone, n_samples=1, lr=1e-3)
    for a, b in zip(reqs, alone):
        assert a.elbo == b.elbo, (a.rid, a.elbo, b.elbo)
    assert out["mean_batch"] >= 1.0


def test_small_budget_forces_queueing(serve):
    reqs = small_stream(serve, 12)
    need = max(serve.workspace_bytes(r.mock, 0, 1) for r in reqs)
    srv = serve.Server(budget_bytes=int(2.5 * need), max_batch=8)
    out = srv.run(reqs, realtime=False)
    assert all(r.finish is not None for r in reqs)
    # the budget holds at most a few systems at once, so batches stay small
    assert srv.peak_used <= int(2.5 * need)
    assert len(srv.batch_sizes) >= 4 and max(srv.batch_sizes) < 8


def test_multi_step_requests_keep_state_on_device(serve):
    reqs = small_stream(serve, 6)
    for r in reqs:
        r.n_steps = 3
    srv = serve.Server(budget_bytes=8 << 30, max_batch=8, keep_resident=True)
    srv.run(reqs, realtime=False)
    assert all(r.done_steps == 3 for r in reqs)
    for r in reqs:
        loc, rho, t = srv.resident[r.system_id].system.elbo_state()
        assert t == 3


def test_workspace_pool_serves_a_second_stream_without_allocating(serve):
    """Released systems hand their workspaces back to the device's pool; the same stream
    served again by a new server takes every workspace from it (no device allocation in
    the serving loop), and the results stay the same bit for bit."""
    pool = serve.workspace_pool("cuda")
    first = small_stream(serve, 16)
    serve.Server(budget_bytes=8 << 30, max_batch=8).run(first, realtime=False)
    made = pool.created
    again = small_stream(serve, 16)
    serve.Server(budget_bytes=8 << 30, max_batch=8).run(again, realtime=False)
    assert pool.created == made
    for a, b in zip(first, again):
        assert a.elbo == b.elbo, (a.rid, a.elbo, b.elbo)


def test_requests_carrying_their_guide_match_guides_built_at_admission(serve):
    """A request may carry its starting guide already packed (start_guide, what a client
    sends); the server then uploads it as given: the same ELBO bit for bit as a guide
    built from the mock at admission, and the plain path agrees."""
    plain = small_stream(serve, 10)
    serve.Server(budget_bytes=8 << 30, max_batch=8).run(plain, realtime=False)
    carried = small_stream(serve, 10)
    for r in carried:
        r.guide = serve.start_guide(r.mock)
    serve.Server(budget_bytes=8 << 30, max_batch=8).run(carried, realtime=True)
    for a, b in zip(plain, carried):
        assert a.elbo == b.elbo, (a.rid, a.elbo, b.elbo)
