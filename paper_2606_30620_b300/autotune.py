"""Autotuner of the library's launch shapes (rtu_system_tune) per problem bucket.

A bucket is (image side, source-grid side, supersampling, precision).  For each
bucket the tuner builds a batch of seeded systems of that shape, and sweeps the
three launch knobs one at a time (coordinate descent from the defaults): the
render adjoint's CTAs per system (adj_div), the near-core adjoint pass's CTAs
(near_ctas) and the near-edge double pass's CTAs (edge_ctas).  Each setting is
timed with CUDA events on the launching stream over the step the bucket serves
(one batched ELBO step for the serving buckets, a batched forward + adjoint for
the benchmark bucket), after warm-up, L2 flushed between timed steps.  The best
setting and both timings go into a JSON cache keyed by GPU name and bucket;
``rtu.System`` applies the cached setting of its bucket when it is created.

    python -m paper_2606_30620_b300.autotune [--serving] [--bench] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuning.json")

KNOBS = (("adj_div", (1, 2, 4, 8, 16)), ("near_ctas", (1, 2, 4, 8, 16)), ("edge_ctas", (4, 8, 16, 32, 64)))
DEFAULT = {"adj_div": 4, "near_ctas": 4, "edge_ctas": 16}
L2_BYTES = 126 * 1024 * 1024

_loaded = None


def bucket_key(n_img: int, n_src: int, s: int, precision: int) -> str:
    return f"{n_img}x{n_src}x{s}:{'f64' if precision else 'f32'}"


def gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def load(path: str = CACHE) -> dict:
    """{gpu name: {bucket: {"tuning": {...}, "ms_default": .., "ms_tuned": ..}}} or {}."""
    global _loaded
    if _loaded is None or _loaded[0] != path:
        data = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
        _loaded = (path, data)
    return _loaded[1]


_memo: dict = {}


def lookup(n_img: int, n_src: int, s: int, precision: int, path: str = CACHE):
    """The cached launch shape of a bucket on this GPU, or None (memoised per bucket:
    a serving loop looks it up for every admitted system)."""
    key = (path, n_img, n_src, s, precision)
    if key in _memo:
        return _memo[key]
    if not torch.cuda.is_available():
        return None
    entry = load(path).get(gpu_name(), {}).get(bucket_key(n_img, n_src, s, precision))
    _memo[key] = None if entry is None else entry["tuning"]
    return _memo[key]


def _time(step, flush, steps: int) -> float:
    stream = torch.cuda.current_stream()
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def tune_batch(systems, step, flush, steps: int = 15):
    """Coordinate descent over the knobs for one batch: returns (best, ms_default, ms_best, trials)."""
    from . import rtu

    def run(t):
        for s in systems:
            s.tune(t)
        return _time(step, flush, steps)

    best = dict(DEFAULT)
    ms_default = best_ms = run(best)
    trials = [(dict(best), best_ms)]
    for name, values in KNOBS:
        for v in values:
            if v == best[name]:
                continue
            t = dict(best, **{name: v})
            ms = run(t)
            trials.append((t, ms))
            if ms < best_ms:
                best, best_ms = t, ms
    for s in systems:
        s.tune(best)
    return best, ms_default, best_ms, trials


def tune_serving(n_per_bucket: int = 16, precision: int = 0, seed: int = 9000, steps: int = 15):
    """Every (image, grid, supersampling) bucket of the serving mix, one ELBO step (S = 1)."""
    from . import inputs as I
    from . import rtu
    from .serve import guide_start
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for n_img in I.SERVE_IMG:
        for n_src in I.SERVE_SRC:
            for s in I.SERVE_S:
                mocks = [I.config_serving_system(seed + k, n_img=n_img, n_src=n_src, s=s) for k in range(n_per_bucket)]
                systems = []
                for k, m in enumerate(mocks):
                    sy = rtu.System.from_mock(m, precision=precision, n_slots=1, tune=False)
                    pr, ph, loc, rho = guide_start(m)
                    sy.elbo_init(pr, ph, loc, rho, tag=k)
                    systems.append(sy)
                res = torch.empty(len(systems), dtype=torch.float64, device="cuda")

                def step():
                    rtu.rtu_elbo_step(systems, 1, 0, 1e-3, res)

                best, ms0, ms1, _ = tune_batch(systems, step, flush, steps)
                out[bucket_key(n_img, n_src, s, precision)] = {"tuning": best, "ms_default": ms0, "ms_tuned": ms1,
                                                              "systems": len(systems), "step": "ELBO step, S = 1"}
                for sy in systems:
                    sy.close()
    return out


def tune_bench(n_mocks: int = 32, seed0: int = 1000, steps: int = 20):
    """The benchmark bucket: 32 mocks of 200^2 pixels, 4x4 rays, 64^2 grid, FP32,
    batched forward + adjoint."""
    from . import inputs as I
    from . import rtu
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    mocks = [I.config_c2(seed0 + k) for k in range(n_mocks)]
    systems = [rtu.System.from_mock(m, precision=rtu.RTU_F32, tune=False) for m in mocks]
    batch = rtu.Batch([rtu.Binding(sy, m.lens, m.latents, m.ps) for sy, m in zip(systems, mocks)])

    def step():
        batch.forward()
        batch.adjoint()

    best, ms0, ms1, _ = tune_batch(systems, step, flush, steps)
    return {bucket_key(200, 64, 4, 0): {"tuning": best, "ms_default": ms0, "ms_tuned": ms1, "systems": n_mocks,
                                         "step": "forward + adjoint"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--serving", action="store_true")
    ap.add_argument("--bench", action="store_true")
    ap.add_argument("--out", default=CACHE)
    args = ap.parse_args()
    entries = {}
    if args.bench or not args.serving:
        entries.update(tune_bench())
    if args.serving or not args.bench:
        entries.update(tune_serving())
    data = {}
    if os.path.exists(args.out):
        with open(args.out) as f:
            data = json.load(f)
    data.setdefault(gpu_name(), {}).update(entries)
    with open(args.out, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    for k, v in sorted(entries.items()):
        print(k, v["tuning"], f"{v['ms_default']:.4f} -> {v['ms_tuned']:.4f} ms")


if __name__ == "__main__":
    main()
