"""Benchmark of the RTU-grid hot path on one node (contract: one JSON line on rank 0).

Workload (default): the FP32 forward+adjoint case -- 32 seeded mocks of a
200x200 image at 0.05"/pix, 4x4 supersampling (640,000 rays each), elliptical
power law + shear, 64x64 RTU grid, Matern-like P(k), 21x21 PSF.  One step is
one batched pass of the whole hot path over all 32 mocks: build grid (centre
trace, order statistics, fit), GP source, render with the rays-per-cell
histogram, PSF + likelihood, and the full adjoint (gradients w.r.t. latents,
lens and power-spectrum parameters).  value = forward+adjoint evaluations per
second over the whole job (N ranks x 32 mocks per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the FP64 CPU oracle is timed on the host cores on a
bounded sample of the same workload (the oracle is the reference of this
build; there is no other implementation to run).
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_30620_b300 import inputs as I  # noqa: E402

N_MOCKS = 32
SEED0 = 1000
L2_BYTES = 126 * 1024 * 1024
# FP32 peak from unit counts: SMs (read from the device) x 128 FP32 lanes x 2 flop per
# FMA x the SM clock (the median sampled under load; the recipe's 2032 MHz maximum if
# no sample was taken)
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_RECIPE = 2032.0
FALLBACK_HBM_GBS = 6400.0
# Algorithmic FP32 flops (an FMA counts two) per ray that ends inside the RTU grid, from
# the operation counts of the code at the c2 mocks' mean EPL series length (7.6 terms):
# the forward trace + map + interpolation 228, its adjoint (lens value and series sums,
# map value, slope and knot partials, bilinear slopes, lens vector-Jacobian product)
# 516.  Rays that leave the grid's reach early, and the culled tiles' rays, are not
# counted: the units are the in-grid rays (the N_IN_GRID statistic), for both kernels.
FLOPS_FWD_RAY = 228.0
FLOPS_ADJ_RAY = 516.0
# DRAM read + write per unit from one ncu capture (dram__bytes_read.sum and
# dram__bytes_write.sum, c2 shape, 8 mocks: 5,120,000 rays, 743,894 of them in the grid),
# valid for the kernel sources with digest TRAFFIC_SRC_DIGEST.
ROOF = {
    "k_render": {"flops_per_unit": FLOPS_FWD_RAY, "units": "in-grid rays",
                 "traffic_per_unit": (345600 + 15616) / 743894},
    "k_render_adj": {"flops_per_unit": FLOPS_ADJ_RAY, "units": "in-grid rays",
                     "traffic_per_unit": (9692928 + 143104) / 743894},
}
TRAFFIC_SRC_DIGEST = "e66e8e4e269de769"
KERNEL_SOURCES = ("k_render.cuh", "rtu_internal.cuh", "rtu_math.cuh", "rtu_df.cuh")


def kernel_digest():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_30620_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.first = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # nvidia-smi takes a moment to start: the timed region begins after its first sample
            self.first.wait(timeout=10.0)
            self.lines.clear()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def __exit__(self, *a):
        if self.proc is not None:
            # at least one sample taken after the region's start
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 2.0:
                time.sleep(0.02)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def make_mocks(rank, n=N_MOCKS):
    return [I.config_c2(SEED0 + rank * n + k) for k in range(n)]


def cpu_oracle_sample(mocks, budget_s=20.0, max_n=None, keep_first=False):
    """The oracle as it stands on the host cores: forward + gradient per mock until
    the budget is spent (at least one mock).  keep_first: also return the first mock's
    oracle result (log L, model, image, gradients), which the bench line's relative
    errors are measured against."""
    from oracle import rtu_oracle as O
    from tests import oracle_io
    torch.set_num_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    n = 0
    first = None
    for m in mocks:
        s = oracle_io.system(m)
        lens, lat, ps, subs = oracle_io.params(m)
        r = O.forward_adjoint(s, lens, lat, ps, subs)
        if first is None and keep_first:
            first = {k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
        n += 1
        if time.perf_counter() - t0 > budget_s or (max_n and n >= max_n):
            break
    dt = time.perf_counter() - t0
    if keep_first:
        return n / dt, n, dt, torch.get_num_threads(), first
    return n / dt, n, dt, torch.get_num_threads()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    mocks = make_mocks(0)
    per = []
    for _ in range(args.warmup if args.warmup < 1 else 1):
        cpu_oracle_sample(mocks[:1], budget_s=0.0)
    t_all = 0.0
    n_all = 0
    for k in range(args.steps):
        v, n, dt, cores = cpu_oracle_sample(mocks[k % N_MOCKS:], budget_s=10.0, max_n=4)
        per.append(dt / n)
        t_all += dt
        n_all += n
    value = n_all / t_all
    line = {"impl": "reference", "metric": "forward+adjoint evals/s", "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded mocks)",
            "config": {"workload": "c2: 200x200 image 0.05\"/pix, 4x4 rays, EPL+shear, 64x64 RTU grid, "
                                   "Matern-like P(k), 21x21 PSF, 32 seeded mocks",
                       "sample": f"{n_all} mock forward+gradient evaluations"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{n_all} of the 32 mocks, FP64 oracle forward + autograd gradient"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    rank, world, local = env_rank()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2606_30620_b300 import rtu

    mocks = make_mocks(rank, args.mocks)
    systems = [rtu.System.from_mock(m, precision=rtu.RTU_F32, device=dev) for m in mocks]
    n = len(mocks)
    n2 = mocks[0].n_src ** 2
    nps = mocks[0].ps.size
    # inputs [lens(8) | ps(3)] as float64 and latents as float32, outputs [stats | g_lens |
    # g_ps] as float64 and g_latents as float32, each direction packed in one byte buffer
    # (one copy each way per step) with typed views for the bindings
    NS = rtu.N_STATS
    a_in, a_out = n * (8 + nps) * 8, n * (NS + 8 + nps) * 8

    def packed(a_bytes, device, pin=False):
        buf = torch.empty(a_bytes + n * n2 * 4, dtype=torch.uint8, device=device)
        if pin:
            buf = buf.pin_memory()
        return buf, buf[:a_bytes].view(torch.float64).view(n, -1), buf[a_bytes:].view(torch.float32).view(n, n2)

    in_buf, in_f64, in_lat = packed(a_in, dev)
    out_buf, out_f64, out_lat = packed(a_out, dev)
    h_in_buf, h_in_f64, h_in_lat = packed(a_in, "cpu", pin=True)
    h_out_buf, h_out_f64, h_out_lat = packed(a_out, "cpu", pin=True)
    h_in_f64.copy_(torch.tensor(np.stack([np.concatenate([m.lens, m.ps]) for m in mocks]), dtype=torch.float64))
    h_in_lat.copy_(torch.tensor(np.stack([m.latents.ravel() for m in mocks]), dtype=torch.float32))
    in_buf.copy_(h_in_buf)
    binds = []
    for k, s in enumerate(systems):
        binds.append(rtu.Binding(s, in_f64[k, :8], in_lat[k].view(mocks[k].n_src, mocks[k].n_src),
                                 in_f64[k, 8:], out={"stats": out_f64[k, :NS], "g_lens": out_f64[k, NS:NS + 8],
                                                     "g_ps": out_f64[k, NS + 8:],
                                                     "g_latents": out_lat[k].view(mocks[k].n_src, mocks[k].n_src)}))
    batch = rtu.Batch(binds)
    singles = [rtu.Batch([b]) for b in binds]
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        batch.forward(stream)
        batch.adjoint(stream)

    def step_single():
        for b in singles:
            b.forward(stream)
            b.adjoint(stream)

    def barrier():
        if dist:
            tdist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, L2 flushed between steps (untimed)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier()
    # ---- per-kernel times: a separate pass with CUDA events around every launch (on the
    # stream each kernel is launched on), same workload and L2 flushes, not in `value`
    rtu.profile_report()          # clear
    rtu.profile_enable(True)
    n_prof = min(args.steps, 50)
    for i in range(n_prof):
        flush.fill_(float(i))
        step()
    torch.cuda.synchronize()
    rtu.profile_enable(False)
    kern = rtu.profile_report()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t)
    value = world * n / (ms / 1e3)

    # ---- the same step captured once as a CUDA graph and replayed (launch overhead
    # of the ~20 kernels and the side-stream fork/join paid once at capture)
    graph_ms = None
    if not args.no_graph:
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            step_on = lambda: (batch.forward(gs), batch.adjoint(gs))
            step_on()                         # warm on the capture stream
            gs.synchronize()
            with torch.cuda.graph(graph, stream=gs):
                step_on()
        torch.cuda.synchronize()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        g0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        g1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        cur = torch.cuda.current_stream()
        for i in range(args.steps):
            flush.fill_(float(i))
            g0[i].record(cur)
            graph.replay()
            g1[i].record(cur)
        torch.cuda.synchronize()
        graph_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(g0, g1))

    # ---- plain per-system path (one call per mock), same work
    per_system_value = None
    if not args.no_single:
        for _ in range(2):
            step_single()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(1, min(args.steps, 5))
        single_ms = []
        for i in range(ks):
            flush.fill_(float(i))
            s0.record(stream)
            step_single()
            s1.record(stream)
            torch.cuda.synchronize()
            single_ms.append(s0.elapsed_time(s1))
        per_system_value = n / (statistics.mean(single_ms) / 1e3)

    # ---- end to end through the public API: pinned host params in, results out
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0.record(stream)
        in_buf.copy_(h_in_buf, non_blocking=True)
        step()
        h_out_buf.copy_(out_buf, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    e2e = world * n / (statistics.mean(e_ms) / 1e3)
    h2d = h_in_f64.numel() * 8 + h_in_lat.numel() * 4
    d2h = h_out_f64.numel() * 8 + h_out_lat.numel() * 4

    # ---- dominant kernel: average launch duration from the events of the timed region
    top = max(kern.items(), key=lambda kv: kv[1][1])
    dom = max(ROOF, key=lambda k: kern[k][1])
    dom_ms = kern[dom][1] / kern[dom][0]
    kern_tot = sum(v[1] for v in kern.values())
    # kernels of this library per step (counted in the profiled pass) x timed steps
    launches = sum(v[0] for v in kern.values()) // n_prof * args.steps

    # ---- mock 0 of the timed batch once more with its image outputs, for the relative
    # errors against the FP64 oracle quoted on the line (the oracle runs in the CPU leg)
    b0 = rtu.Binding(systems[0], mocks[0].lens, mocks[0].latents, mocks[0].ps, want_model=True, want_image=True)
    rtu.Batch([b0]).forward(stream)
    rtu.Batch([b0]).adjoint(stream)
    torch.cuda.synchronize()
    gpu0 = {"logL": float(b0.stats[rtu.STAT_LOGL]), "model": b0.model.cpu().numpy(),
            "image": b0.image.cpu().numpy(), "g_latents": b0.g_latents.cpu().numpy(),
            "g_lens": b0.g_lens.cpu().numpy(), "g_ps": b0.g_ps.cpu().numpy()}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    # ---- the autotuner: the benchmark bucket timed live with the default launch shapes
    # and with the cached tuned ones; the serving buckets' speed-ups as cached
    tune_info = run_autotune_report(systems, step, flush, stream) if not args.no_autotune else None

    clocks = clk.summary()
    variants = run_variants(args, dev, mocks, flush, stream) if not args.no_variants else None
    serving = run_serving(args, dev) if args.serve_n > 0 else None
    if rank != 0:
        if dist:
            tdist.destroy_process_group()
        return 0
    peaks, peak_kind = measured_peaks()
    # the adjoint differentiates the rays inside the RTU grid (zero gradient elsewhere)
    rays_in = float(out_f64[:, rtu.STAT_N_IN_GRID].sum())
    rays = sum(m.n_rays for m in mocks)
    units = rays_in
    achieved = ROOF[dom]["flops_per_unit"] * units / (dom_ms / 1e3) / 1e12
    clock_mhz = clocks["sm_mhz"] or clocks["sm_max_mhz"] or SM_MAX_MHZ_RECIPE
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    # both ray kernels against the same peak (the dominant one is the line's roofline)
    per_kernel = {k: {"launch_ms": kern[k][1] / kern[k][0],
                      "frac": ROOF[k]["flops_per_unit"] * units / (kern[k][1] / kern[k][0] / 1e3) / 1e12 / fp32_peak}
                  for k in ROOF}
    # DRAM bytes from one ncu capture, per unit, scaled to this launch; null when the
    # kernel sources differ from the ones that were captured
    traffic = (ROOF[dom]["traffic_per_unit"] * units) if kernel_digest() == TRAFFIC_SRC_DIGEST else None
    # cpu baseline: the oracle on the host cores, a bounded sample of the same mocks
    cpu_v, cpu_n, cpu_dt, cores, orc0 = (cpu_oracle_sample(mocks, budget_s=args.cpu_budget, keep_first=True)
                                         if not args.no_cpu else (None, 0, 0.0, 0, None))
    rel_err = None
    if orc0 is not None:
        rel_err = {"mock": mocks[0].name, "tolerance": 1e-5,
                   "logL": abs(gpu0["logL"] - float(orc0["logL"])) / abs(float(orc0["logL"])),
                   **{k: rel_l2(gpu0[k], orc0[k]) for k in ("image", "model", "g_latents", "g_lens", "g_ps")}}
    line = {
        "metric": "forward+adjoint evals/s", "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded mocks)",
        "config": {"workload": "c2: 200x200 image 0.05\"/pix, 4x4 rays (640k per mock), EPL+shear, "
                               f"64x64 RTU grid, Matern-like P(k), 21x21 PSF, {n} seeded mocks batched per step",
                   "mocks_per_rank": n, "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}", "wall_s_timed_loop": t_wall},
        "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernels": {k: {"launches": c, "avg_ms": t / c, "share": t / kern_tot} for k, (c, t) in kern.items()},
        "cuda_graph": None if graph_ms is None else {
            "value": world * n / (graph_ms / 1e3), "unit": "evals/s", "ms_per_step": graph_ms,
            "note": "the batched step captured once as a CUDA graph, replayed per step"},
        "per_system_path": {"value": per_system_value, "unit": "evals/s",
                            "note": "same 32 evaluations issued as 32 single-system calls"},
        "roofline": {"kernel": dom + "<float>", "top_kernel": top[0], "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic, "launch_ms": dom_ms, "units": ROOF[dom]["units"],
                     "units_per_launch": units, "rays_per_launch": rays, "in_grid_rays_per_launch": rays_in,
                     "flops_per_unit": ROOF[dom]["flops_per_unit"], "ray_kernels": per_kernel,
                     "peak_note": f"FP32 FMA peak from unit counts: {sm_count} SMs (device) x "
                                  f"{FP32_LANES_PER_SM} lanes x 2 x {clock_mhz:.0f} MHz (median SM clock "
                                  "sampled in the timed region)",
                     "sm_count": sm_count, "sm_mhz": clock_mhz,
                     "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_kind": peak_kind},
        "cpu_baseline": {"value": cpu_v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cpu_n} of the {n} mocks ({cpu_dt:.1f} s): FP64 oracle forward + autograd gradient"},
        "rel_err": rel_err,
        "autotune": tune_info,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "variants": variants,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    if dist:
        tdist.destroy_process_group()
    return 0


# the NEXT variants of the hot path on the same mocks: the kernels each one adds or
# swaps, and its whole-step throughput
VARIANT_KERNELS = ("k_select_fit", "k_lin_sort", "k_render", "k_render_edge", "k_render_adj", "k_cdf_adj",
                   "k_centre_adj", "k_sel_jac", "k_lin_centre_adj", "k_light_fwd", "k_light_adj", "k_sub_adj",
                   "k_render_adj_near")


def run_variants(args, dev, mocks, flush, stream):
    from paper_2606_30620_b300 import inputs as I
    from paper_2606_30620_b300 import rtu
    specs = [("uniform_grid", "box around the masked rays (Sec. 2.1)",
              lambda m: m, rtu.RTU_TRANSFORM_UNIFORM),
             ("weighted_grid", "integer SNR weights, cap 100 (Sec. 6.3)",
              lambda m: I.with_snr_weights(copy.copy(m)), rtu.RTU_TRANSFORM_RTU),
             ("lens_light", "5-component MGE lens light (App. A.3)",
              lambda m: I.with_light(copy.copy(m), n=5, seed=3, amp=0.3), rtu.RTU_TRANSFORM_RTU),
             ("linear_ecdf", "unsmoothed linear-interpolated eCDF (App. C)",
              lambda m: m, rtu.RTU_TRANSFORM_LINEAR)]
    # config c4 on its own mocks (8 seeds): 400^2 at 0.03"/pix, 3x3 rays, 128^2 grid,
    # EPL + shear with 1-10 truncated NFW subhaloes, and the same systems without them
    c4 = {sub: [I.config_c4(3000 + k, with_subs=sub) for k in range(8)] for sub in (True, False)}
    specs += [("c4_subhaloes", "c4: 400^2, 3x3 rays, 128^2 grid, EPL + shear + 1-10 tNFW subhaloes, 8 mocks",
               c4[True], rtu.RTU_TRANSFORM_RTU),
              ("c4_no_subhaloes", "c4: the same 8 systems without subhaloes",
               c4[False], rtu.RTU_TRANSFORM_RTU)]
    out = {}
    k_steps = max(1, min(args.steps, 100))
    for name, what, make, transform in specs:
        ms_ = make if isinstance(make, list) else [make(m) for m in mocks]
        systems = [rtu.System.from_mock(m, precision=rtu.RTU_F32, device=dev, transform=transform) for m in ms_]
        batch = rtu.Batch([rtu.Binding(s, m.lens if m.subs is None else np.concatenate([m.lens, m.subs.ravel()]),
                                       m.latents, m.ps, light=getattr(m, "light", None))
                           for s, m in zip(systems, ms_)])

        def step():
            batch.forward(stream)
            batch.adjoint(stream)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        for i in range(k_steps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        rtu.profile_report()
        rtu.profile_enable(True)
        n_prof = min(k_steps, 20)
        for i in range(n_prof):
            flush.fill_(float(i))
            step()
        torch.cuda.synchronize()
        rtu.profile_enable(False)
        kern = rtu.profile_report()
        out[name] = {"what": what, "value": len(ms_) / (ms / 1e3), "unit": "evals/s", "ms_per_step": ms,
                     "steps": k_steps,
                     "kernels_ms": {k: kern[k][1] / n_prof for k in VARIANT_KERNELS if k in kern}}
        del batch, systems
    return out


def run_autotune_report(systems, step, flush, stream, steps=50):
    from paper_2606_30620_b300 import autotune
    cached = autotune.lookup(systems[0].n_img, systems[0].n_src, systems[0].s_super, systems[0].precision)

    def timed(tuning):
        for s in systems:
            s.tune(tuning)
        return autotune._time(step, flush, steps)

    ms_default = timed(autotune.DEFAULT)
    ms_tuned = timed(cached) if cached is not None else ms_default
    for s in systems:                       # leave the systems as the timed region ran them
        s.tune(cached if cached is not None else autotune.DEFAULT)
    entries = autotune.load().get(autotune.gpu_name(), {})
    sp = [v["ms_default"] / v["ms_tuned"] for k, v in entries.items() if v.get("step", "").startswith("ELBO")]
    return {"cache": "paper_2606_30620_b300/tuning.json", "gpu": autotune.gpu_name(), "buckets": len(entries),
            "bench_bucket": {"tuning": cached, "ms_default": ms_default, "ms_tuned": ms_tuned,
                             "note": "batched forward + adjoint of the 32 mocks, live (median of 50 steps)"},
            "serving_buckets": None if not sp else {
                "n": len(sp), "speedup_median": float(np.median(sp)), "speedup_min": float(min(sp)),
                "speedup_max": float(max(sp)),
                "note": "one batched ELBO step of 16 systems per bucket, default / tuned, as measured by the tuner"}}


def run_serving(args, dev):
    """The serving workload: a stream of lens systems (image 64-256^2, grid 32-128^2,
    2-4x rays, SIE or EPL + shear) arriving Poisson at 2000/s, one ELBO step each with
    the state kept on the device, 120 GB admission budget; each request carries its
    observation and its starting guide.  Measured three ways on the same systems: the
    continuous-batching server in real time (latency; three runs, the run with the
    median p99 reported and every run's p50 / p99 beside it, since one host stall in a
    2-second run moves the p99 of that run alone), the server with every request
    queued at t = 0 (saturation throughput), the same under a 64 MB admission budget
    (the budget binds: admission waits for completions to free workspace), and the
    plain per-system path.
    An untimed warm-up pass of the same stream (every request queued at t = 0) runs
    first, as the step timings run warm-up steps: it fills the device workspace pool
    that admission draws on (the serving loop then makes no device allocation); every
    system is built again from its observation when the timed runs admit it."""
    from paper_2606_30620_b300 import serve
    base = serve.make_stream(args.serve_n, 2000.0, seed=5000)

    def fresh():
        return [serve.Request(rid=r.rid, system_id=r.system_id, mock=r.mock, arrival=r.arrival, guide=r.guide)
                for r in base]

    serve.Server(budget_bytes=120 << 30, max_batch=32, n_samples=1, device=dev).run(fresh(), realtime=False)
    torch.cuda.synchronize()
    runs = [serve.Server(budget_bytes=120 << 30, max_batch=32, n_samples=1, device=dev).run(fresh(), realtime=True)
            for _ in range(3)]
    live = sorted(runs, key=lambda r: r["p99_ms"])[1]
    sat = serve.Server(budget_bytes=120 << 30, max_batch=32, n_samples=1, device=dev).run(fresh(), realtime=False)
    tight = serve.Server(budget_bytes=64 << 20, max_batch=32, n_samples=1, device=dev)
    small = tight.run(fresh(), realtime=False)
    plain = serve.serve_plain(fresh(), n_samples=1, device=dev)
    keep = ("systems", "wall_s", "systems_per_s", "p50_ms", "p99_ms", "mean_batch")
    return {"stream": f"{args.serve_n} systems, Poisson 2000/s, one ELBO step (S=1) each, 120 GB budget",
            "open_loop": dict({k: live[k] for k in keep},
                              runs_p50_p99_ms=[[round(r["p50_ms"], 2), round(r["p99_ms"], 2)] for r in runs]),
            "saturation": {k: sat[k] for k in keep},
            "budget_64mb": dict({k: small[k] for k in keep}, peak_bytes=small["peak_bytes"],
                                budget_bytes=64 << 20, batches=small["batches"]),
            "plain_per_system": {k: plain[k] for k in ("systems", "wall_s", "systems_per_s")}}


def run_timeline(args):
    """Per-launch timeline of one batched step (forward + adjoint) with every launch
    bracketed by events (the library's tracing aid, which launches plainly and adds a
    little time per launch): the median over 5 steps after warm-up and an L2 flush,
    one line per launch "<kernel> <stream> <start_us> <end_us> <us>", stream 0 the
    call's, 1 the library's side stream.  A diagnostic, not a bench line."""
    from paper_2606_30620_b300 import rtu
    mocks = make_mocks(0, args.mocks)
    binds = [rtu.Binding(rtu.System.from_mock(m, precision=rtu.RTU_F32), m.lens, m.latents, m.ps) for m in mocks]
    batch = rtu.Batch(binds)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        batch.forward()
        batch.adjoint()
    torch.cuda.synchronize()
    rtu.profile_report()
    runs = []
    for _ in range(5):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        rtu.profile_enable(True)
        batch.forward()
        batch.adjoint()
        rtu.profile_enable(False)
        torch.cuda.synchronize()
        runs.append(rtu.profile_timeline())
    rows = []
    for i in range(len(runs[0])):
        a = float(np.median([r[i][2] for r in runs]))
        b = float(np.median([r[i][3] for r in runs]))
        rows.append((runs[0][i][0], runs[0][i][1], a, b))
    for name, side, a, b in sorted(rows, key=lambda r: r[2]):
        print(f"{name} {side} {a * 1e3:.1f} {b * 1e3:.1f} {(b - a) * 1e3:.1f}")
    print(f"end {max(r[3] for r in rows) * 1e3:.1f}")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--mocks", type=int, default=N_MOCKS, help="mocks per rank (32 is the benchmark workload)")
    ap.add_argument("--no-single", action="store_true", help="skip the per-system comparison path")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-variants", action="store_true", help="skip the timing of the grid / light variants")
    ap.add_argument("--serve-n", type=int, default=4096, help="systems in the serving stream (0 = skip)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the tuned / default launch-shape timing")
    ap.add_argument("--timeline", action="store_true",
                    help="print the per-launch timeline of one traced step instead of the bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.timeline:
        return run_timeline(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
