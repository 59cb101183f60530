"""Continuous-batching server of ELBO-step requests for many lens systems.

Each request asks for optimiser steps of one lens system (its observation
and starting guide).  The server keeps every admitted system's workspace,
latents and Adam state on the device, admits new systems while their
workspace fits an HBM budget, and batches the ready requests of systems of
uneven image and grid sizes into one ``rtu_elbo_step`` call (one launch per
step of the hot path for the whole batch).  Up to ``n_streams`` batches are in
flight on separate CUDA streams, so requests that arrive while others run
are admitted as memory and stream slots free up and their work overlaps on
the device.  Admission uploads a system's observation, tables and guide with
copies ordered on an admission stream that the batches' streams wait for, so
the host never waits for the device to admit; its workspace comes from a
per-device pool of released workspaces (by size class), so a warm server makes
no device allocation.  A request completes when the
CUDA event recorded after its batch (and the copy of its ELBO into pinned host
memory) has been reached; its latency is completion minus arrival time.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs as I
from . import rtu


@dataclass
class Request:
    rid: int
    system_id: int
    mock: I.Mock
    arrival: float                  # seconds after the stream starts
    n_steps: int = 1
    # the starting guide the client sends, as start_guide returns it (packed priors, fixed
    # values, loc, rho); None: built from the mock at admission (guide_start)
    guide: tuple | None = None
    done_steps: int = 0
    finish: float | None = None
    elbo: float | None = None


@dataclass
class Resident:
    system: rtu.System
    nbytes: int
    last_used: float
    pending: int = 0


def guide_start(m: I.Mock, rho0: float = -3.0):
    """Priors (Table A1), fixed physical values and the starting guide of a mock:
    loc at the mock's own parameters, softplus(rho0) scale."""
    n_sub = 0 if m.subs is None else m.subs.shape[0]
    priors = I.default_priors(m.profile, m.sub_kind, n_sub, m.ps_family, m.subs)
    phys = list(m.lens) + ([] if m.subs is None else list(m.subs.ravel())) + list(m.ps)
    targets = _targets(m.profile, m.sub_kind, n_sub, len(m.ps))
    light = [] if getattr(m, "light", None) is None else list(m.light.ravel())     # held fixed
    loc = [I.unconstrain(math.log10(phys[t]) if p[1] == I.SPACE_LOG10 else phys[t], p)
           for t, p in zip(targets, priors)]
    loc = np.concatenate([np.asarray(loc, dtype=np.float64), m.latents.ravel()])
    rho = np.full(loc.size, rho0)
    return priors, np.array(phys + light), loc, rho


def start_guide(m: I.Mock, rho0: float = -3.0):
    """guide_start with the priors packed for the ABI (rtu.pack_priors) and the arrays in
    the types the library reads: what a client sends with its request."""
    pr, ph, loc, rho = guide_start(m, rho0)
    return (rtu.pack_priors(pr), np.ascontiguousarray(ph, dtype=np.float64),
            np.ascontiguousarray(loc, dtype=np.float64), np.ascontiguousarray(rho, dtype=np.float64))


def _targets(profile, sub_kind, n_sub, nps):
    # site order of the ABI: theta_E, [gamma], e1, e2, x0, y0, G1, G2, per subhalo
    # (kappa_s, r_s, x_s, y_s), then the nps power-spectrum entries (alpha_src last)
    idx = [0] + ([1] if profile == I.PROFILE_EPL else []) + [2, 3, 4, 5, 6, 7]
    ns = n_sub if sub_kind else 0
    for h in range(ns):
        idx += [8 + 5 * h, 8 + 5 * h + 1, 8 + 5 * h + 3, 8 + 5 * h + 4]
    nl = 8 + 5 * ns
    return idx + [nl + k for k in range(nps)]


def workspace_bytes(m: I.Mock, precision: int, n_samples: int) -> int:
    """Device bytes a system occupies while resident (its workspace + observation)."""
    d = rtu.SystemDesc(m.n_img, m.s_super, m.n_src, m.psf.shape[0], m.profile, m.sub_kind,
                       0 if m.subs is None else m.subs.shape[0], m.ps_family, precision, 22, 21, n_samples,
                       0, 0 if getattr(m, "light", None) is None else m.light.shape[0],
                       m.pix, m.src_pitch, m.sigma, 1 << 20, 1 << 20, 1 << 20, None)
    import ctypes
    ws = rtu._lib.rtu_workspace_size(ctypes.byref(d))
    tb = 8 if precision == rtu.RTU_F64 else 4
    return int(ws) + m.n_img * m.n_img * (tb + 1) + m.psf.size * tb + 4096


class WorkspacePool:
    """Device workspaces of admitted systems, kept by size class (rounded up to a multiple
    of an eighth of the power of two below the size: at most 12.5% more) and handed out again once their system is released: after a
    warm-up, admission makes no device allocation (a stream of systems of many sizes
    otherwise keeps fragmenting the caching allocator, and a fresh device allocation in
    the serving loop delays every request behind it).  Blocks are never freed."""

    def __init__(self, device):
        self.device = torch.device(device)
        self.free: dict[int, list] = {}
        self.created = 0                  # blocks allocated so far

    @staticmethod
    def size_class(nbytes: int) -> int:
        p = 1 << max(0, nbytes.bit_length() - 4)             # an eighth of the power of two below
        return -(-nbytes // p) * p

    def take(self, nbytes: int):
        c = self.size_class(nbytes)
        lst = self.free.get(c)
        if lst:
            return lst.pop()
        self.created += 1
        return torch.empty(c, dtype=torch.uint8, device=self.device)

    def give(self, block):
        self.free.setdefault(block.numel(), []).append(block)


_POOLS: dict = {}


def workspace_pool(device) -> WorkspacePool:
    """The process's workspace pool of a device (shared by every server on it)."""
    d = torch.device(device)
    key = (d.type, d.index if d.index is not None else torch.cuda.current_device())
    if key not in _POOLS:
        _POOLS[key] = WorkspacePool(d)
    return _POOLS[key]


class PinnedRing:
    """Pinned host memory for the admission copies, handed out in FIFO order: a slice
    is reused once the event recorded after its copy has been reached (no pinned
    allocation per admitted system)."""

    def __init__(self, nbytes: int):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        self.n = nbytes
        self.head = 0                     # next free byte (wraps)
        self.live = deque()               # (start, end, event) of slices still being copied

    def _retire(self, block: bool):
        while self.live and (block or self.live[0][2].query()):
            self.live[0][2].synchronize()
            self.live.popleft()
            block = False

    def take(self, nbytes: int):
        if nbytes > self.n:
            return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        self._retire(False)
        while True:
            start = self.head if self.head + nbytes <= self.n else 0
            end = start + nbytes
            busy = any(a < end and start < b for a, b, _ in self.live)
            if not busy:
                self.head = end
                return self.buf[start:end], (start, end)
            self._retire(True)

    def commit(self, span, event):
        if span is not None:
            self.live.append((span[0], span[1], event))


class Server:
    def __init__(self, budget_bytes: int, max_batch: int = 32, n_samples: int = 1, lr: float = 1e-3,
                 seed: int = 0, precision: int = rtu.RTU_F32, n_streams: int = 2, device: str = "cuda",
                 keep_resident: bool = False, staging_bytes: int = 64 << 20):
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.n_samples = n_samples
        self.lr = lr
        self.seed = seed
        self.precision = precision
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.admit_stream = torch.cuda.Stream(device=self.device)
        self.keep_resident = keep_resident
        self.resident: dict[int, Resident] = {}
        self.used = 0
        self.peak_used = 0
        self.inflight = []        # (event, stream index, [requests], pinned ELBO values)
        self.batches = 0
        self.batch_sizes = []
        # per stream: the batch's ELBO outputs on the device and their pinned host copy
        self.out_dev = [torch.empty(max_batch, dtype=torch.float64, device=self.device) for _ in self.streams]
        self.out_host = [torch.empty(max_batch, dtype=torch.float64, pin_memory=True) for _ in self.streams]
        self.staging = PinnedRing(staging_bytes)
        self.pool = workspace_pool(self.device)

    # ---------------------------------------------------------------- admission
    def _admit(self, req: Request, now: float) -> bool:
        r = self.resident.get(req.system_id)
        if r is not None:
            r.last_used = now
            return True
        need = workspace_bytes(req.mock, self.precision, self.n_samples)
        if need > self.budget:
            raise ValueError(f"system {req.system_id} needs {need} bytes, above the budget")
        if self.used + need > self.budget:
            self._evict(need)
            if self.used + need > self.budget:
                return False
        # the observation in one pinned copy, the library's tables and the guide with
        # uploads ordered on the admission stream; nothing waits for the device here
        # (the batch's stream waits for the admission stream before its step)
        m = req.mock
        got = self.staging.take(rtu.System.staging_bytes(m.data.size, m.psf.size, self.precision,
                                                          getattr(m, "weights", None) is not None))
        buf, span = got if isinstance(got, tuple) else (got, None)
        s = rtu.System.from_mock(m, precision=self.precision, n_slots=self.n_samples, device=self.device,
                                 stream=self.admit_stream, host_staging=buf, alloc=self.pool.take)
        pr, ph, loc, rho = req.guide if req.guide is not None else guide_start(m)
        s.elbo_init(pr, ph, loc, rho, tag=req.system_id, stream=self.admit_stream)
        ev = torch.cuda.Event()
        ev.record(self.admit_stream)
        self.staging.commit(span, ev)
        self.resident[req.system_id] = Resident(s, need, now)
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        return True

    def _evict(self, need: int):
        # idle residents (no queued or running request), least recently used first
        idle = sorted((r.last_used, sid) for sid, r in self.resident.items() if r.pending == 0)
        for _, sid in idle:
            if self.used + need <= self.budget:
                break
            self._release(sid)

    def _release(self, sid: int):
        # called once the system's last batch has completed (its event was reached),
        # so its workspace can serve the next admission
        r = self.resident.pop(sid)
        r.system.close()
        for block in r.system.pool_blocks:
            self.pool.give(block)
        self.used -= r.nbytes

    # ----------------------------------------------------------------- batching
    def _launch(self, reqs, k):
        st = self.streams[k]
        out = self.out_dev[k][:len(reqs)]
        host = self.out_host[k][:len(reqs)]
        systems = [self.resident[r.system_id].system for r in reqs]
        st.wait_stream(self.admit_stream)
        rtu.rtu_elbo_step(systems, self.n_samples, self.seed, self.lr, out, stream=st)
        # the ELBO values into pinned host memory behind the step; read once the event is reached
        with torch.cuda.stream(st):
            host.copy_(out, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(st)
        self.inflight.append((ev, k, reqs, host))
        self.batches += 1
        self.batch_sizes.append(len(reqs))

    def _complete(self, t, ready):
        """Retire the batches whose event has been reached; re-queue requests with
        steps left, release finished systems unless they are kept resident."""
        keep = []
        for item in self.inflight:
            ev, k, reqs, out = item
            if not ev.query():
                keep.append(item)
                continue
            vals = out.numpy()              # pinned host copy, complete once the event is reached
            for r, v in zip(reqs, vals):
                r.done_steps += 1
                r.elbo = float(v)
                res = self.resident[r.system_id]
                res.pending -= 1
                res.last_used = t
                if r.done_steps < r.n_steps:
                    ready.append(r)
                else:
                    r.finish = t
                    if not self.keep_resident and res.pending == 0:
                        self._release(r.system_id)
        self.inflight = keep

    def run(self, requests, realtime: bool = True):
        """Serve a list of requests; with realtime=False all arrive at t = 0
        (saturation).  Returns the latency/throughput summary."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            r.done_steps, r.finish = 0, None
            if not realtime:
                r.arrival = 0.0
        arrivals = deque(reqs)
        ready = deque()
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while arrivals or ready or self.inflight:
            t = now()
            while arrivals and arrivals[0].arrival <= t:
                ready.append(arrivals.popleft())
            self._complete(t, ready)
            busy = {k for _, k, _, _ in self.inflight}
            free = [k for k in range(len(self.streams)) if k not in busy]
            if ready and free:
                batch, defer, ids = [], [], set()
                while ready and len(batch) < self.max_batch:
                    r = ready.popleft()
                    if r.system_id in ids:
                        defer.append(r)
                        continue
                    if not self._admit(r, t):
                        defer.append(r)          # budget full: wait for completions
                        break
                    self.resident[r.system_id].pending += 1
                    ids.add(r.system_id)
                    batch.append(r)
                ready.extendleft(reversed(defer))
                if batch:
                    self._launch(batch, free[0])
                    continue
            if self.inflight:
                if not arrivals or arrivals[0].arrival > now():
                    self.inflight[0][0].synchronize()
            elif arrivals:
                time.sleep(max(0.0, min(2e-3, arrivals[0].arrival - now())))
        wall = now()
        lat = np.array([r.finish - r.arrival for r in reqs])
        return {"systems": len(reqs), "wall_s": wall, "systems_per_s": len(reqs) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "batches": self.batches, "peak_bytes": self.peak_used}


def serve_plain(requests, n_samples=1, lr=1e-3, seed=0, precision=rtu.RTU_F32, device="cuda"):
    """The plain per-system path: each request alone, one call per system, in order."""
    t0 = time.perf_counter()
    lat = []
    for r in sorted(requests, key=lambda q: q.arrival):
        s = rtu.System.from_mock(r.mock, precision=precision, n_slots=n_samples, device=device)
        pr, ph, loc, rho = guide_start(r.mock)
        s.elbo_init(pr, ph, loc, rho, tag=r.system_id)
        out = torch.empty(1, dtype=torch.float64, device=device)
        for _ in range(r.n_steps):
            rtu.rtu_elbo_step([s], n_samples, seed, lr, out)
        r.elbo = float(out.cpu()[0])
        r.finish = time.perf_counter() - t0
        lat.append(r.finish - 0.0)
        s.close()
    wall = time.perf_counter() - t0
    return {"systems": len(requests), "wall_s": wall, "systems_per_s": len(requests) / wall}


def make_stream(n: int, rate_hz: float, seed: int = 5000):
    """The serving workload: n systems, Poisson arrivals, mixed sizes and profiles; each
    request carries its observation and its starting guide."""
    times = I.poisson_arrivals(n, rate_hz, seed)
    out = []
    for k in range(n):
        m = I.config_serving_system(seed + 1 + k)
        out.append(Request(rid=k, system_id=k, mock=m, arrival=float(times[k]), guide=start_guide(m)))
    return out
