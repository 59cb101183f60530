"""ctypes binding of the C ABI in ``include/rtu.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA kernels of ``librtu.so``; PyTorch
supplies device memory and streams.  Importing this module on a machine
without the built library raises immediately: there is no fallback.

Names follow the ABI: ``rtu_build_grid``, ``rtu_forward``, ``rtu_adjoint``
(and the batched ``Batch`` helper, the ``RTUForward`` autograd Function).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtu.so")

RTU_F32, RTU_F64 = 0, 1
RTU_SIE, RTU_EPL = 0, 1
RTU_SUB_NONE, RTU_SUB_NFW, RTU_SUB_TNFW = 0, 1, 2
RTU_PS_POWER_LAW, RTU_PS_MATERN_LIKE, RTU_PS_MATERN = 0, 1, 2
RTU_TRANSFORM_RTU, RTU_TRANSFORM_UNIFORM, RTU_TRANSFORM_LINEAR = 0, 1, 2
STAT_LOGL, STAT_CHI2, STAT_NMASK, STAT_FLAGS, STAT_N_IN_GRID = 0, 1, 2, 3, 4
W_NONMONOTONE, W_SELECT, W_TIMEOUT, W_RANGE = 1, 2, 4, 8
N_STATS = 5
SEL_BINS = 65536
N_PS = {RTU_PS_POWER_LAW: 2, RTU_PS_MATERN_LIKE: 2, RTU_PS_MATERN: 3}


class RTUError(RuntimeError):
    pass


if not os.path.exists(LIB_PATH):
    raise ImportError(f"librtu.so is not built at {LIB_PATH}: run `python -m paper_2606_30620_b300.build`"
                      " (the CUDA path has no fallback)")
_lib = ctypes.CDLL(LIB_PATH)


class SystemDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_img", "s_super", "n_src", "psf_k", "profile", "sub_kind", "n_sub", "ps_family",
        "precision", "n_nodes", "degree", "n_slots", "transform", "n_light")] + [
        ("pix", ctypes.c_double), ("src_pitch", ctypes.c_double), ("sigma", ctypes.c_double),
        ("data", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("psf", ctypes.c_void_p),
        ("weights", ctypes.c_void_p)]


class Eval(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int32), ("pad_", ctypes.c_int32)] + [(n, ctypes.c_void_p) for n in (
        "lens", "latents", "ps", "dlogL", "stats", "model", "image", "source", "cdf", "ray_hist",
        "g_latents", "g_lens", "g_ps", "light", "g_light", "sel_hist", "centres")]


class HostInputs(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_void_p), ("psf", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("upload_src", ctypes.c_void_p), ("upload_dst", ctypes.c_void_p), ("upload_bytes", ctypes.c_uint64)]


def pack_priors(priors):
    """The rtu_prior array of a sequence of (kind, space, a, b, c, d) rows, built from one
    packed record array of the same layout."""
    pv = np.asarray(priors, dtype=np.float64).reshape(-1, 6)
    rec = np.zeros(pv.shape[0], dtype=_PRIOR_DT)
    rec["kind"], rec["space"] = pv[:, 0].astype(np.int32), pv[:, 1].astype(np.int32)
    rec["a"], rec["b"], rec["c"], rec["d"] = pv[:, 2], pv[:, 3], pv[:, 4], pv[:, 5]
    return (Prior * pv.shape[0]).from_buffer_copy(rec.tobytes())


class Tuning(ctypes.Structure):
    _fields_ = [("adj_div", ctypes.c_int32), ("near_ctas", ctypes.c_int32), ("edge_ctas", ctypes.c_int32)]


class Prior(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("space", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double), ("d", ctypes.c_double)]


_PRIOR_DT = np.dtype([("kind", "<i4"), ("space", "<i4"), ("a", "<f8"), ("b", "<f8"), ("c", "<f8"), ("d", "<f8")],
                     align=True)
assert _PRIOR_DT.itemsize == ctypes.sizeof(Prior)


_lib.rtu_workspace_size.argtypes = [ctypes.POINTER(SystemDesc)]
_lib.rtu_workspace_size.restype = ctypes.c_size_t
_lib.rtu_system_create.argtypes = [ctypes.POINTER(SystemDesc), ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_void_p)]
_lib.rtu_system_create.restype = ctypes.c_int32
_lib.rtu_system_create_on.argtypes = [ctypes.POINTER(SystemDesc), ctypes.POINTER(HostInputs), ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
_lib.rtu_system_create_on.restype = ctypes.c_int32
_lib.rtu_system_tune.argtypes = [ctypes.c_void_p, ctypes.POINTER(Tuning)]
_lib.rtu_system_tune.restype = ctypes.c_int32
_lib.rtu_system_destroy.argtypes = [ctypes.c_void_p]
_lib.rtu_system_destroy.restype = ctypes.c_int32
for _name in ("rtu_build_grid", "rtu_forward", "rtu_adjoint"):
    getattr(_lib, _name).argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Eval), ctypes.c_int32,
                                     ctypes.c_void_p]
    getattr(_lib, _name).restype = ctypes.c_int32
_lib.rtu_n_sites.argtypes = [ctypes.POINTER(SystemDesc)]
_lib.rtu_n_sites.restype = ctypes.c_int32
_lib.rtu_elbo_init.argtypes = [ctypes.c_void_p, ctypes.POINTER(Prior), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_uint32]
_lib.rtu_elbo_init.restype = ctypes.c_int32
_lib.rtu_elbo_init_on.argtypes = [ctypes.c_void_p, ctypes.POINTER(Prior), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_uint32,
                                  ctypes.c_void_p]
_lib.rtu_elbo_init_on.restype = ctypes.c_int32
_lib.rtu_elbo_step.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
_lib.rtu_elbo_step.restype = ctypes.c_int32
_lib.rtu_elbo_state_bytes.argtypes = [ctypes.c_void_p]
_lib.rtu_elbo_state_bytes.restype = ctypes.c_size_t
_lib.rtu_elbo_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
_lib.rtu_elbo_export.restype = ctypes.c_int32
_lib.rtu_elbo_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
_lib.rtu_elbo_grad.restype = ctypes.c_int32
_lib.rtu_elbo_import.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
_lib.rtu_elbo_import.restype = ctypes.c_int32
_lib.rtu_gp_source_static.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.rtu_gp_source_static.restype = ctypes.c_int32
_lib.rtu_selftest_df.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
_lib.rtu_selftest_df.restype = ctypes.c_int32
_lib.rtu_graph_replay.argtypes = [ctypes.c_int32]
_lib.rtu_graph_replay.restype = ctypes.c_int32
_lib.rtu_profile_enable.argtypes = [ctypes.c_int32]
_lib.rtu_profile_enable.restype = ctypes.c_int32
_lib.rtu_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
_lib.rtu_profile_report.restype = ctypes.c_int32
_lib.rtu_profile_timeline.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
_lib.rtu_profile_timeline.restype = ctypes.c_int32
_lib.rtu_last_error.restype = ctypes.c_char_p
_lib.rtu_version.restype = ctypes.c_char_p

EXPORTED = ("rtu_workspace_size", "rtu_system_create", "rtu_system_create_on", "rtu_system_tune",
            "rtu_system_destroy",
            "rtu_build_grid", "rtu_forward", "rtu_adjoint", "rtu_n_sites", "rtu_elbo_init", "rtu_elbo_init_on",
            "rtu_elbo_step",
            "rtu_elbo_state_bytes", "rtu_elbo_export", "rtu_elbo_import", "rtu_elbo_grad", "rtu_gp_source_static",
            "rtu_selftest_df",
            "rtu_graph_replay", "rtu_profile_enable",
            "rtu_profile_report", "rtu_profile_timeline", "rtu_last_error", "rtu_version")


def _check(rc: int, what: str):
    if rc < 0:
        raise RTUError(f"{what} failed ({rc}): {_lib.rtu_last_error().decode()}")


def version() -> str:
    return _lib.rtu_version().decode()


def graph_replay(on: bool = True):
    """Replay of recorded launch sequences for repeated calls (on by default)."""
    _check(_lib.rtu_graph_replay(1 if on else 0), "rtu_graph_replay")


def profile_enable(on: bool = True):
    _check(_lib.rtu_profile_enable(1 if on else 0), "rtu_profile_enable")


def profile_report() -> dict:
    """{kernel: (launches, total_ms)} since the last report (waits for the events)."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.rtu_profile_report(buf, len(buf)), "rtu_profile_report")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def profile_timeline() -> list:
    """[(kernel, stream, start_ms, end_ms)] of the recorded launches in launch order,
    relative to the first one's start; stream 0 = the call's, 1 and 2 = the side streams."""
    buf = ctypes.create_string_buffer(1 << 20)
    _check(_lib.rtu_profile_timeline(buf, len(buf)), "rtu_profile_timeline")
    out = []
    for line in buf.value.decode().splitlines():
        name, side, a, b = line.split()
        out.append((name, int(side), float(a), float(b)))
    return out


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class System:
    """One lens system: the caller-owned observation tensors plus its workspace."""

    def __init__(self, data, mask, psf, sigma, pix, s_super, n_src, src_pitch, profile=RTU_SIE,
                 ps_family=RTU_PS_POWER_LAW, sub_kind=RTU_SUB_NONE, n_sub=0, precision=RTU_F32,
                 n_nodes=22, degree=21, n_slots=1, device="cuda", transform=RTU_TRANSFORM_RTU, n_light=0,
                 weights=None, stream=None, host_staging=None, tune=True, alloc=None):
        """stream=None: synchronous creation (rtu_system_create).  With a torch stream
        and host (numpy) data, mask and psf: the observation travels in one pinned
        copy and the library builds the system from the host copies with uploads
        ordered on that stream (rtu_system_create_on); calls ordered after the stream
        may use the system.  host_staging: a pinned uint8 tensor of at least
        staging_bytes(...) to stage that copy in (the caller keeps it untouched until
        the stream has passed the copy), else one is allocated.  tune: apply the
        autotuner's cached launch shape for this GPU and problem bucket, if any.
        alloc: a callable returning a uint8 CUDA tensor of at least the given number of
        bytes (a caller's pool) for the workspace and, on a stream, the observation's
        device copy, else torch allocates them; the blocks taken are in pool_blocks."""
        self.dtype = torch.float64 if precision == RTU_F64 else torch.float32
        self.device = torch.device(device)
        self.pool_blocks = []
        on_stream = stream is not None
        if on_stream:
            if not (isinstance(data, np.ndarray) and isinstance(psf, np.ndarray) and isinstance(mask, np.ndarray)):
                raise ValueError("creation on a stream takes host (numpy) data, mask and psf")
            npdt = np.float64 if precision == RTU_F64 else np.float32
            tb = np.dtype(npdt).itemsize
            nd, nk, nm = data.size, psf.size, mask.size
            nw = 0 if weights is None else nm
            total = System.staging_bytes(data.size, psf.size, precision, weights is not None)
            pad = 0
            host = (host_staging[:total] if host_staging is not None
                    else torch.empty(total, dtype=torch.uint8, pin_memory=True))
            hb = host.numpy()
            hdp = hb[:nd * tb].view(npdt)
            hdp[:] = np.asarray(data, npdt).ravel()
            hpsf = hb[nd * tb:(nd + nk) * tb].view(npdt)
            hpsf[:] = np.asarray(psf, npdt).ravel()
            hmask = hb[(nd + nk) * tb:(nd + nk) * tb + nm]
            hmask[:] = (np.asarray(mask).ravel() != 0)
            hw = None
            if weights is not None:
                hw = hb[(nd + nk) * tb + nm:(nd + nk) * tb + nm + 4 * nw].view(np.uint32)
                hw[:] = np.asarray(weights).astype(np.uint32).ravel()
            if alloc is not None:
                dev = alloc(total)
                self.pool_blocks.append(dev)
            else:
                dev = torch.empty(total, dtype=torch.uint8, device=self.device)
            dev = dev[:total]
            self._host = host          # kept until the system is closed (the copy reads it)
            self.data = dev[:nd * tb].view(self.dtype).view(data.shape)
            self.psf = dev[nd * tb:(nd + nk) * tb].view(self.dtype).view(psf.shape)
            self.mask = dev[(nd + nk) * tb:(nd + nk) * tb + nm].view(mask.shape)
            self.weights = None if hw is None else dev[(nd + nk) * tb + nm:(nd + nk) * tb + nm + 4 * nw].view(
                torch.int32)
            # the library copies the whole block up on the stream, before its own uploads
            self._host_in = HostInputs(hmask.ctypes.data, hpsf.ctypes.data, None if hw is None else hw.ctypes.data,
                                       host.data_ptr(), dev.data_ptr(), total)
        elif isinstance(data, np.ndarray) and isinstance(psf, np.ndarray):
            # host arrays: the image and the PSF travel in one copy
            npdt = np.float64 if precision == RTU_F64 else np.float32
            both = np.concatenate([np.asarray(data, npdt).ravel(), np.asarray(psf, npdt).ravel()])
            dev = torch.from_numpy(both).to(self.device)
            self.data = dev[:data.size].view(data.shape)
            self.psf = dev[data.size:].view(psf.shape)
        else:
            self.data = torch.as_tensor(data, dtype=self.dtype, device=self.device).contiguous()
            self.psf = torch.as_tensor(psf, dtype=self.dtype, device=self.device).contiguous()
        if not on_stream:
            self.mask = torch.as_tensor(mask, dtype=torch.uint8, device=self.device).contiguous()
            # weighted RTU grid: integer ray weights per pixel (read once at create)
            self.weights = None if weights is None else torch.as_tensor(
                weights.astype("int32") if hasattr(weights, "astype") else weights,
                dtype=torch.int32, device=self.device).contiguous()
        self.n_img = int(self.data.shape[0])
        self.n_src = int(n_src)
        self.s_super = int(s_super)
        self.profile = int(profile)
        self.ps_family = int(ps_family)
        self.sub_kind = int(sub_kind)
        self.n_sub = int(n_sub) if sub_kind else 0
        self.n_slots = int(n_slots)
        self.precision = int(precision)
        self.n_nodes = int(n_nodes)
        self.desc = SystemDesc(self.n_img, self.s_super, self.n_src, int(self.psf.shape[0]), self.profile,
                               self.sub_kind, self.n_sub, self.ps_family, self.precision, int(n_nodes),
                               int(degree), self.n_slots, int(transform), int(n_light), float(pix), float(src_pitch),
                               float(sigma),
                               self.data.data_ptr(), self.mask.data_ptr(), self.psf.data_ptr(),
                               None if self.weights is None else self.weights.data_ptr())
        nbytes = _lib.rtu_workspace_size(ctypes.byref(self.desc))
        if nbytes == 0:
            raise RTUError("invalid system description (rtu_workspace_size returned 0)")
        if alloc is not None:
            self.workspace = alloc(nbytes + 256)
            self.pool_blocks.append(self.workspace)
            wd = self.workspace.device
            same_dev = wd.type == self.device.type and (self.device.index is None or wd.index == self.device.index)
            if self.workspace.dtype != torch.uint8 or not same_dev or self.workspace.numel() < nbytes + 256:
                raise ValueError("alloc must return a uint8 tensor on the system's device of the bytes asked for")
        else:
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p()
        if on_stream:
            _check(_lib.rtu_system_create_on(ctypes.byref(self.desc), ctypes.byref(self._host_in),
                                             ctypes.c_void_p(base + off), nbytes, ctypes.c_void_p(stream.cuda_stream),
                                             ctypes.byref(h)), "rtu_system_create_on")
        else:
            _check(_lib.rtu_system_create(ctypes.byref(self.desc), ctypes.c_void_p(base + off), nbytes,
                                          ctypes.byref(h)), "rtu_system_create")
        self.handle = h
        self.n_lens = 8 + 5 * self.n_sub
        self.n_ps = N_PS[self.ps_family] + 1
        self.n_knots = self.n_nodes + 2
        self.n_light = int(n_light)
        self._n_mask = None
        self.tuning = None
        if tune:
            from . import autotune
            t = autotune.lookup(self.n_img, self.n_src, self.s_super, self.precision)
            if t is not None:
                self.tune(t)

    def tune(self, tuning: dict):
        """Launch shapes for later calls (rtu_system_tune): adj_div, near_ctas, edge_ctas."""
        t = Tuning(int(tuning["adj_div"]), int(tuning["near_ctas"]), int(tuning["edge_ctas"]))
        _check(_lib.rtu_system_tune(self.handle, ctypes.byref(t)), "rtu_system_tune")
        self.tuning = dict(tuning)

    @staticmethod
    def staging_bytes(n_pixels: int, n_psf: int, precision: int, weighted: bool) -> int:
        """Bytes of the pinned staging copy of an observation created on a stream: the
        image and PSF in the precision's type, the mask bytes and the weights, rounded up
        to 16."""
        tb = 8 if precision == RTU_F64 else 4
        total = (n_pixels + n_psf) * tb + n_pixels + (4 * n_pixels if weighted else 0)
        return total + (-total) % 16

    @property
    def n_mask(self) -> int:
        """Arc-mask pixels (the centre rays of the eCDFs); counted on first use."""
        if self._n_mask is None:
            self._n_mask = int(self.mask.count_nonzero())
        return self._n_mask

    @classmethod
    def from_mock(cls, m, precision=RTU_F32, n_slots=1, device="cuda", transform=RTU_TRANSFORM_RTU, stream=None,
                  host_staging=None, tune=True, alloc=None):
        return cls(m.data, m.mask, m.psf, m.sigma, m.pix, m.s_super, m.n_src, m.src_pitch, m.profile,
                   m.ps_family, m.sub_kind, 0 if m.subs is None else m.subs.shape[0], precision,
                   n_slots=n_slots, device=device, transform=transform,
                   n_light=0 if getattr(m, "light", None) is None else m.light.shape[0],
                   weights=getattr(m, "weights", None), stream=stream, host_staging=host_staging, tune=tune,
                   alloc=alloc)

    @property
    def n_sites(self) -> int:
        return int(_lib.rtu_n_sites(ctypes.byref(self.desc)))

    def elbo_init(self, priors, fixed, loc, rho, tag: int, stream=None):
        """Set the guide: priors[n_sites] as (kind, space, a, b, c, d), the physical
        values of the non-site entries, loc/rho over n_sites + n_src^2, random-stream
        tag.  stream=None: synchronous (rtu_elbo_init); else the upload is ordered on
        that torch stream (rtu_elbo_init_on)."""
        ns = self.n_sites
        if len(priors) != ns:
            raise ValueError(f"{ns} priors expected")
        arr = priors if isinstance(priors, ctypes.Array) and priors._type_ is Prior else pack_priors(priors)
        fixed = np.ascontiguousarray(fixed, dtype=np.float64)
        loc = np.ascontiguousarray(loc, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        if fixed.size != self.n_lens + self.n_ps + 6 * self.n_light or loc.size != ns + self.n_src ** 2 \
                or rho.size != loc.size:
            raise ValueError("fixed / loc / rho sizes do not match the system")
        dp = ctypes.POINTER(ctypes.c_double)
        if stream is None:
            _check(_lib.rtu_elbo_init(self.handle, arr, fixed.ctypes.data_as(dp), loc.ctypes.data_as(dp),
                                      rho.ctypes.data_as(dp), int(tag) & 0xFFFFFFFF), "rtu_elbo_init")
        else:
            _check(_lib.rtu_elbo_init_on(self.handle, arr, fixed.ctypes.data_as(dp), loc.ctypes.data_as(dp),
                                         rho.ctypes.data_as(dp), int(tag) & 0xFFFFFFFF,
                                         ctypes.c_void_p(stream.cuda_stream)), "rtu_elbo_init_on")

    def elbo_export(self) -> bytes:
        n = _lib.rtu_elbo_state_bytes(self.handle)
        buf = ctypes.create_string_buffer(n)
        _check(_lib.rtu_elbo_export(self.handle, buf, n), "rtu_elbo_export")
        return buf.raw

    def elbo_import(self, blob: bytes):
        _check(_lib.rtu_elbo_import(self.handle, blob, len(blob)), "rtu_elbo_import")

    def elbo_grad(self):
        """(d ELBO / d loc, d ELBO / d rho) of the last rtu_elbo_step, before Adam
        (numpy arrays; a synchronous copy)."""
        n = self.n_sites + self.n_src ** 2
        out = np.zeros(2 * n, dtype=np.float64)
        _check(_lib.rtu_elbo_grad(self.handle, out.ctypes.data, out.nbytes), "rtu_elbo_grad")
        return out[:n].copy(), out[n:].copy()

    def elbo_state(self):
        """(loc, rho, step) of the guide as numpy arrays (a synchronous copy)."""
        raw = np.frombuffer(self.elbo_export(), dtype=np.float64)
        n = self.n_sites + self.n_src ** 2
        return raw[:n].copy(), raw[n:2 * n].copy(), int(np.frombuffer(raw[6 * n:6 * n + 1].tobytes(), np.int64)[0])

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.rtu_system_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Binding:
    """Device buffers of one evaluation (inputs, and outputs allocated on demand)."""

    def __init__(self, system: System, lens, latents, ps, slot=0, want_model=False, want_image=False,
                 want_source=False, want_cdf=False, want_hist=False, grads=True, dlogL=None, out=None,
                 light=None, want_selection=False):
        dev, dt = system.device, system.dtype
        self.system = system
        self.slot = slot
        self.lens = torch.as_tensor(lens, dtype=torch.float64, device=dev).contiguous().reshape(-1)
        self.latents = torch.as_tensor(latents, dtype=dt, device=dev).contiguous()
        self.ps = torch.as_tensor(ps, dtype=torch.float64, device=dev).contiguous()
        if self.lens.numel() != system.n_lens:
            raise ValueError(f"lens must hold {system.n_lens} values")
        if self.latents.numel() != system.n_src ** 2:
            raise ValueError("latents must hold n_src^2 values")
        if self.ps.numel() != system.n_ps:
            raise ValueError(f"ps must hold {system.n_ps} values")
        self.light = None
        if system.n_light > 0:
            if light is None:
                raise ValueError("this system has lens light: pass light [n_light, 6]")
            self.light = torch.as_tensor(light, dtype=torch.float64, device=dev).contiguous().reshape(-1)
            if self.light.numel() != 6 * system.n_light:
                raise ValueError(f"light must hold {6 * system.n_light} values")
        self.dlogL = None if dlogL is None else torch.as_tensor(dlogL, dtype=torch.float64, device=dev)
        out = out or {}
        self.stats = out["stats"] if "stats" in out else torch.zeros(N_STATS, dtype=torch.float64, device=dev)
        n_img, n_src = system.n_img, system.n_src
        self.model = torch.empty(n_img, n_img, dtype=dt, device=dev) if want_model else None
        self.image = torch.empty(n_img, n_img, dtype=dt, device=dev) if want_image else None
        self.source = torch.empty(n_src, n_src, dtype=dt, device=dev) if want_source else None
        self.cdf = torch.empty(3 + 4 * system.n_knots, dtype=torch.float64, device=dev) if want_cdf else None
        self.ray_hist = torch.empty((n_src - 1) ** 2, dtype=torch.int32, device=dev) if want_hist else None
        # the order statistics' integer histograms and the traced centre rays (build outputs)
        self.sel_hist = torch.empty(2, SEL_BINS, dtype=torch.int32, device=dev) if want_selection else None
        self.centres = (torch.empty(2, system.n_mask, dtype=torch.float64, device=dev)
                        if want_selection else None)
        if grads:
            # caller-provided output views (e.g. slices of one packed buffer) are used as they are
            self.g_latents = out.get("g_latents", None)
            if self.g_latents is None:
                self.g_latents = torch.empty(n_src, n_src, dtype=dt, device=dev)
            self.g_lens = out.get("g_lens", None)
            if self.g_lens is None:
                self.g_lens = torch.empty(system.n_lens, dtype=torch.float64, device=dev)
            self.g_ps = out.get("g_ps", None)
            if self.g_ps is None:
                self.g_ps = torch.empty(system.n_ps, dtype=torch.float64, device=dev)
            for t in (self.g_latents, self.g_lens, self.g_ps):
                if not t.is_contiguous():
                    raise ValueError("output views must be contiguous")
            self.g_light = (torch.empty(6 * system.n_light, dtype=torch.float64, device=dev)
                            if system.n_light > 0 else None)
        else:
            self.g_latents = self.g_lens = self.g_ps = self.g_light = None

    def as_struct(self) -> Eval:
        return Eval(self.slot, 0, *[None if t is None else t.data_ptr() for t in (
            self.lens, self.latents, self.ps, self.dlogL, self.stats, self.model, self.image, self.source,
            self.cdf, self.ray_hist, self.g_latents, self.g_lens, self.g_ps, self.light, self.g_light,
            self.sel_hist, self.centres)])


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _arrays(bindings):
    n = len(bindings)
    sys_arr = (ctypes.c_void_p * n)(*[b.system.handle.value for b in bindings])
    ev_arr = (Eval * n)(*[b.as_struct() for b in bindings])
    return sys_arr, ev_arr, n


class Batch:
    """Pre-marshalled argument arrays for repeated calls over the same bindings."""

    def __init__(self, bindings):
        self.bindings = list(bindings)
        self.sys_arr, self.ev_arr, self.n = _arrays(self.bindings)

    def build_grid(self, stream=None):
        _check(_lib.rtu_build_grid(self.sys_arr, self.ev_arr, self.n, _stream_ptr(stream)), "rtu_build_grid")

    def forward(self, stream=None):
        _check(_lib.rtu_forward(self.sys_arr, self.ev_arr, self.n, _stream_ptr(stream)), "rtu_forward")

    def adjoint(self, stream=None):
        _check(_lib.rtu_adjoint(self.sys_arr, self.ev_arr, self.n, _stream_ptr(stream)), "rtu_adjoint")


def rtu_build_grid(bindings, stream=None):
    Batch(bindings).build_grid(stream)


def rtu_forward(bindings, stream=None):
    Batch(bindings).forward(stream)


def rtu_adjoint(bindings, stream=None):
    Batch(bindings).adjoint(stream)


def rtu_elbo_step(systems, n_samples: int, seed: int, lr: float, elbo_out=None, stream=None):
    """One SVI step for each system (batched); elbo_out: device float64 [len(systems)]."""
    n = len(systems)
    arr = (ctypes.c_void_p * n)(*[s.handle.value for s in systems])
    out = None if elbo_out is None else ctypes.c_void_p(elbo_out.data_ptr())
    _check(_lib.rtu_elbo_step(arr, n, int(n_samples), int(seed) & 0xFFFFFFFFFFFFFFFF, float(lr), out,
                              _stream_ptr(stream)), "rtu_elbo_step")


DF_OPS = {"exp": 0, "log": 1, "sqrt": 2, "div": 3, "mul": 4, "add": 5, "floor": 6, "edge_dist": 7, "fix_pair": 8}
DF_BINARY = (3, 4, 5, 8)


def rtu_selftest_df(op: str, x):
    """The double-float arithmetic of the FP32 path's islands on the device: x a float64
    CUDA tensor ([n] for exp / log / sqrt / floor / edge_dist, [n, 2] for div / mul / add /
    fix_pair); returns [n]."""
    code = DF_OPS[op]
    x = x.contiguous()
    n = x.shape[0]
    binary = code in DF_BINARY
    if x.dtype != torch.float64 or not x.is_cuda or (binary and tuple(x.shape) != (n, 2)) or \
            (not binary and x.dim() != 1):
        raise ValueError("x must be a float64 CUDA tensor of shape [n] or [n, 2]")
    y = torch.empty(n, dtype=torch.float64, device=x.device)
    _check(_lib.rtu_selftest_df(code, x.data_ptr(), y.data_ptr(), n, _stream_ptr(None)), "rtu_selftest_df")
    return y


STATIC_MAX_NSRC = 128


def rtu_gp_source_static(n_src: int, src_pitch: float, ps_family: int, latents, ps, source, stream=None):
    """GP source without a workspace (the latents filtered by sqrt(P) through FFTs, then
    the softplus map and the alpha_src power): latents / source are float32 CUDA tensors
    of n_src^2 elements, ps a float64 CUDA tensor of the family's parameters and
    alpha_src, all on the current device.  Allocates no device memory; calls share one
    static scratch array, so do not overlap them on the GPU."""
    for t, dt in ((latents, torch.float32), (source, torch.float32), (ps, torch.float64)):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError("latents/source must be contiguous float32 CUDA tensors, ps float64")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("latents, ps and source must be on the current CUDA device")
    if ps_family not in N_PS:
        raise ValueError("unknown ps_family")
    if latents.numel() != n_src * n_src or source.numel() != n_src * n_src:
        raise ValueError(f"latents and source must hold n_src^2 = {n_src * n_src} values")
    if ps.numel() != N_PS[ps_family] + 1:
        raise ValueError(f"ps must hold {N_PS[ps_family] + 1} values (the family's parameters, alpha_src)")
    _check(_lib.rtu_gp_source_static(int(n_src), float(src_pitch), int(ps_family), latents.data_ptr(),
                                     ps.data_ptr(), source.data_ptr(), _stream_ptr(stream)),
           "rtu_gp_source_static")


class RTUForward(torch.autograd.Function):
    """log L(lens, latents, ps[, light]) of one system; backward runs rtu_adjoint,
    which recomputes the rays instead of saving them.  The adjoint reads what the
    forward left in the system's workspace slot, so when another forward on the same
    system ran in between (two forwards, then their backwards), backward first runs
    its own forward again."""

    @staticmethod
    def forward(ctx, system: System, lens, latents, ps, light=None):
        b = Binding(system, lens.detach(), latents.detach(), ps.detach(), grads=True,
                    dlogL=torch.ones(1, dtype=torch.float64, device=system.device),
                    light=None if light is None else light.detach())
        Batch([b]).forward()
        ctx.binding = b
        ctx.token = object()
        system._slot0_owner = ctx.token
        ctx.light_shape = None if light is None else light.shape
        return b.stats[STAT_LOGL].clone()

    @staticmethod
    def backward(ctx, g):
        b = ctx.binding
        if getattr(b.system, "_slot0_owner", None) is not ctx.token:
            Batch([b]).forward()            # the slot holds another forward's state
            b.system._slot0_owner = ctx.token
        b.dlogL.copy_(g.reshape(1).to(torch.float64))
        Batch([b]).adjoint()
        g_light = None if ctx.light_shape is None else b.g_light.clone().reshape(ctx.light_shape)
        return None, b.g_lens.clone(), b.g_latents.clone(), b.g_ps.clone(), g_light


def log_likelihood(system: System, lens, latents, ps, light=None):
    return RTUForward.apply(system, lens, latents, ps, light)
