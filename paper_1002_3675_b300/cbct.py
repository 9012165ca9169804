"""Thin Python binding of the C ABI in ``include/cbct.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Tensors are torch CUDA
float32 tensors in the ABI's layouts (volumes [nz][ny][nx], sinograms
[n_angles][nv][nu]); work is enqueued on torch's current CUDA stream.  A non-OK
status raises ``CbctError`` carrying ``cbct_last_error()``.  There is no fallback:
if the shared library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cbct.h")

NUM_KERNEL_CLASSES = 5
KERNEL_CLASSES = ("project", "backproject", "tv", "reduce", "transfer")
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "UNSUPPORTED", 6: "BUSY"}


class CbctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cbct status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class GeometryDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int), ("du", C.c_double), ("dv", C.c_double),
                ("dso", C.c_double), ("dsd", C.c_double)]


class Options(C.Structure):
    _fields_ = [("beta", C.c_double), ("betas", C.POINTER(C.c_double)), ("eps", C.c_double),
                ("inner_iters", C.c_int), ("clamp_mode", C.c_int), ("sino_fp16", C.c_int),
                ("power_iters", C.c_int), ("start_level", C.c_int), ("f_init_dev", C.c_void_p),
                ("use_graphs", C.c_int), ("energy_trace", C.POINTER(C.c_double)),
                ("beta_out", C.POINTER(C.c_double)), ("kernel_ms", C.POINTER(C.c_float)),
                ("kernel_launches", C.POINTER(C.c_int)), ("kernel_mask", C.c_uint), ("reuse_lambda", C.c_int),
                ("tv_mode", C.c_int),
                ("adjoint_mode", C.c_int), ("mg_cycle", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int),
                ("mg_coarse", C.c_int), ("mg_accepted", C.POINTER(C.c_int)),
                ("step_trace", C.POINTER(C.c_double)), ("serial_power", C.c_int),
                ("kernel_ms_finest", C.POINTER(C.c_float)), ("kernel_launches_finest", C.POINTER(C.c_int)),
                ("level_ms", C.POINTER(C.c_float))]


class Request(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("Y_dev", C.c_void_p), ("mu", C.c_double), ("iters", C.c_int),
                ("levels", C.c_int), ("opts", C.POINTER(Options)), ("f_out_dev", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("proj_threads", C.c_int), ("bp_vpl", C.c_int), ("bp_threads", C.c_int),
                ("proj_ms", C.c_float), ("bp_ms", C.c_float), ("proj_smem", C.c_int), ("proj_levels", C.c_int),
                ("bp_layout", C.c_int), ("tv_sweeps", C.c_int), ("tv_warps", C.c_int), ("tv_planes", C.c_int)]


class ServerRequest(C.Structure):
    _fields_ = [("desc", GeometryDesc), ("angles_host", C.POINTER(C.c_double)), ("n_angles", C.c_int),
                ("Y_dev", C.c_void_p), ("mu", C.c_double), ("iters", C.c_int), ("levels", C.c_int),
                ("opts", Options), ("f_out_dev", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("latency_s", C.c_double), ("queue_s", C.c_double),
                ("betas", C.c_double * 8)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("slots_in_use", C.c_int),
                ("completed", C.c_uint64), ("hbm_in_use", C.c_size_t), ("busy_s", C.c_double)]


def _load() -> C.CDLL:
    # CBCT_LIBRARY: an explicitly chosen build of the library (e.g. one with other
    # launch shapes); otherwise the in-tree build, compiled if missing or stale
    path = os.environ.get("CBCT_LIBRARY") or _build.build()
    return C.CDLL(path)


lib = _load()
_P, _D, _I, _V = C.c_void_p, C.c_double, C.c_int, C.c_void_p
_SIGS = {
    "cbct_geometry_create": [C.POINTER(GeometryDesc), C.POINTER(C.c_double), _I, C.POINTER(C.c_void_p)],
    "cbct_geometry_destroy": [_P],
    "cbct_level_dims": [_P, _I, C.POINTER(C.c_int)],
    "cbct_project": [_P, _P, _P, _V],
    "cbct_backproject": [_P, _P, _P, _V],
    "cbct_backproject_eq2": [_P, _P, _P, _V],
    "cbct_tv_prox": [_P, _P, _P, _D, _D, _I, _I, _V],
    "cbct_fbs": [_P, _P, _D, _D, _D, _I, _I, _I, _I, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), _V],
    "cbct_power_iteration": [_P, _I, C.POINTER(C.c_double), _V],
    "cbct_energy": [_P, _P, _P, _D, _D, _I, C.POINTER(C.c_double), _V],
    "cbct_reconstruct": [_P, _P, C.POINTER(C.c_double), _I, _D, _I, _I, C.POINTER(Options), _P, _V],
    "cbct_restrict_sino": [_I, _I, _I, _P, _P, _V],
    "cbct_prolong_vol": [_I, _I, _I, _P, _I, _I, _I, _P, _V],
    "cbct_tv_energy_noalloc": [_I, _I, _I, _D, _D, _D, _D, _P, _P, _V],
    "cbct_reconstruct_batch": [C.POINTER(Request), _I, _I, _V],
    "cbct_autotune": [_P, _I, C.POINTER(Tuning), _V],
    "cbct_set_tuning": [_P, _I, C.POINTER(Tuning)],
    "cbct_server_create": [C.c_size_t, _I, _I, C.POINTER(C.c_void_p)],
    "cbct_server_submit": [_P, C.POINTER(ServerRequest), C.POINTER(C.c_uint64)],
    "cbct_server_wait": [_P, C.c_uint64, _I, C.POINTER(Result)],
    "cbct_server_cancel": [_P, C.c_uint64],
    "cbct_server_get_stats": [_P, C.POINTER(ServerStats)],
    "cbct_server_destroy": [_P],
    "cbct_debug_fail_next_allocations": [_I],
    "cbct_last_error": [],
    "cbct_version": [],
    "cbct_kernel_launch_count": [],
}
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = C.c_char_p if _name in ("cbct_last_error", "cbct_version") else (
        None if _name in ("cbct_geometry_destroy", "cbct_server_destroy", "cbct_debug_fail_next_allocations")
        else C.c_ulonglong if _name == "cbct_kernel_launch_count" else C.c_int)


def header_functions(path: str = HEADER):
    """Names of the functions declared in the C header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbct_[a-z0-9_]+)\s*\(", text)))


def cbct_last_error() -> str:
    return lib.cbct_last_error().decode()


def cbct_version() -> str:
    return lib.cbct_version().decode()


def cbct_kernel_launch_count() -> int:
    """Kernels launched through the library by this process so far."""
    return int(lib.cbct_kernel_launch_count())


def _check(status: int):
    if status != 0:
        raise CbctError(status, cbct_last_error())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Geometry:
    """Owning wrapper of a ``cbct_geometry`` handle."""

    def __init__(self, handle, desc: GeometryDesc, angles: np.ndarray):
        self.handle = handle
        self.desc = desc
        self.angles = angles

    @property
    def vol_shape(self):
        return (self.desc.nz, self.desc.ny, self.desc.nx)

    @property
    def sino_shape(self):
        return (len(self.angles), self.desc.nv, self.desc.nu)

    def close(self):
        if self.handle:
            lib.cbct_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(geom: dict) -> GeometryDesc:
    return GeometryDesc(geom["nx"], geom["ny"], geom["nz"], geom["hx"], geom["hy"], geom["hz"],
                        geom["nu"], geom["nv"], geom["du"], geom["dv"], geom["dso"], geom["dsd"])


def cbct_geometry_create(geom: dict) -> Geometry:
    desc = make_desc(geom)
    ang = np.ascontiguousarray(geom["angles"], dtype=np.float64)
    h = C.c_void_p()
    _check(lib.cbct_geometry_create(C.byref(desc), ang.ctypes.data_as(C.POINTER(C.c_double)), len(ang),
                                    C.byref(h)))
    return Geometry(h, desc, ang)


def cbct_level_dims(g: Geometry, level: int):
    out = (C.c_int * 5)()
    _check(lib.cbct_level_dims(g.handle, level, out))
    return tuple(out)


def _empty(shape, like=None):
    import torch
    return torch.empty(shape, dtype=torch.float32, device="cuda")


def cbct_project(g: Geometry, f, y=None):
    y = _empty(g.sino_shape) if y is None else y
    _check(lib.cbct_project(g.handle, _ptr(f, "f"), _ptr(y, "y"), _stream()))
    return y


def cbct_backproject(g: Geometry, y, f=None):
    f = _empty(g.vol_shape) if f is None else f
    _check(lib.cbct_backproject(g.handle, _ptr(y, "y"), _ptr(f, "f"), _stream()))
    return f


def cbct_backproject_eq2(g: Geometry, y, f=None):
    f = _empty(g.vol_shape) if f is None else f
    _check(lib.cbct_backproject_eq2(g.handle, _ptr(y, "y"), _ptr(f, "f"), _stream()))
    return f


def cbct_tv_prox(g: Geometry, gvol, f, beta: float, eps: float, inner_iters: int, tv_mode: int = 0):
    _check(lib.cbct_tv_prox(g.handle, _ptr(gvol, "g"), _ptr(f, "f"), beta, eps, inner_iters, tv_mode, _stream()))
    return f


def cbct_fbs(g: Geometry, Y, mu, beta, eps, inner_iters, clamp_mode, iters, f, trace=False, tv_mode=0,
             step_trace=False):
    """Returns f, or (f, trace [iters][3]) with trace=True, or (f, trace, steps [iters])
    with step_trace=True as well (steps alone: (f, steps))."""
    tr = np.zeros((max(iters, 1), 3)) if trace else None
    st = np.zeros(max(iters, 1)) if step_trace else None
    _check(lib.cbct_fbs(g.handle, _ptr(Y, "Y"), mu, beta, eps, inner_iters, clamp_mode, tv_mode, iters,
                        _ptr(f, "f"), tr.ctypes.data_as(C.POINTER(C.c_double)) if trace else None,
                        st.ctypes.data_as(C.POINTER(C.c_double)) if step_trace else None, _stream()))
    out = (f,) + ((tr[:iters],) if trace else ()) + ((st[:iters],) if step_trace else ())
    return out if len(out) > 1 else f


def cbct_power_iteration(g: Geometry, iters: int = 30) -> float:
    lam = C.c_double()
    _check(lib.cbct_power_iteration(g.handle, iters, C.byref(lam), _stream()))
    return lam.value


def cbct_energy(g: Geometry, Y, f, mu, eps, tv_mode=0):
    out = (C.c_double * 3)()
    _check(lib.cbct_energy(g.handle, _ptr(Y, "Y"), _ptr(f, "f"), mu, eps, tv_mode, out, _stream()))
    return np.array(out[:])


def make_options(levels, *, beta=0.0, betas=None, eps=0.0, inner_iters=0, clamp_mode=0, sino_fp16=False,
                 power_iters=0, f_init=None, start_level=0, use_graphs=False, reuse_lambda=False, tv_mode=0,
                 adjoint_mode=0, mg_cycle=0, mg_pre=0, mg_post=0, mg_coarse=0, keep=None):
    """cbct_options from keyword arguments; `keep` (a list) holds arrays the struct points to."""
    o = Options()
    o.beta = beta
    if betas is not None:
        bet = np.ascontiguousarray(betas, dtype=np.float64)
        if keep is not None:
            keep.append(bet)
        o.betas = bet.ctypes.data_as(C.POINTER(C.c_double))
    o.eps = eps
    o.inner_iters = inner_iters
    o.clamp_mode = clamp_mode
    o.sino_fp16 = int(bool(sino_fp16))
    o.power_iters = power_iters
    o.start_level = start_level
    o.f_init_dev = _ptr(f_init, "f_init") if f_init is not None else None
    o.use_graphs = int(bool(use_graphs))
    o.reuse_lambda = int(bool(reuse_lambda))
    o.tv_mode = int(tv_mode)
    o.adjoint_mode = int(adjoint_mode)
    o.mg_cycle, o.mg_pre, o.mg_post, o.mg_coarse = int(mg_cycle), int(mg_pre), int(mg_post), int(mg_coarse)
    return o


def cbct_reconstruct(g: Geometry, Y, mu: float, iters: int, levels: int, f_out=None, *, beta=0.0,
                     betas=None, eps=0.0, inner_iters=0, clamp_mode=0, sino_fp16=False, power_iters=0,
                     f_init=None, start_level=0, use_graphs=False, trace=False, kernel_times=False,
                     reuse_lambda=False, tv_mode=0, adjoint_mode=0, mg_cycle=0, mg_pre=0, mg_post=0, mg_coarse=0,
                     kernel_mask=0, serial_power=False, level_times=False):
    """Returns f_out, or (f_out, info) when trace/kernel_times is requested; info holds
    'trace' [levels][iters][3] ([iters][3] after each V-cycle when mg_cycle=1),
    'step_trace' [levels][iters] |f_k+1 - f_k| ([iters], the change over each V-cycle),
    'betas' [levels], 'accepted' [levels] (V-cycles), 'kernel_ms'/'kernel_launches' and
    'kernel_ms_finest'/'kernel_launches_finest' (the finest level's A1 iterations), and
    with level_times=True 'level_ms' [levels] (index 0 finest: each level's A1 iterations
    timed by one event pair, without per-launch events)."""
    f_out = _empty(g.vol_shape) if f_out is None else f_out
    o = Options()
    o.beta = beta
    bet = np.ascontiguousarray(betas, dtype=np.float64) if betas is not None else None
    if bet is not None:
        o.betas = bet.ctypes.data_as(C.POINTER(C.c_double))
    o.eps = eps
    o.inner_iters = inner_iters
    o.clamp_mode = clamp_mode
    o.sino_fp16 = int(bool(sino_fp16))
    o.power_iters = power_iters
    o.start_level = start_level
    o.f_init_dev = _ptr(f_init, "f_init") if f_init is not None else None
    o.use_graphs = int(bool(use_graphs))
    o.reuse_lambda = int(bool(reuse_lambda))
    o.tv_mode = int(tv_mode)
    o.adjoint_mode = int(adjoint_mode)
    o.mg_cycle, o.mg_pre, o.mg_post, o.mg_coarse = int(mg_cycle), int(mg_pre), int(mg_post), int(mg_coarse)
    o.serial_power = int(bool(serial_power))
    acc = (C.c_int * 8)()
    o.mg_accepted = acc
    tr = np.full((levels, max(iters, 1), 3), np.nan) if trace else None
    if trace:
        o.energy_trace = tr.ctypes.data_as(C.POINTER(C.c_double))
        sp = np.full((levels, max(iters, 1)), np.nan)
        o.step_trace = sp.ctypes.data_as(C.POINTER(C.c_double))
    bo = np.zeros(levels)
    o.beta_out = bo.ctypes.data_as(C.POINTER(C.c_double))
    km = (C.c_float * NUM_KERNEL_CLASSES)() if kernel_times else None
    kl = (C.c_int * NUM_KERNEL_CLASSES)() if kernel_times else None
    kmf = (C.c_float * NUM_KERNEL_CLASSES)() if kernel_times else None
    klf = (C.c_int * NUM_KERNEL_CLASSES)() if kernel_times else None
    if kernel_times:
        o.kernel_ms = km
        o.kernel_launches = kl
        o.kernel_ms_finest = kmf
        o.kernel_launches_finest = klf
        o.kernel_mask = int(kernel_mask)
    lm = (C.c_float * levels)() if level_times else None
    if level_times:
        o.level_ms = lm
    _check(lib.cbct_reconstruct(g.handle, _ptr(Y, "Y"), g.angles.ctypes.data_as(C.POINTER(C.c_double)),
                                len(g.angles), mu, iters, levels, C.byref(o), _ptr(f_out, "f_out"), _stream()))
    if not (trace or kernel_times or level_times):
        return f_out
    info = {"betas": bo}
    if level_times:
        info["level_ms"] = list(lm)
    if mg_cycle:
        info["accepted"] = np.array(acc[:levels])
    if trace:
        info["trace"] = tr.reshape(-1, 3)[:iters] if mg_cycle else tr[:, :iters]
        info["step_trace"] = sp.reshape(-1)[:iters] if mg_cycle else sp[:, :iters]
    if kernel_times:
        info["kernel_ms"] = dict(zip(KERNEL_CLASSES, list(km)))
        info["kernel_launches"] = dict(zip(KERNEL_CLASSES, list(kl)))
        info["kernel_ms_finest"] = dict(zip(KERNEL_CLASSES, list(kmf)))
        info["kernel_launches_finest"] = dict(zip(KERNEL_CLASSES, list(klf)))
    return f_out, info


def cbct_reconstruct_batch(requests, use_graphs=False):
    """requests: list of dicts with keys geom (Geometry), Y, mu, iters, levels, f_out
    (optional) and any cbct_reconstruct keyword (betas, beta, inner_iters, ...),
    plus trace=True to get the energy trace.  Returns (volumes, infos)."""
    keep, reqs, outs, infos = [], [], [], []
    for r in requests:
        g = r["geom"]
        levels = r["levels"]
        kw = {k: v for k, v in r.items() if k in ("beta", "betas", "eps", "inner_iters", "clamp_mode", "sino_fp16",
                                                  "power_iters", "f_init", "start_level", "reuse_lambda", "tv_mode", "adjoint_mode",
                                                  "mg_cycle", "mg_pre", "mg_post", "mg_coarse")}
        o = make_options(levels, keep=keep, **kw)
        info = {"betas": np.zeros(levels)}
        o.beta_out = info["betas"].ctypes.data_as(C.POINTER(C.c_double))
        if r.get("trace"):
            info["trace"] = np.full((levels, max(r["iters"], 1), 3), np.nan)
            o.energy_trace = info["trace"].ctypes.data_as(C.POINTER(C.c_double))
            info["step_trace"] = np.full((levels, max(r["iters"], 1)), np.nan)
            o.step_trace = info["step_trace"].ctypes.data_as(C.POINTER(C.c_double))
        keep.append(o)
        f = r.get("f_out")
        f = _empty(g.vol_shape) if f is None else f
        outs.append(f)
        infos.append(info)
        reqs.append(Request(g.handle, _ptr(r["Y"], "Y"), r["mu"], r["iters"], levels, C.pointer(o), _ptr(f, "f_out")))
    arr = (Request * len(reqs))(*reqs)
    _check(lib.cbct_reconstruct_batch(arr, len(reqs), int(bool(use_graphs)), _stream()))
    for info, r in zip(infos, requests):
        if "trace" in info:
            info["trace"] = info["trace"][:, :r["iters"]]
            info["step_trace"] = info["step_trace"][:, :r["iters"]]
    return outs, infos


def cbct_autotune(g: Geometry, level: int = 0) -> dict:
    t = Tuning()
    _check(lib.cbct_autotune(g.handle, level, C.byref(t), _stream()))
    return dict(proj_threads=t.proj_threads, proj_smem=t.proj_smem, bp_vpl=t.bp_vpl, bp_threads=t.bp_threads,
                proj_ms=t.proj_ms, bp_ms=t.bp_ms, proj_levels=t.proj_levels, bp_layout=t.bp_layout,
                tv_sweeps=t.tv_sweeps, tv_warps=t.tv_warps, tv_planes=t.tv_planes)


def cbct_set_tuning(g: Geometry, level: int, tuning: dict):
    t = Tuning(int(tuning.get("proj_threads", 0)), int(tuning.get("bp_vpl", 0)), int(tuning.get("bp_threads", 0)),
               0.0, 0.0, int(tuning.get("proj_smem", 0)), int(tuning.get("proj_levels", 0)),
               int(tuning.get("bp_layout", 0)), int(tuning.get("tv_sweeps", 0)), int(tuning.get("tv_warps", 0)),
               int(tuning.get("tv_planes", 0)))
    _check(lib.cbct_set_tuning(g.handle, level, C.byref(t)))


class Server:
    """Owning wrapper of cbct_server (continuous-batching reconstruction server)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, use_graphs: bool = False):
        h = C.c_void_p()
        _check(lib.cbct_server_create(int(hbm_budget_bytes), max_slots, int(bool(use_graphs)), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, geom: dict, Y, mu, iters, levels, f_out, **kw) -> int:
        keep = []
        o = make_options(levels, keep=keep, **kw)
        ang = np.ascontiguousarray(geom["angles"], dtype=np.float64)
        keep.append(ang)
        req = ServerRequest(make_desc(geom), ang.ctypes.data_as(C.POINTER(C.c_double)), len(ang), _ptr(Y, "Y"),
                            mu, iters, levels, o, _ptr(f_out, "f_out"))
        t = C.c_uint64()
        _check(lib.cbct_server_submit(self.handle, C.byref(req), C.byref(t)))
        self._keep[t.value] = (keep, Y, f_out)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = Result()
        st = lib.cbct_server_wait(self.handle, ticket, timeout_ms, C.byref(r))
        if st == 4:  # timeout: the ticket stays valid
            raise CbctError(st, cbct_last_error())
        self._keep.pop(ticket, None)
        out = dict(status=r.status, latency_s=r.latency_s, queue_s=r.queue_s, betas=list(r.betas))
        if st != 0:
            raise CbctError(st, f"request failed: {out}")
        return out

    def cancel(self, ticket: int):
        _check(lib.cbct_server_cancel(self.handle, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib.cbct_server_get_stats(self.handle, C.byref(s)))
        return dict(queued=s.queued, running=s.running, slots_in_use=s.slots_in_use, completed=s.completed,
                    hbm_in_use=s.hbm_in_use, busy_s=s.busy_s)

    def close(self):
        if self.handle:
            lib.cbct_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cbct_debug_fail_next_allocations(n: int):
    lib.cbct_debug_fail_next_allocations(n)


def cbct_tv_energy_noalloc(f, h, eps, out=None):
    """E1 = TV_eps(f) / Nv into a one-element float64 CUDA tensor, through the entry
    point that allocates nothing inside the library (for callers that cannot call
    cudaMalloc); `out` may be preallocated by the caller."""
    import torch
    nz, ny, nx = f.shape
    out = torch.empty(1, dtype=torch.float64, device=f.device) if out is None else out
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise TypeError("out must be a float64 CUDA tensor")
    _check(lib.cbct_tv_energy_noalloc(nx, ny, nz, float(h[0]), float(h[1]), float(h[2]), eps, _ptr(f, "f"),
                                      C.c_void_p(out.data_ptr()), _stream()))
    return out


def cbct_restrict_sino(y):
    import torch
    na, nv, nu = y.shape
    out = torch.empty((na, (nv + 1) // 2, (nu + 1) // 2), dtype=torch.float32, device=y.device)
    _check(lib.cbct_restrict_sino(na, nv, nu, _ptr(y, "y"), _ptr(out, "out"), _stream()))
    return out


def cbct_prolong_vol(fc, shape):
    import torch
    nzc, nyc, nxc = fc.shape
    nz, ny, nx = shape
    out = torch.empty(shape, dtype=torch.float32, device=fc.device)
    _check(lib.cbct_prolong_vol(nxc, nyc, nzc, _ptr(fc, "fc"), nx, ny, nz, _ptr(out, "out"), _stream()))
    return out
