"""FP64 CPU oracle (ctypes binding of cbct_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product library (``paper_1002_3675_b300``) never does;
the oracle and the CUDA path share no code.

Arrays are float64 NumPy: volumes [nz][ny][nx], projection stacks [na][nv][nu].  A
geometry is the plain dict produced by ``synth.geometry_for``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbct_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP) if needed."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int), ("du", C.c_double), ("dv", C.c_double),
                ("dso", C.c_double), ("dsd", C.c_double),
                ("na", C.c_int), ("angles", C.POINTER(C.c_double)), ("tv_mode", C.c_int),
                ("adjoint_mode", C.c_int)]


class _Vol(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double), ("tv_mode", C.c_int)]


_lib = None
_D = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        G, V = C.POINTER(_Geom), C.POINTER(_Vol)
        sig = {
            "or_project": (None, [G, _D, _D]),
            "or_backproject": (None, [G, _D, _D]),
            "or_backproject_voxel": (C.c_double, [G, _D, C.c_int, C.c_int, C.c_int]),
            "or_backproject_eq2": (None, [G, _D, _D]),
            "or_project_ray": (C.c_double, [G, _D, C.c_int, C.c_int, C.c_int]),
            "or_ray_segments": (C.c_int, [G, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_long), _D, C.c_int]),
            "or_ray_voxel_length": (C.c_double, [G] + [C.c_int] * 6),
            "or_count_nnz": (C.c_longlong, [G]),
            "or_tv": (C.c_double, [V, _D, C.c_double]),
            "or_tv_grad": (None, [V, _D, C.c_double, _D]),
            "or_tv_lipschitz": (C.c_double, [V, C.c_double]),
            "or_prox": (None, [V, _D, _D, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, _D]),
            "or_gamma": (C.c_double, [G, C.c_double]),
            "or_default_eps": (C.c_double, [G]),
            "or_energy": (None, [G, _D, _D, C.c_double, C.c_double, _D, _D]),
            "or_power_iteration": (C.c_double, [G, C.c_int]),
            "or_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
            "or_uniform01": (C.c_double, [C.c_uint64, C.c_uint64]),
            "or_auto_beta": (C.c_double, [G, C.c_double, C.c_int]),
            "or_fbs": (None, [G, _D, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                              C.c_double, C.c_int, _D, _D, _D]),
            "or_restrict_vol": (None, [C.c_int, C.c_int, C.c_int, _D, _D]),
            "or_prolong_vol_adjoint": (None, [C.c_int] * 6 + [_D, _D]),
            "or_energy_grad": (None, [G, _D, _D, C.c_double, C.c_double, _D]),
            "or_vcycle": (None, [G, _D, C.c_double, C.c_int, C.c_int, _D, C.c_double, C.c_int, C.c_int, C.c_int,
                                 C.c_int, C.c_int, _D, _D, C.POINTER(C.c_int)]),
            "or_restrict_sino": (None, [C.c_int, C.c_int, C.c_int, _D, _D]),
            "or_prolong_vol": (None, [C.c_int, C.c_int, C.c_int, _D, C.c_int, C.c_int, C.c_int, _D]),
            "or_level_geom": (None, [G, C.c_int, G]),
            "or_reconstruct": (None, [G, _D, C.c_double, C.c_int, C.c_int, _D, C.c_double, C.c_int,
                                      C.c_int, C.c_int, _D, _D]),
            "or_num_threads": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _GeomHolder:
    """Keeps the angle array alive while the C struct points into it."""

    def __init__(self, geom: dict, tv_mode: int = 0, adjoint_mode: int = 0):
        self.angles = _f64(geom["angles"])
        self.s = _Geom(geom["nx"], geom["ny"], geom["nz"], geom["hx"], geom["hy"], geom["hz"],
                       geom["nu"], geom["nv"], geom["du"], geom["dv"], geom["dso"], geom["dsd"],
                       len(self.angles), _ptr(self.angles), int(tv_mode), int(adjoint_mode))


def _g(geom, tv_mode=0, adjoint_mode=0):
    return _GeomHolder(geom, tv_mode, adjoint_mode)


def _vol(shape, h, tv_mode=0):
    nz, ny, nx = shape
    return _Vol(nx, ny, nz, float(h[0]), float(h[1]), float(h[2]), int(tv_mode))


def vol_shape(geom):
    return (geom["nz"], geom["ny"], geom["nx"])


def sino_shape(geom):
    return (len(geom["angles"]), geom["nv"], geom["nu"])


def spacing(geom):
    return (geom["hx"], geom["hy"], geom["hz"])


def num_threads() -> int:
    return _load().or_num_threads()


# --- projector and adjoint (problem statement, Eq. 1; transpose before Eq. 2) --------

def project(geom, f):
    f = _f64(f)
    y = np.empty(sino_shape(geom))
    h = _g(geom)
    _load().or_project(C.byref(h.s), _ptr(f), _ptr(y))
    return y


def backproject(geom, y):
    y = _f64(y)
    f = np.empty(vol_shape(geom))
    h = _g(geom)
    _load().or_backproject(C.byref(h.s), _ptr(y), _ptr(f))
    return f


def backproject_eq2(geom, y):
    """B y of Eq. 2: per voxel centre and view, y bilinearly interpolated at (u*, v*)
    times L^3/(L0 l^2), summed over views and scaled by dV/(du dv)."""
    y = _f64(y)
    f = np.empty(vol_shape(geom))
    h = _g(geom)
    _load().or_backproject_eq2(C.byref(h.s), _ptr(y), _ptr(f))
    return f


def backproject_voxel(geom, y, i, j, k):
    y = _f64(y)
    h = _g(geom)
    return _load().or_backproject_voxel(C.byref(h.s), _ptr(y), i, j, k)


def project_ray(geom, f, ia, b, a):
    f = _f64(f)
    h = _g(geom)
    return _load().or_project_ray(C.byref(h.s), _ptr(f), ia, b, a)


def ray_segments(geom, ia, b, a):
    cap = geom["nx"] + geom["ny"] + geom["nz"] + 8
    idx = np.empty(cap, dtype=np.int64)
    ln = np.empty(cap)
    h = _g(geom)
    m = _load().or_ray_segments(C.byref(h.s), ia, b, a, idx.ctypes.data_as(C.POINTER(C.c_long)), _ptr(ln), cap)
    return idx[:m].copy(), ln[:m].copy()


def ray_voxel_length(geom, ia, b, a, i, j, k):
    h = _g(geom)
    return _load().or_ray_voxel_length(C.byref(h.s), ia, b, a, i, j, k)


def count_nnz(geom) -> int:
    h = _g(geom)
    return int(_load().or_count_nnz(C.byref(h.s)))


# --- TV (E1) and the step-2 prox ------------------------------------------------------
# tv_mode 0: isotropic sum_j sqrt(|grad f|^2 + eps^2); 1: anisotropic
# sum_j sum_d sqrt((D_d f)^2 + eps^2).

def tv(f, h, eps, tv_mode=0):
    f = _f64(f)
    v = _vol(f.shape, h, tv_mode)
    return _load().or_tv(C.byref(v), _ptr(f), eps)


def tv_grad(f, h, eps, tv_mode=0):
    f = _f64(f)
    out = np.empty_like(f)
    v = _vol(f.shape, h, tv_mode)
    _load().or_tv_grad(C.byref(v), _ptr(f), eps, _ptr(out))
    return out


def tv_lipschitz(h, eps):
    v = _vol((1, 1, 1), h)
    return _load().or_tv_lipschitz(C.byref(v), eps)


def prox(g, f0, h, beta, eps, M, clamp_mode=0, tv_weight=1.0, return_phi=False, tv_mode=0):
    g = _f64(g)
    f = _f64(f0).copy() if f0 is not None else np.zeros_like(g)
    phi = np.empty(M + 1) if return_phi else None
    v = _vol(g.shape, h, tv_mode)
    _load().or_prox(C.byref(v), _ptr(g), _ptr(f), beta, eps, M, clamp_mode, tv_weight, _ptr(phi))
    return (f, phi) if return_phi else f


# --- energy, step size, Algorithm A1, multigrid ---------------------------------------

def gamma(geom, mu):
    h = _g(geom)
    return _load().or_gamma(C.byref(h.s), mu)


def default_eps(geom):
    h = _g(geom)
    return _load().or_default_eps(C.byref(h.s))


def energy(geom, Y, f, mu, eps, return_residual=False, tv_mode=0):
    Y, f = _f64(Y), _f64(f)
    out = np.empty(3)
    r = np.empty(sino_shape(geom)) if return_residual else None
    h = _g(geom, tv_mode)
    _load().or_energy(C.byref(h.s), _ptr(Y), _ptr(f), mu, eps, _ptr(out), _ptr(r))
    return (out, r) if return_residual else out


def splitmix64(seed, i):
    """Value i of the counter-based SplitMix64 generator with seed `seed`."""
    return int(_load().or_splitmix64(seed, i))


def uniform01(seed, i):
    """The top 24 bits of splitmix64(seed, i) as a number in [0, 1)."""
    return float(_load().or_uniform01(seed, i))


POWER_SEED = 10023675  # seed of the power iteration's start volume


def power_iteration(geom, K=30):
    h = _g(geom)
    return _load().or_power_iteration(C.byref(h.s), K)


def auto_beta(geom, mu, K=30):
    h = _g(geom)
    return _load().or_auto_beta(C.byref(h.s), mu, K)


def fbs(geom, Y, mu, beta, eps, M, iters, f0=None, clamp_mode=0, tv_weight=1.0, tv_mode=0, adjoint_mode=0,
        v=None, steps=False):
    """Algorithm A1; v (optional volume) adds the linear term -<v, f> to the energy.
    Returns (f, trace [iters][3]), or (f, trace, |f_k+1 - f_k| [iters]) with steps=True."""
    Y = _f64(Y)
    f = _f64(f0).copy() if f0 is not None else np.zeros(vol_shape(geom))
    trace = np.empty((iters, 3))
    st = np.empty(max(iters, 1)) if steps else None
    vv = _f64(v) if v is not None else None
    h = _g(geom, tv_mode, adjoint_mode)
    _load().or_fbs(C.byref(h.s), _ptr(Y), mu, beta, eps, M, clamp_mode, tv_weight, iters, _ptr(f), _ptr(trace),
                   _ptr(vv), _ptr(st))
    return (f, trace, st[:iters]) if steps else (f, trace)


def restrict_sino(y):
    y = _f64(y)
    na, nv, nu = y.shape
    out = np.empty((na, (nv + 1) // 2, (nu + 1) // 2))
    _load().or_restrict_sino(na, nv, nu, _ptr(y), _ptr(out))
    return out


def prolong_vol(fc, shape):
    fc = _f64(fc)
    nzc, nyc, nxc = fc.shape
    nz, ny, nx = shape
    out = np.empty(shape)
    _load().or_prolong_vol(nxc, nyc, nzc, _ptr(fc), nx, ny, nz, _ptr(out))
    return out


def level_geom(geom, level):
    h = _g(geom)
    out = _Geom()
    _load().or_level_geom(C.byref(h.s), level, C.byref(out))
    g2 = dict(geom)
    for k in ("nx", "ny", "nz", "hx", "hy", "hz", "nu", "nv", "du", "dv"):
        g2[k] = getattr(out, k)
    return g2


def reconstruct(geom, Y, mu, iters, levels, betas=None, eps=0.0, M=10, clamp_mode=0, K_pi=30, tv_mode=0,
                adjoint_mode=0):
    Y = _f64(Y)
    f = np.empty(vol_shape(geom))
    trace = np.empty((levels, iters, 3))
    b = _f64(betas) if betas is not None else None
    h = _g(geom, tv_mode, adjoint_mode)
    _load().or_reconstruct(C.byref(h.s), _ptr(Y), mu, iters, levels, _ptr(b), eps, M, clamp_mode,
                           K_pi, _ptr(f), _ptr(trace))
    return f, trace


# --- V-cycle (full-approximation multigrid reading of the cited method) --------------

def restrict_vol(f):
    f = _f64(f)
    nz, ny, nx = f.shape
    out = np.empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2))
    _load().or_restrict_vol(nx, ny, nz, _ptr(f), _ptr(out))
    return out


def prolong_vol_adjoint(x, coarse_shape):
    x = _f64(x)
    nz, ny, nx = x.shape
    nzc, nyc, nxc = coarse_shape
    out = np.empty(coarse_shape)
    _load().or_prolong_vol_adjoint(nxc, nyc, nzc, nx, ny, nz, _ptr(x), _ptr(out))
    return out


def energy_grad(geom, Y, f, mu, eps):
    Y, f = _f64(Y), _f64(f)
    out = np.empty_like(f)
    h = _g(geom)
    _load().or_energy_grad(C.byref(h.s), _ptr(Y), _ptr(f), mu, eps, _ptr(out))
    return out


def vcycle(geom, Y, mu, cycles, levels, betas=None, eps=0.0, M=10, pre=2, post=2, coarse=10, K_pi=30, tv_mode=0):
    """Returns (f, trace [cycles][3], accepted [levels])."""
    Y = _f64(Y)
    f = np.empty(vol_shape(geom))
    trace = np.empty((cycles, 3))
    acc = (C.c_int * levels)()
    b = _f64(betas) if betas is not None else None
    h = _g(geom, tv_mode)
    _load().or_vcycle(C.byref(h.s), _ptr(Y), mu, cycles, levels, _ptr(b), eps, M, pre, post, coarse, K_pi,
                      _ptr(f), _ptr(trace), acc)
    return f, trace, np.array(acc[:])
