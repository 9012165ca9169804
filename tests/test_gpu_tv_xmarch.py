"""The x-marching TV prox (two fused projected-gradient sweeps per launch, each voxel's
own term handed to its three lower neighbours) against the one-sweep-per-launch warp
tiles and the FP64 oracle (Algorithm A1 steps 2 and 3; E1 of Eq. 1).

The arithmetic per voxel is the same expressions in the same order in every form, so
the volumes must be bitwise equal across forms and launch shapes; the float64 energy
sums are grouped by tile and agree to rounding.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

LEGACY = {"tv_sweeps": -1}
SHAPES = [
    {"tv_sweeps": 2},                                       # the default shape
    {"tv_sweeps": 2, "tv_warps": 16, "tv_planes": 8},       # 13 output rows, many x-chunks
    {"tv_sweeps": 2, "tv_warps": 16, "tv_planes": 13},      # ragged chunks
    {"tv_sweeps": 2, "tv_warps": 32, "tv_planes": 64},
    {"tv_sweeps": 1, "tv_warps": 16, "tv_planes": 11},
    {"tv_sweeps": 1, "tv_warps": 32, "tv_planes": 40},
]


@pytest.fixture(scope="module")
def lib(cuda):
    from paper_1002_3675_b300 import cbct
    return cbct


def dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _geom(dims):
    nz, ny, nx = dims
    return dict(nx=nx, ny=ny, nz=nz, hx=1.0, hy=1.25, hz=2.0, nu=16, nv=16, du=30.0, dv=30.0, dso=800.0,
                dsd=1200.0, angles=np.array([0.0, 1.0]))


def _prox(lib, g, f0, gv, beta, eps, M, tv_mode, shape):
    G = lib.cbct_geometry_create(g)
    lib.cbct_set_tuning(G, 0, shape)
    ft = dev(f0)
    lib.cbct_tv_prox(G, dev(gv), ft, beta, eps, M, tv_mode=tv_mode)
    return host(ft)


# z-columns of 28, 44, 72 and 96 voxels (1, 2, 3 and 3 per lane, partly idle lanes), an
# odd x-size, and 45 voxels (not whole lanes and 16-byte pieces: the sweep tiles run)
@pytest.mark.parametrize("dims", [(28, 206, 160), (44, 206, 163), (72, 256, 180), (96, 200, 170), (45, 206, 163)])
@pytest.mark.parametrize("tv_mode", [0, 1])
def test_xmarch_prox_bitwise_equals_sweep_tiles(lib, dims, tv_mode):
    """Every x-marching launch shape gives the bits of the one-sweep-per-launch tiles, for
    an even and an odd number of sweeps and for one sweep, and matches the oracle."""
    rng = np.random.default_rng(41)
    f0 = np.clip(rng.normal(0.01, 0.006, size=dims), 0.0, None)
    gv = f0 + rng.normal(scale=0.003, size=dims)
    g = _geom(dims)
    eps, beta = 1e-3, 5.0e3
    for M in (10, 5, 1):
        ref = _prox(lib, g, f0, gv, beta, eps, M, tv_mode, LEGACY)
        for shape in SHAPES:
            out = _prox(lib, g, f0, gv, beta, eps, M, tv_mode, shape)
            assert np.array_equal(out, ref), (dims, tv_mode, M, shape)
            assert not np.signbit(out).any()
        if M == 10:
            o = oracle.prox(f32(gv), f32(f0), (1.0, 1.25, 2.0), beta, eps, M, tv_mode=tv_mode)
            d_ref = o - f32(f0)
            assert np.linalg.norm((ref - f32(f0)) - d_ref) <= 1e-4 * np.linalg.norm(d_ref)


@pytest.mark.parametrize("clamp_mode", [0, 1])
def test_xmarch_fbs_trace_and_volume_match_sweep_tiles(lib, clamp_mode):
    """Algorithm A1 iterations on a level in the x-marching domain: the volume is bitwise
    that of the sweep tiles, and the E1 / step-norm sums (fused into the first and last
    launch of each prox) agree to rounding; also the literal clamp mode (unconstrained
    descent from g, clamp at the last sweep)."""
    dims = (40, 180, 200)
    g = dict(nx=200, ny=180, nz=40, hx=1.5, hy=1.5, hz=2.5, nu=200, nv=60, du=2.0, dv=2.0, dso=800.0,
             dsd=1200.0, angles=2 * math.pi * np.arange(9) / 9 + 0.05)
    rng = np.random.default_rng(42)
    f_true = np.clip(rng.normal(0.01, 0.005, size=dims), 0.0, None)
    Y = oracle.project(g, f_true)
    mu, eps, beta = 2.0, 1e-4, 4.0e4
    res = {}
    for name, shape in (("legacy", LEGACY), ("x2", {"tv_sweeps": 2}), ("x1", {"tv_sweeps": 1, "tv_warps": 16})):
        G = lib.cbct_geometry_create(g)
        lib.cbct_set_tuning(G, 0, shape)
        ft, tr, st = lib.cbct_fbs(G, dev(Y), mu, beta, eps, 7, clamp_mode, 4, dev(np.zeros(dims)), trace=True,
                                  step_trace=True)
        res[name] = (host(ft), tr, st)
    f_l, tr_l, st_l = res["legacy"]
    for name in ("x2", "x1"):
        f_x, tr_x, st_x = res[name]
        assert np.array_equal(f_x, f_l), name
        assert np.allclose(tr_x, tr_l, rtol=1e-6, atol=0), name
        assert np.allclose(st_x, st_l, rtol=1e-6, atol=0), name
    assert (f_l >= 0).all()


def test_xmarch_tuning_rejects_bad_shapes(lib):
    g = _geom((40, 180, 170))
    G = lib.cbct_geometry_create(g)
    for bad in ({"tv_sweeps": 3}, {"tv_warps": 12}, {"tv_warps": 8}, {"tv_sweeps": 2, "tv_planes": 4},
                {"tv_sweeps": -2}):
        with pytest.raises(RuntimeError):
            lib.cbct_set_tuning(G, 0, bad)
