"""The Eq. 2 adjoint (cbct_backproject_eq2) against the FP64 oracle at full size.

The small and ragged cases are in test_gpu_variants.py.  These cover the medium
geometry's full imager (256x192, 40 views) on the whole 256x256x64 volume, the large
geometry's full imager (512x384, 40 views) on the 4 central z-levels of 512x512x96, and
a geometry with a fine imager pitch (many imager columns per voxel, nx and ny not
multiples of 4, nv + 2 not a multiple of 4).
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / np.linalg.norm(b))


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


def _smooth(g, seed):
    # a residual that varies smoothly over the imager (as projections of a volume do);
    # for data with jumps between neighbouring pixels the float32 row coordinate v*
    # (about 1e-5 relative at a few hundred rows) moves the interpolated value by that
    # much times the jump, which is inherent in a float32 evaluation of Eq. 2
    rng = np.random.default_rng(seed)
    na, nv, nu = len(g["angles"]), g["nv"], g["nu"]
    ph = rng.uniform(0, 2 * math.pi, size=(na, 1, 1))
    u = np.arange(nu)[None, None, :] / nu
    v = np.arange(nv)[None, :, None] / nv
    return (0.4 + np.cos(2 * math.pi * 1.3 * u + ph) * np.sin(math.pi * 2.1 * v + 0.5 * ph)).astype(np.float32)


def _check_eq2(lib, g, seed, tol=1e-5):
    y = _smooth(g, seed)
    G = lib.cbct_geometry_create(g)
    out = host(lib.cbct_backproject_eq2(G, dev(y)))
    ref = oracle.backproject_eq2(g, y.astype(np.float64))
    assert rel(out, ref) <= tol, rel(out, ref)
    assert np.abs(out - ref).max() <= tol * np.abs(ref).max()
    # a second call on the same geometry reuses the workspace and gives the same bits
    assert np.array_equal(host(lib.cbct_backproject_eq2(G, dev(y))), out)


def test_eq2_medium_full_size(lib):
    _check_eq2(lib, synth.geometry_for(synth.CONFIGS["medium"]), 71)


def test_eq2_fine_imager_pitch(lib):
    # 4 mm voxels on a 0.5 mm pitch imager: a voxel spans about a dozen imager columns
    g = dict(nx=18, ny=13, nz=11, hx=4.0, hy=4.0, hz=4.0, nu=301, nv=29, du=0.5, dv=4.0, dso=500.0, dsd=800.0,
             angles=2 * math.pi * np.arange(7) / 7 + 0.3)
    _check_eq2(lib, g, 72)


def test_eq2_large_central_slab(lib):
    # the full large imager (512x384, 40 views) on 512x512x96; the oracle evaluates the 4
    # central z-levels (a volume of nz = 4 has the same voxel centres as levels 46-49)
    g = synth.geometry_for(synth.CONFIGS["large"])
    y = _smooth(g, 73)
    G = lib.cbct_geometry_create(g)
    out = host(lib.cbct_backproject_eq2(G, dev(y)))   # [nz][ny][nx]
    k0 = g["nz"] // 2 - 2
    ref = oracle.backproject_eq2(dict(g, nz=4), y.astype(np.float64))
    got = out[k0:k0 + 4]
    assert rel(got, ref) <= 1e-5, rel(got, ref)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
