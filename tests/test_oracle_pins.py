"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test names the passage of Jia et al. (2010) it pins and the independent fact used:
closed forms, a brute-force system matrix, invariants, a library optimiser, exact
hand-derived lengths, and the paper's own Eq. 2.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.brute_matrix import ray_endpoints, system_matrix, tiny_geometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _box_chord(S, P, lo, hi):
    """Closed-form length of the segment S->P inside the box [lo, hi] (slab method)."""
    d = P - S
    t0, t1 = 0.0, 1.0
    for ax in range(3):
        if d[ax] == 0.0:
            if not (lo[ax] <= S[ax] < hi[ax]):
                return 0.0
            continue
        a, b = (lo[ax] - S[ax]) / d[ax], (hi[ax] - S[ax]) / d[ax]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(t1 - t0, 0.0) * float(np.linalg.norm(d))


# ---------------------------------------------------------------------------------
# Projector P^theta (problem statement, Eq. 1)
# ---------------------------------------------------------------------------------

def test_P_of_ones_is_box_chord():
    """f = 1 on the volume: every line integral is the ray's chord through the box."""
    g = tiny_geometry(n=8, h=4.0, nu=10, nv=7, du=7.0, dv=9.0, n_angles=5, theta0=0.3)
    y = oracle.project(g, np.ones((8, 8, 8)))
    S, P = ray_endpoints(g)
    half = np.array([16.0, 16.0, 16.0])
    ref = np.array([[[_box_chord(S[ia], P[ia, b, a], -half, half) for a in range(10)]
                     for b in range(7)] for ia in range(5)])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    assert (ref > 0).sum() > 100


def test_P_single_voxel_indicator():
    """f = e_j: the projection is the ray's intersection length with voxel j's box."""
    g = tiny_geometry(n=6, h=5.0, nu=9, nv=9, du=6.0, dv=6.0, n_angles=3, theta0=0.1)
    S, P = ray_endpoints(g)
    for (i, j, k) in [(0, 0, 0), (2, 3, 1), (5, 5, 5), (3, 2, 4)]:
        f = np.zeros((6, 6, 6))
        f[k, j, i] = 1.0
        y = oracle.project(g, f)
        lo = np.array([(i - 3) * 5.0, (j - 3) * 5.0, (k - 3) * 5.0])
        ref = np.array([[[_box_chord(S[ia], P[ia, b, a], lo, lo + 5.0) for a in range(9)]
                         for b in range(9)] for ia in range(3)])
        assert np.abs(y - ref).max() <= 1e-12 * 5.0


def test_P_and_PT_equal_brute_force_matrix():
    """8^3 volume, 8x8 imager, 6 views: P = A and P^T = A^T for a dense A built by
    testing every ray against every voxel box."""
    g = tiny_geometry()
    A = system_matrix(g)
    rng = np.random.default_rng(1)
    for _ in range(3):
        f = rng.uniform(-1, 1, size=(8, 8, 8))
        y = rng.normal(size=(6, 8, 8))
        Pf = oracle.project(g, f)
        assert np.abs(Pf.ravel() - A @ f.ravel()).max() <= 1e-12 * np.abs(A @ f.ravel()).max()
        PTy = oracle.backproject(g, y)
        assert np.abs(PTy.ravel() - A.T @ y.ravel()).max() <= 1e-12 * np.abs(A.T @ y.ravel()).max()
    assert oracle.count_nnz(g) == int((A > 0).sum())


def test_degenerate_rays_match_brute_force():
    """Odd imager sizes put central rays exactly in voxel planes (d_y = 0, d_z = 0 at
    theta = 0); the half-open voxel convention decides their voxel.  Compared with the
    brute-force matrix, which applies the same convention by slab tests."""
    g = tiny_geometry(n=8, h=4.0, nu=9, nv=9, du=8.0, dv=8.0, n_angles=4)
    A = system_matrix(g)
    rng = np.random.default_rng(2)
    f = rng.uniform(size=(8, 8, 8))
    assert np.abs(oracle.project(g, f).ravel() - A @ f.ravel()).max() <= 1e-12 * 100
    y = rng.normal(size=(4, 9, 9))
    assert np.abs(oracle.backproject(g, y).ravel() - A.T @ y.ravel()).max() <= 1e-12 * 100
    # the central ray at theta = 0 lies in y = 0 and z = 0 and belongs to j = 4, k = 4
    idx, ln = oracle.ray_segments(g, 0, 4, 4)
    ks, js = idx // 64, (idx // 8) % 8
    assert set(ks.tolist()) == {4} and set(js.tolist()) == {4}
    assert abs(ln.sum() - 32.0) < 1e-12


def test_golden_hand_derived_rays():
    with open(os.path.join(GOLDEN, "hand_rays.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        g = dict(case["geom"])
        g["angles"] = np.array(g["angles"], dtype=np.float64)
        ia, b, a = case["ray"]
        idx, ln = oracle.ray_segments(g, ia, b, a)
        got = {int(q): float(L) for q, L in zip(idx, ln) if L > 0}
        want = {(k * g["ny"] + j) * g["nx"] + i: L for i, j, k, L in case["voxels"]}
        assert set(got) == set(want), case["name"]
        for q in want:
            assert abs(got[q] - want[q]) <= 1e-14 * 4, case["name"]


def test_P_converges_to_analytic_chords():
    """Voxelised ellipsoid phantom: P f_h tends to the exact line integrals as h -> 0
    (error falling with h, about first order overall)."""
    errs = []
    for n in (16, 32, 64, 128):
        h = 128.0 / n
        g = dict(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, nu=40, nv=30, du=6.0, dv=6.0,
                 dso=1000.0, dsd=1500.0, angles=2 * math.pi * np.arange(4) / 4 + 0.2)
        ells = synth.make_ellipsoids(g, np.random.default_rng(5), n=4)
        exact = synth.analytic_sinogram(ells, g)
        f = synth.voxelize(ells, g, ss=4)
        errs.append(np.linalg.norm(oracle.project(g, f) - exact) / np.linalg.norm(exact))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 0.15 * errs[0]     # 8x finer grid, first-order convergence
    assert errs[3] < 0.012


def test_P_rotation_symmetry():
    """With nx = ny and hx = hy, the view at theta + 90 deg of the volume rotated by
    90 deg about z equals the view at theta of the original volume."""
    n = 10
    base = dict(nx=n, ny=n, nz=6, hx=3.0, hy=3.0, hz=4.0, nu=12, nv=8, du=5.0, dv=5.0, dso=150.0, dsd=240.0)
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(6, n, n))
    th = np.array([0.37, 1.1])
    y0 = oracle.project(dict(base, angles=th), f)
    # rotation (x, y) -> (-y, x): f'[k, J, I] = f[k, n-1-I, J]
    fr = f[:, ::-1, :].transpose(0, 2, 1)
    y1 = oracle.project(dict(base, angles=th + math.pi / 2), fr)
    assert np.abs(y0 - y1).max() <= 1e-12 * np.abs(y0).max()


# ---------------------------------------------------------------------------------
# Adjoint (matrix transpose before Eq. 2; Eq. 2 itself)
# ---------------------------------------------------------------------------------

def test_adjoint_identity():
    case = synth.make_case("small")
    g = case["geom"]
    rng = np.random.default_rng(4)
    f = rng.uniform(size=(64, 64, 64))
    y = rng.normal(size=(20, 48, 64))
    Pf = oracle.project(g, f)
    lhs = float(np.sum(Pf * y))
    rhs = float(np.sum(f * oracle.backproject(g, y)))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Pf) * np.linalg.norm(y)


def test_scatter_adjoint_equals_voxel_brute_force():
    """The scatter adjoint at sampled voxels of the 64^3 workload equals a per-voxel
    sum over every ray of its slab-test length (no Siddon walk involved)."""
    g = synth.geometry_for(synth.CONFIGS["small"])
    rng = np.random.default_rng(6)
    y = rng.normal(size=(20, 48, 64))
    bt = oracle.backproject(g, y)
    for _ in range(6):
        i, j, k = rng.integers(0, 64, size=3)
        v = oracle.backproject_voxel(g, y, int(i), int(j), int(k))
        assert abs(v - bt[k, j, i]) <= 1e-11 * max(1.0, abs(v))


def test_adjoint_matches_eq2_jacobian():
    """Eq. 2: the variation of E2 weighs the residual at (u*, v*) by 2 L^3/(L0 l^2).
    Summed over a voxel's rays, the exact transpose of 1 therefore approaches
    sum_theta dV L^3 / (L0 l^2 du dv) when the imager samples the voxel finely."""
    n, h = 12, 4.0
    g = dict(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, nu=200, nv=200, du=0.6, dv=0.6,
             dso=300.0, dsd=450.0, angles=2 * math.pi * np.arange(8) / 8 + 0.05)
    bt = oracle.backproject(g, np.ones((8, 200, 200)))
    ratios = []
    for k in range(3, 9):
        for j in range(3, 9):
            for i in range(3, 9):
                x = np.array([(i - (n - 1) / 2) * h, (j - (n - 1) / 2) * h, (k - (n - 1) / 2) * h])
                ref = 0.0
                for th in g["angles"]:
                    S = np.array([g["dso"] * math.cos(th), g["dso"] * math.sin(th), 0.0])
                    w = np.array([-math.cos(th), -math.sin(th), 0.0])     # central-ray direction
                    d = x - S
                    l = np.linalg.norm(d)
                    L = l * g["dsd"] / float(d @ w)                       # source to (u*, v*)
                    ref += h ** 3 * L ** 3 / (g["dsd"] * l * l * g["du"] * g["dv"])
                ratios.append(bt[k, j, i] / ref)
    ratios = np.array(ratios)
    assert abs(ratios.mean() - 1.0) < 0.01
    assert np.abs(ratios - 1.0).max() < 0.05


def _imager_point(g, th, x):
    """(a*, b*, L, l) for voxel centre x: the line from the source through x meets the
    imager plane; solved as a 3x3 linear system (independent of the oracle's closed
    form)."""
    S = np.array([g["dso"] * math.cos(th), g["dso"] * math.sin(th), 0.0])
    C = S + g["dsd"] * np.array([-math.cos(th), -math.sin(th), 0.0])
    eu = np.array([-math.sin(th), math.cos(th), 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    # S + t (x - S) = C + u eu + v ev
    t, u, v = np.linalg.solve(np.column_stack([x - S, -eu, -ev]), C - S)
    P = S + t * (x - S)
    a = u / g["du"] + (g["nu"] - 1) / 2
    b = v / g["dv"] + (g["nv"] - 1) / 2
    return a, b, float(np.linalg.norm(P - S)), float(np.linalg.norm(x - S))


def _eq2_geom():
    return dict(nx=10, ny=9, nz=8, hx=4.0, hy=4.5, hz=5.0, nu=36, nv=30, du=3.0, dv=3.5,
                dso=300.0, dsd=450.0, angles=2 * math.pi * np.arange(5) / 5 + 0.13)


def _centre(g, i, j, k):
    return np.array([(i - (g["nx"] - 1) / 2) * g["hx"], (j - (g["ny"] - 1) / 2) * g["hy"],
                     (k - (g["nz"] - 1) / 2) * g["hz"]])


def test_eq2_adjoint_single_pixel_impulse():
    """B of Eq. 2 applied to one pixel of one view: every voxel whose imager point lies
    within one pixel of it (in both directions) gets dV/(du dv) L^3/(L0 l^2) times the
    bilinear hat weight, every other voxel exactly 0."""
    g = _eq2_geom()
    ia, bp, ap = 2, 17, 14
    y = np.zeros((5, 30, 36))
    y[ia, bp, ap] = 1.0
    B = oracle.backproject_eq2(g, y)
    scale = g["hx"] * g["hy"] * g["hz"] / (g["du"] * g["dv"])
    hit = 0
    for k in range(g["nz"]):
        for j in range(g["ny"]):
            for i in range(g["nx"]):
                a, b, L, l = _imager_point(g, g["angles"][ia], _centre(g, i, j, k))
                wa, wb = 1 - abs(a - ap), 1 - abs(b - bp)
                ref = scale * L ** 3 / (g["dsd"] * l * l) * wa * wb if (wa > 0 and wb > 0) else 0.0
                hit += ref > 0
                assert abs(B[k, j, i] - ref) <= 1e-12 * max(1.0, abs(ref))
    assert hit >= 2


def test_eq2_adjoint_reproduces_linear_residuals():
    """Bilinear interpolation is exact for residuals linear in the pixel indices, so
    B y is a closed form in (a*, b*) for voxels that project inside the pixel grid."""
    g = _eq2_geom()
    ia_, b_, a_ = np.meshgrid(np.arange(5), np.arange(30), np.arange(36), indexing="ij")
    y = 0.7 + 0.013 * a_ - 0.021 * b_ + 0.05 * ia_
    B = oracle.backproject_eq2(g, y)
    scale = g["hx"] * g["hy"] * g["hz"] / (g["du"] * g["dv"])
    for (i, j, k) in [(0, 0, 0), (9, 8, 7), (4, 4, 4), (2, 7, 5), (8, 1, 3)]:
        ref = 0.0
        for t, th in enumerate(g["angles"]):
            a, b, L, l = _imager_point(g, th, _centre(g, i, j, k))
            assert 0 <= a <= 35 and 0 <= b <= 29
            ref += scale * L ** 3 / (g["dsd"] * l * l) * (0.7 + 0.013 * a - 0.021 * b + 0.05 * t)
        assert abs(B[k, j, i] - ref) <= 1e-12 * abs(ref)


def test_eq2_adjoint_approaches_the_transpose():
    """With an imager that samples every voxel finely, B 1 and P^T 1 agree on interior
    voxels (Eq. 2 is the continuum form of the transpose)."""
    n, h = 12, 4.0
    g = dict(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, nu=200, nv=200, du=0.6, dv=0.6,
             dso=300.0, dsd=450.0, angles=2 * math.pi * np.arange(8) / 8 + 0.05)
    ones = np.ones((8, 200, 200))
    ratio = oracle.backproject_eq2(g, ones)[3:9, 3:9, 3:9] / oracle.backproject(g, ones)[3:9, 3:9, 3:9]
    assert abs(ratio.mean() - 1.0) < 0.01
    assert np.abs(ratio - 1.0).max() < 0.05


def test_fbs_with_eq2_adjoint_reduces_the_energy():
    case = synth.make_case("small")
    g = case["geom"]
    mu, eps = case["mu"], oracle.default_eps(g)
    beta = oracle.auto_beta(g, mu)
    f, tr = oracle.fbs(g, case["Y"], mu, beta, eps, 10, 20, adjoint_mode=1)
    E_end = oracle.energy(g, case["Y"], f, mu, eps)[0]
    assert E_end < 0.3 * tr[0, 0] and (f >= 0).all()
    f0, _ = oracle.fbs(g, case["Y"], mu, beta, eps, 10, 20)
    assert np.linalg.norm(f - f0) > 1e-3 * np.linalg.norm(f0)   # a different operator


# ---------------------------------------------------------------------------------
# E1 and the step-2 prox (Algorithm A1 steps 2 and 3)
# ---------------------------------------------------------------------------------

H = (1.3, 0.7, 2.1)


def test_tv_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    f = rng.uniform(size=(5, 6, 7))
    eps = 0.05
    gr = oracle.tv_grad(f, H, eps)
    step = 1e-6
    for _ in range(20):
        k, j, i = rng.integers(0, 5), rng.integers(0, 6), rng.integers(0, 7)
        fp, fm = f.copy(), f.copy()
        fp[k, j, i] += step
        fm[k, j, i] -= step
        fd = (oracle.tv(fp, H, eps) - oracle.tv(fm, H, eps)) / (2 * step)
        assert abs(fd - gr[k, j, i]) <= 1e-7 * max(1.0, abs(fd))


def test_tv_of_constant_and_of_a_step():
    eps = 0.01
    f = np.full((4, 5, 6), 3.0)
    assert abs(oracle.tv(f, H, eps) - f.size * eps) <= 1e-12 * f.size * eps
    assert np.abs(oracle.tv_grad(f, H, eps)).max() == 0.0
    # a step of height 0.7 along x between i = 2 and i = 3: TV_0 = ny nz 0.7 / hx
    s = np.zeros((4, 5, 6))
    s[:, :, 3:] = 0.7
    assert abs(oracle.tv(s, H, 0.0) - 4 * 5 * 0.7 / H[0]) <= 1e-12


def test_tv_matches_autograd_definition():
    """TV_eps and its gradient against an independent torch autograd statement."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    f = rng.uniform(size=(6, 5, 7))
    eps = 0.02
    t = torch.tensor(f, requires_grad=True, dtype=torch.float64)
    dz = torch.nn.functional.pad(torch.diff(t, dim=0), (0, 0, 0, 0, 0, 1)) / H[2]
    dy = torch.nn.functional.pad(torch.diff(t, dim=1), (0, 0, 0, 1)) / H[1]
    dx = torch.nn.functional.pad(torch.diff(t, dim=2), (0, 1)) / H[0]
    val = torch.sqrt(dx * dx + dy * dy + dz * dz + eps * eps).sum()
    val.backward()
    assert abs(val.item() - oracle.tv(f, H, eps)) <= 1e-12 * val.item()
    assert np.abs(t.grad.numpy() - oracle.tv_grad(f, H, eps)).max() <= 1e-10


def test_anisotropic_tv_gradient_and_closed_forms():
    """tv_mode 1 (sum_d sqrt((D_d f)^2 + eps^2)): central finite differences of the
    value, the constant volume (3 Nv eps, zero gradient) and a ramp in x and y whose
    isotropic and anisotropic totals have different closed forms."""
    rng = np.random.default_rng(17)
    f = rng.uniform(size=(5, 6, 7))
    eps = 0.05
    gr = oracle.tv_grad(f, H, eps, tv_mode=1)
    step = 1e-6
    for _ in range(20):
        k, j, i = rng.integers(0, 5), rng.integers(0, 6), rng.integers(0, 7)
        fp, fm = f.copy(), f.copy()
        fp[k, j, i] += step
        fm[k, j, i] -= step
        fd = (oracle.tv(fp, H, eps, tv_mode=1) - oracle.tv(fm, H, eps, tv_mode=1)) / (2 * step)
        assert abs(fd - gr[k, j, i]) <= 1e-7 * max(1.0, abs(fd))
    c = np.full((4, 5, 6), 3.0)
    assert abs(oracle.tv(c, H, 0.01, tv_mode=1) - 3 * c.size * 0.01) <= 1e-12 * c.size
    assert np.abs(oracle.tv_grad(c, H, 0.01, tv_mode=1)).max() == 0.0
    nz, ny, nx = 4, 5, 6
    a, b = 0.3, -0.8
    ramp = a * np.arange(nx)[None, None, :] + b * np.arange(ny)[None, :, None] + np.zeros((nz, ny, nx))
    A, B = abs(a) / H[0], abs(b) / H[1]
    aniso = nz * ny * (nx - 1) * A + nz * nx * (ny - 1) * B
    iso = nz * ((nx - 1) * (ny - 1) * np.hypot(A, B) + (nx - 1) * A + (ny - 1) * B)
    assert abs(oracle.tv(ramp, H, 0.0, tv_mode=1) - aniso) <= 1e-12 * aniso
    assert abs(oracle.tv(ramp, H, 0.0) - iso) <= 1e-12 * iso
    assert aniso > iso


def test_anisotropic_tv_matches_autograd_definition():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(18)
    f = rng.uniform(size=(6, 5, 7))
    eps = 0.02
    t = torch.tensor(f, requires_grad=True, dtype=torch.float64)
    dz = torch.nn.functional.pad(torch.diff(t, dim=0), (0, 0, 0, 0, 0, 1)) / H[2]
    dy = torch.nn.functional.pad(torch.diff(t, dim=1), (0, 0, 0, 1)) / H[1]
    dx = torch.nn.functional.pad(torch.diff(t, dim=2), (0, 1)) / H[0]
    val = sum(torch.sqrt(d * d + eps * eps).sum() for d in (dx, dy, dz))
    val.backward()
    assert abs(val.item() - oracle.tv(f, H, eps, tv_mode=1)) <= 1e-12 * val.item()
    assert np.abs(t.grad.numpy() - oracle.tv_grad(f, H, eps, tv_mode=1)).max() <= 1e-10


def test_prox_limits_and_monotonicity():
    rng = np.random.default_rng(9)
    g = rng.normal(size=(6, 7, 8))
    f0 = np.maximum(rng.normal(size=g.shape), 0.0)
    eps = 0.05
    # beta -> infinity: the prox is the projection max(g, 0)
    f = oracle.prox(g, f0, H, 1e9, eps, 60)
    assert np.abs(f - np.maximum(g, 0)).max() < 1e-6
    # Phi = TV_eps + beta/2 |f - g|^2 never increases; f >= 0 exactly
    f, phi = oracle.prox(g, f0, H, 3.0, eps, 25, return_phi=True)
    assert np.all(np.diff(phi) <= 1e-12 * np.abs(phi[:-1]))
    assert (f >= 0).all()
    # paper-literal clamp (descend from g, clamp once): still non-negative
    f1 = oracle.prox(g, None, H, 3.0, eps, 25, clamp_mode=1)
    assert (f1 >= 0).all() and np.any(f1 == 0)
    # the anisotropic E1 keeps both properties (same Lipschitz bound)
    f2, phi2 = oracle.prox(g, f0, H, 3.0, eps, 25, return_phi=True, tv_mode=1)
    assert np.all(np.diff(phi2) <= 1e-12 * np.abs(phi2[:-1])) and (f2 >= 0).all()
    assert np.abs(oracle.prox(g, f0, H, 1e9, eps, 60, tv_mode=1) - np.maximum(g, 0)).max() < 1e-6


# ---------------------------------------------------------------------------------
# Algorithm A1 (FBS) and the energy of Eq. 1
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("tv_mode", [0, 1])
def test_fbs_energy_monotone_small_workload(tv_mode):
    case = synth.make_case("small")
    g = case["geom"]
    beta = oracle.auto_beta(g, case["mu"])
    eps = oracle.default_eps(g)
    f, tr = oracle.fbs(g, case["Y"], case["mu"], beta, eps, 10, 20, tv_mode=tv_mode)
    E = list(tr[:, 0]) + [oracle.energy(g, case["Y"], f, case["mu"], eps, tv_mode=tv_mode)[0]]
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a * (1 + 1e-12)
    assert E[-1] < 0.2 * E[0]
    assert (f >= 0).all()


def test_beta_ten_mu_regime_on_a_scaled_geometry():
    """Scaling every length by s scales P by s and lambda_max(P^T P) by s^2; at
    s = 1e-3 the bound 1.05 gamma lambda falls below 10 mu, so the automatic beta is
    the paper's 10 mu, and Algorithm A1 still decreases the energy there."""
    case = synth.make_case("small")
    g = case["geom"]
    s = 1e-3
    gs = dict(g, **{k: g[k] * s for k in ("hx", "hy", "hz", "du", "dv", "dso", "dsd")})
    lam, lam_s = oracle.power_iteration(g, 30), oracle.power_iteration(gs, 30)
    assert abs(lam_s - s * s * lam) <= 1e-9 * s * s * lam
    mu = case["mu"]
    assert oracle.auto_beta(gs, mu) == 10.0 * mu
    Ys = case["Y"] * s          # line integrals of the same densities over shorter chords
    eps = oracle.default_eps(gs)
    f, tr = oracle.fbs(gs, Ys, mu, 10.0 * mu, eps, 10, 10)
    E = list(tr[:, 0]) + [oracle.energy(gs, Ys, f, mu, eps)[0]]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E[:-1], E[1:]))


def test_fbs_fixed_point():
    """f* constant and Y = P f*: E1 = eps (TV_eps / Nv), E2 = 0 and f stays at f*."""
    g = tiny_geometry(n=8, h=4.0, nu=10, nv=10, du=7.0, dv=7.0, n_angles=5)
    fstar = np.full((8, 8, 8), 0.013)
    Y = oracle.project(g, fstar)
    eps = 1e-3
    E = oracle.energy(g, Y, fstar, 2.0, eps)
    assert abs(E[1] - eps) <= 1e-15 and E[2] == 0.0
    f, _, st = oracle.fbs(g, Y, 2.0, 50.0, eps, 5, 3, f0=fstar, steps=True)
    assert np.abs(f - fstar).max() <= 1e-15
    assert st.shape == (3,) and st.max() <= 1e-14   # |f_k+1 - f_k| at the fixed point


def test_fbs_without_tv_is_projected_landweber():
    """Removing the TV term (weight 0, one inner step of length 1/beta) reduces
    Algorithm A1 to f <- max(0, f - (gamma/beta) A^T (A f - Y)) on the dense matrix;
    the step norms |f_k+1 - f_k| are those of that iteration."""
    g = tiny_geometry()
    A = system_matrix(g)
    rng = np.random.default_rng(10)
    Y = rng.uniform(0, 3, size=(6, 8, 8))
    mu, beta = 1.5, 4000.0
    f, _, st = oracle.fbs(g, Y, mu, beta, 1e-3, 1, 15, tv_weight=0.0, steps=True)
    gam = 2 * mu * 512 / (6 * 64)
    x = np.zeros(512)
    dx = []
    for _ in range(15):
        xn = np.maximum(0.0, x - gam / beta * (A.T @ (A @ x - Y.ravel())))
        dx.append(np.linalg.norm(xn - x))
        x = xn
    assert np.abs(f.ravel() - x).max() <= 1e-12 * max(1.0, np.abs(x).max())
    assert np.allclose(st, dx, rtol=1e-10, atol=1e-14)


@pytest.mark.slow
def test_fbs_converges_to_lbfgsb_minimiser():
    """On 8^3 the FBS limit equals SciPy's L-BFGS-B minimiser of the same objective
    Nv E = TV_eps + (gamma/2)|A f - Y|^2 over f >= 0 (TV via torch autograd)."""
    torch = pytest.importorskip("torch")
    from scipy.optimize import minimize

    g = tiny_geometry(n=8, h=4.0, nu=10, nv=10, du=6.0, dv=6.0, n_angles=8)
    A = system_matrix(g)
    rng = np.random.default_rng(11)
    ftrue = np.zeros((8, 8, 8))
    ftrue[2:6, 2:6, 2:6] = 0.02
    ftrue[3:5, 3:5, 1:4] += 0.01
    Y = oracle.project(g, ftrue) + rng.normal(scale=0.01, size=(8, 10, 10))
    mu, eps = 0.5, 2e-3
    gam = 2 * mu * 512 / (8 * 100)

    def obj(x):
        t = torch.tensor(x.reshape(8, 8, 8), requires_grad=True, dtype=torch.float64)
        dz = torch.nn.functional.pad(torch.diff(t, dim=0), (0, 0, 0, 0, 0, 1)) / 4.0
        dy = torch.nn.functional.pad(torch.diff(t, dim=1), (0, 0, 0, 1)) / 4.0
        dx = torch.nn.functional.pad(torch.diff(t, dim=2), (0, 1)) / 4.0
        r = torch.tensor(A) @ t.reshape(-1) - torch.tensor(Y.ravel())
        val = torch.sqrt(dx * dx + dy * dy + dz * dz + eps * eps).sum() + 0.5 * gam * (r * r).sum()
        val.backward()
        return val.item(), t.grad.numpy().ravel().copy()

    res = minimize(obj, np.zeros(512), jac=True, method="L-BFGS-B", bounds=[(0, None)] * 512,
                   options=dict(maxiter=20000, ftol=1e-16, gtol=1e-13, maxcor=30))
    beta = oracle.auto_beta(g, mu)
    f, _ = oracle.fbs(g, Y, mu, beta, eps, 50, 1500)
    fo = res.x.reshape(8, 8, 8)
    assert np.linalg.norm(f - fo) / np.linalg.norm(fo) < 1e-5
    # the V-cycle (8^3 over 4^3) has the same minimiser
    fv, tr, acc = oracle.vcycle(g, Y, mu, 400, 2, eps=eps, M=50, pre=2, post=2, coarse=5)
    assert np.linalg.norm(fv - fo) / np.linalg.norm(fo) < 1e-5
    assert acc[0] >= 1
    assert obj(f.ravel())[0] <= res.fun * (1 + 1e-9)


def test_power_start_generator_matches_published_vectors():
    """The power iteration's start volume comes from SplitMix64 used as a counter-based
    generator (value i of seed s = output i + 1 of the generator started at state s);
    pinned to the generator's published test vectors."""
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    for v in ref["vectors"]:
        got = [f"{oracle.splitmix64(v['seed'], i):016x}" for i in range(len(v["outputs"]))]
        assert got == v["outputs"], (v["seed"], got)
    # uniform(0,1) from the top 24 bits: exact multiples of 2^-24, mean 1/2, variance 1/12
    u = np.array([oracle.uniform01(oracle.POWER_SEED, i) for i in range(100000)])
    assert np.all((u >= 0) & (u < 1)) and np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    assert u[0] == (oracle.splitmix64(oracle.POWER_SEED, 0) >> 40) / 2 ** 24
    n = u.size
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * np.sqrt(1 / 180 / n)


def test_power_iteration_bounds_spectrum():
    """lambda_hat from 30 power iterations is within 1% below the largest eigenvalue
    of A^T A (numpy eigvalsh on the dense matrix)."""
    g = tiny_geometry()
    A = system_matrix(g)
    lmax = np.linalg.eigvalsh(A.T @ A)[-1]
    lam = oracle.power_iteration(g, 30)
    assert lam <= lmax * (1 + 1e-12) and lam >= 0.99 * lmax


# ---------------------------------------------------------------------------------
# Multigrid transfers and the cascade
# ---------------------------------------------------------------------------------

def test_prolongation_reproduces_constants_and_linears():
    fc = np.full((3, 4, 5), 0.25)
    assert np.abs(oracle.prolong_vol(fc, (6, 8, 10)) - 0.25).max() <= 1e-16
    # linear function sampled at coarse cell centres -> exact at fine interior centres
    nz, ny, nx = 6, 8, 10
    kc, jc, ic = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    lin = lambda x, y, z: 0.3 * x - 0.7 * y + 1.1 * z + 2.0  # noqa: E731
    fcl = lin((ic - 2.0) * 2, (jc - 1.5) * 2, (kc - 1.0) * 2)
    f = oracle.prolong_vol(fcl, (nz, ny, nx))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = lin(i - 4.5, j - 3.5, k - 2.5)
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(f[inner] - ref[inner]).max() <= 1e-13


def test_restriction_is_block_mean():
    rng = np.random.default_rng(12)
    y = rng.normal(size=(3, 7, 9))
    yc = oracle.restrict_sino(y)
    assert yc.shape == (3, 4, 5)
    assert abs(yc[1, 2, 3] - y[1, 4:6, 6:8].mean()) <= 1e-15
    assert abs(yc[2, 3, 4] - y[2, 6, 8]) <= 1e-15           # corner bin: one pixel
    assert abs(yc[0, 3, 1] - y[0, 6, 2:4].mean()) <= 1e-15  # edge bin: two pixels


def test_single_level_cascade_equals_fbs():
    case = synth.make_case("small")
    g = case["geom"]
    beta = 1.4e6      # above 1.05 gamma lambda_max for this workload
    eps = oracle.default_eps(g)
    f1, tr1 = oracle.reconstruct(g, case["Y"], case["mu"], 4, 1, betas=[beta], M=5)
    f2, tr2 = oracle.fbs(g, case["Y"], case["mu"], beta, eps, 5, 4)
    assert np.array_equal(f1, f2)
    assert np.array_equal(tr1[0], tr2)


def test_two_level_cascade_runs_and_descends():
    case = synth.make_case("small")
    g = case["geom"]
    f, tr = oracle.reconstruct(g, case["Y"], case["mu"], 5, 2, M=5)
    assert f.shape == (64, 64, 64) and (f >= 0).all()
    assert np.all(np.diff(tr[0, :, 0]) <= 1e-12 * tr[0, :-1, 0])
    assert np.all(np.diff(tr[1, :, 0]) <= 1e-12 * tr[1, :-1, 0])
    lg = oracle.level_geom(g, 1)
    assert (lg["nx"], lg["nu"], lg["nv"], lg["hx"], lg["du"]) == (32, 32, 24, 8.0, 16.0)


def _cascade_by_hand(g, Y, mu, iters, levels, betas, M, start_zero=False, wrong_data=False):
    """The coarse-to-fine cascade (multigrid sentence after Eq. 2) composed from its
    separately pinned parts: 2x2 binning of the data per level, Algorithm A1 on each
    level, trilinear prolongation to the next finer level, starting from 0 on the
    coarsest.  start_zero / wrong_data plant the two wiring mistakes the cascade must
    not make (a finer level restarted from 0, a coarse level fed decimated instead of
    binned data)."""
    Ys = [np.asarray(Y, dtype=np.float64)]
    for _ in range(1, levels):
        Ys.append(oracle.restrict_sino(Ys[-1]))
    lg = [oracle.level_geom(g, l) for l in range(levels)]
    f, traces = None, []
    for l in range(levels - 1, -1, -1):
        shape = oracle.vol_shape(lg[l])
        f0 = np.zeros(shape) if (f is None or start_zero) else oracle.prolong_vol(f, shape)
        # a plausible wiring slip: decimating the finer data instead of binning it
        data = Ys[l - 1][:, ::2, ::2].copy() if (wrong_data and l > 0) else Ys[l]
        eps = oracle.default_eps(lg[l])
        f, tr = oracle.fbs(lg[l], data, mu, betas[l], eps, M, iters, f0=f0)
        traces.append((l, f0, tr))
    return f, traces


@pytest.mark.parametrize("levels", [2, 3])
def test_cascade_wiring_matches_composed_parts(levels):
    """or_reconstruct is bitwise the composition of restriction, A1 and prolongation in
    the cascade's order; a finer level restarted from 0, or a level fed the wrong data,
    gives another volume; the finer level's first trace energy is the energy of the
    prolonged coarse result."""
    case = synth.make_case("small")
    g, Y, mu = case["geom"], case["Y"], case["mu"]
    iters, M = 3, 4
    betas = [1.05 * oracle.gamma(oracle.level_geom(g, l), mu) * 1.3e4 / 4 ** l for l in range(levels)]
    f_rec, tr_rec = oracle.reconstruct(g, Y, mu, iters, levels, betas=betas, M=M)
    f_hand, traces = _cascade_by_hand(g, Y, mu, iters, levels, betas, M)
    assert np.array_equal(f_rec, f_hand)
    # trace entries, coarsest level first in or_reconstruct
    for q, (l, f0, tr) in enumerate(traces):
        np.testing.assert_allclose(tr_rec[q], tr, rtol=1e-12, atol=0)
        if l < levels - 1:
            lgl = oracle.level_geom(g, l)
            Yl = np.asarray(Y, dtype=np.float64)
            for _ in range(l):
                Yl = oracle.restrict_sino(Yl)
            E0 = oracle.energy(lgl, Yl, f0, mu, oracle.default_eps(lgl))
            assert abs(tr_rec[q][0, 0] - E0[0]) <= 1e-12 * abs(E0[0])
            assert np.abs(f0).max() > 0    # the finer level starts from the coarse result
    f_zero, _ = _cascade_by_hand(g, Y, mu, iters, levels, betas, M, start_zero=True)
    f_data, _ = _cascade_by_hand(g, Y, mu, iters, levels, betas, M, wrong_data=True)
    scale = np.linalg.norm(f_rec)
    assert np.linalg.norm(f_zero - f_rec) > 1e-6 * scale
    assert np.linalg.norm(f_data - f_rec) > 1e-6 * scale


# ---------------------------------------------------------------------------------
# Synthetic data (inputs only)
# ---------------------------------------------------------------------------------

def test_poisson_noise_statistics():
    rng = np.random.default_rng(13)
    Y = np.full(200000, 1.5)
    I0 = 1e4
    N = np.exp(-synth.poisson_log(Y, I0, rng)) * I0
    lam = I0 * math.exp(-1.5)
    assert abs(N.mean() - lam) < 3 * math.sqrt(lam / N.size)
    assert abs(N.var() / lam - 1.0) < 3 * math.sqrt(2.0 / N.size)


# ---------------------------------------------------------------------------------
# V-cycle: a full-approximation (coarse model with a first-order correction) reading
# of the multigrid method the paper cites
# ---------------------------------------------------------------------------------

def test_prolongation_adjoint_is_the_transpose():
    rng = np.random.default_rng(70)
    for fine, coarse in [((7, 9, 10), (4, 5, 5)), ((8, 8, 8), (4, 4, 4))]:
        x = rng.normal(size=coarse)
        y = rng.normal(size=fine)
        lhs = float(np.sum(oracle.prolong_vol(x, fine) * y))
        rhs = float(np.sum(x * oracle.prolong_vol_adjoint(y, coarse)))
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * 8


def test_volume_restriction_is_the_block_mean():
    rng = np.random.default_rng(71)
    f = rng.normal(size=(6, 4, 8))
    fc = oracle.restrict_vol(f)
    assert np.allclose(fc, f.reshape(3, 2, 2, 2, 4, 2).mean(axis=(1, 3, 5)), rtol=0, atol=1e-14)
    g = rng.normal(size=(5, 3, 7))        # odd sizes: the edge blocks average what exists
    gc = oracle.restrict_vol(g)
    assert gc.shape == (3, 2, 4)
    assert abs(gc[2, 1, 3] - g[4, 2, 6]) <= 1e-15
    assert abs(gc[0, 1, 3] - g[0:2, 2, 6].mean()) <= 1e-15
    assert np.all(oracle.restrict_vol(np.full((5, 3, 7), 2.5)) == 2.5)


def _tiny_case(seed):
    g = tiny_geometry(n=8, h=4.0, nu=10, nv=10, du=6.0, dv=6.0, n_angles=6)
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.0, 0.02, size=(8, 8, 8))
    Y = oracle.project(g, f) + rng.normal(scale=0.01, size=(6, 10, 10))
    return g, Y, rng


def test_energy_gradient_matches_finite_differences():
    g, Y, rng = _tiny_case(72)
    f = rng.uniform(0.0, 0.03, size=(8, 8, 8))
    mu, eps = 0.7, 3e-3
    gr = oracle.energy_grad(g, Y, f, mu, eps)
    d = 1e-5
    for _ in range(12):
        k, j, i = rng.integers(0, 8, size=3)
        fp, fm = f.copy(), f.copy()
        fp[k, j, i] += d
        fm[k, j, i] -= d
        fd = (oracle.energy(g, Y, fp, mu, eps)[0] - oracle.energy(g, Y, fm, mu, eps)[0]) / (2 * d)
        assert abs(fd - gr[k, j, i]) <= 1e-6 * np.abs(gr).max()


def test_fbs_linear_term_without_tv_is_shifted_landweber():
    """TV weight 0, one inner step: A1 on E - <v, f> is
    f <- max(0, f - (gamma/beta) A^T (A f - Y) + (Nv/beta) v)."""
    g = tiny_geometry()
    A = system_matrix(g)
    rng = np.random.default_rng(73)
    Y = rng.uniform(0, 3, size=(6, 8, 8))
    v = rng.normal(scale=1e-3, size=(8, 8, 8))
    mu, beta = 1.5, 4000.0
    f, _ = oracle.fbs(g, Y, mu, beta, 1e-3, 1, 12, tv_weight=0.0, v=v)
    gam = 2 * mu * 512 / (6 * 64)
    x = np.zeros(512)
    for _ in range(12):
        x = np.maximum(0.0, x - gam / beta * (A.T @ (A @ x - Y.ravel())) + 512 / beta * v.ravel())
    assert np.abs(f.ravel() - x).max() <= 1e-12 * max(1.0, np.abs(x).max())


def test_coarse_model_is_first_order_coherent():
    """The coarse model's gradient at R f, grad E_c(R f) - v_c, equals Q^T grad E(f),
    and Q^T grad E(f) is the derivative of x -> E(f + Q x) (finite differences of the
    fine energy along prolonged coarse unit vectors)."""
    g, Y, rng = _tiny_case(74)
    gc = oracle.level_geom(g, 1)
    Yc = oracle.restrict_sino(Y)
    f = rng.uniform(0.0, 0.03, size=(8, 8, 8))
    mu = 0.7
    eps, epsc = oracle.default_eps(g), oracle.default_eps(gc)
    qt = oracle.prolong_vol_adjoint(oracle.energy_grad(g, Y, f, mu, eps), (4, 4, 4))
    vc = oracle.energy_grad(gc, Yc, oracle.restrict_vol(f), mu, epsc) - qt
    model_grad = oracle.energy_grad(gc, Yc, oracle.restrict_vol(f), mu, epsc) - vc
    assert np.abs(model_grad - qt).max() <= 1e-15 * max(1.0, np.abs(qt).max()) * 100
    d = 1e-5
    for _ in range(6):
        e = np.zeros((4, 4, 4))
        e[tuple(rng.integers(0, 4, size=3))] = 1.0
        q = oracle.prolong_vol(e, (8, 8, 8))
        fd = (oracle.energy(g, Y, f + d * q, mu, eps)[0] - oracle.energy(g, Y, f - d * q, mu, eps)[0]) / (2 * d)
        assert abs(fd - float(np.sum(qt * e))) <= 1e-6 * np.abs(qt).max()


def test_vcycle_decreases_the_energy_faster_than_single_grid():
    case = synth.make_case("small")
    g = case["geom"]
    mu = case["mu"]
    f, tr, acc = oracle.vcycle(g, case["Y"], mu, 4, 2, pre=2, post=2, coarse=10)
    assert np.all(np.diff(tr[:, 0]) < 0) and (f >= 0).all()
    assert acc[0] >= 1                                    # coarse corrections were taken
    beta, eps = oracle.auto_beta(g, mu), oracle.default_eps(g)
    f1, _ = oracle.fbs(g, case["Y"], mu, beta, eps, 10, 16)    # the same fine-level work
    assert tr[-1, 0] < 0.5 * oracle.energy(g, case["Y"], f1, mu, eps)[0]
