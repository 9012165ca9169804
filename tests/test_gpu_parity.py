"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Gates (float32 bulk arithmetic, float64 reductions):
  projections      relative L2 <= 1e-5 and max |diff| <= 1e-5 max |P f|
  adjoint          relative L2 <= 1e-5; GPU adjoint identity <= 1e-6
  volumes after a fixed number of Algorithm A1 iterations: relative L2 <= 1e-4
  f >= 0 exactly (every stored voxel >= +0.0)
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.brute_matrix import tiny_geometry

pytestmark = pytest.mark.gpu

P_TOL = 1e-5
VOL_TOL = 1e-4


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


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def check_projection(lib, geom, f):
    G = lib.cbct_geometry_create(geom)
    y = host(lib.cbct_project(G, dev(f)))
    ref = oracle.project(geom, f32(f))
    assert rel(y, ref) <= P_TOL, rel(y, ref)
    assert np.abs(y - ref).max() <= P_TOL * np.abs(ref).max()
    return y, ref


def ragged_geometry():
    # sizes off every multiple of 32 and odd imager sizes (rays in voxel planes)
    return dict(nx=45, ny=38, nz=37, hx=2.0, hy=2.5, hz=3.0, nu=53, nv=41, du=4.0, dv=4.5,
                dso=400.0, dsd=640.0, angles=2 * math.pi * np.arange(7) / 7 + 0.1)


# ---------------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------------

def test_project_small_random_and_phantom(lib):
    case = synth.make_case("small", with_truth=True, truth_ss=1)
    g = case["geom"]
    rng = np.random.default_rng(20)
    check_projection(lib, g, rng.uniform(size=(64, 64, 64)) * 0.02)
    check_projection(lib, g, case["f_true"])


def test_project_degenerate_and_ragged(lib):
    rng = np.random.default_rng(21)
    g = tiny_geometry(n=8, h=4.0, nu=9, nv=9, du=8.0, dv=8.0, n_angles=4)   # in-plane rays
    check_projection(lib, g, rng.uniform(size=(8, 8, 8)))
    g = ragged_geometry()
    check_projection(lib, g, rng.uniform(size=(37, 38, 45)))


def test_project_medium_full_size(lib):
    g = synth.geometry_for(synth.CONFIGS["medium"])
    rng = np.random.default_rng(22)
    f = rng.uniform(size=(64, 256, 256)) * 0.02
    check_projection(lib, g, f)


def test_project_large_sampled_rays(lib):
    g = synth.geometry_for(synth.CONFIGS["large"])
    rng = np.random.default_rng(23)
    f = (rng.uniform(size=(96, 512, 512)) * 0.02).astype(np.float32)
    G = lib.cbct_geometry_create(g)
    y = host(lib.cbct_project(G, dev(f)))
    f64 = f.astype(np.float64)
    for _ in range(40):
        ia, b, a = rng.integers(0, 40), rng.integers(0, 384), rng.integers(0, 512)
        ref = oracle.project_ray(g, f64, int(ia), int(b), int(a))
        assert abs(y[ia, b, a] - ref) <= P_TOL * max(abs(ref), 1.0), (ia, b, a, y[ia, b, a], ref)
    # every ray through the central column of the volume is non-zero
    assert (y[:, 150:234, 200:312] > 0).all()


def test_project_large_two_full_views(lib):
    # every ray of two whole views (2 x 512 x 384) of the large workload, projected on the
    # GPU with all 40 views and by the oracle with those two views alone
    g = synth.geometry_for(synth.CONFIGS["large"])
    rng = np.random.default_rng(27)
    f = (rng.uniform(size=(96, 512, 512)) * 0.02).astype(np.float32)
    G = lib.cbct_geometry_create(g)
    y = host(lib.cbct_project(G, dev(f)))
    views = [3, 26]   # 27 and 234 degrees: columns in every direction of the xy-grid
    ref = oracle.project(dict(g, angles=g["angles"][views]), f.astype(np.float64))
    got = y[views]
    assert rel(got, ref) <= P_TOL, rel(got, ref)
    assert np.abs(got - ref).max() <= P_TOL * np.abs(ref).max()


def test_projection_split_over_level_launches_is_bitwise_identical(lib):
    """A projection run as consecutive launches over slabs of z-levels (the default for
    volumes larger than the L2 cache) equals the single launch bit for bit, in every
    epilogue: plain projection, the power iteration's scaled one and the residual with
    the E2 partials of an Algorithm A1 iteration."""
    rng = np.random.default_rng(28)
    small = synth.make_case("small")
    for g, shape in ((ragged_geometry(), (37, 38, 45)), (small["geom"], (64, 64, 64))):
        f = rng.uniform(size=shape) * 0.02
        G = lib.cbct_geometry_create(g)
        fd = dev(f)
        n0 = lib.cbct_kernel_launch_count()
        y0 = host(lib.cbct_project(G, fd))
        single = lib.cbct_kernel_launch_count() - n0
        for levels in (1, 5, 32):
            lib.cbct_set_tuning(G, 0, {"proj_levels": levels})
            n0 = lib.cbct_kernel_launch_count()
            assert np.array_equal(host(lib.cbct_project(G, fd)), y0), levels
            # the launch counter sees one projector launch per slab of levels
            assert lib.cbct_kernel_launch_count() - n0 == single - 1 + -(-shape[0] // levels)
        lib.cbct_set_tuning(G, 0, {})
    g = small["geom"]
    Y = f32(small["Y"])
    runs = []
    for levels in (0, 7):
        G = lib.cbct_geometry_create(g)
        lib.cbct_set_tuning(G, 0, {"proj_levels": levels})
        lam = lib.cbct_power_iteration(G, 5)
        f, tr, st = lib.cbct_fbs(G, dev(Y), small["mu"], 1.05 * oracle.gamma(g, small["mu"]) * lam, 1e-3, 10, 0, 3,
                                 dev(np.zeros((64, 64, 64))), trace=True, step_trace=True)
        runs.append((lam, host(f), tr, st))
    assert runs[0][0] == runs[1][0]
    for a, b in zip(runs[0][1:], runs[1][1:]):
        assert np.array_equal(a, b)


def tall_geometry():
    # 600 imager rows: more than one 512-thread projector tile per detector column, and
    # thick voxels (several rows per voxel) against thin rows
    return dict(nx=24, ny=20, nz=40, hx=3.0, hy=3.0, hz=6.0, nu=30, nv=600, du=4.0, dv=0.6,
                dso=500.0, dsd=800.0, angles=2 * math.pi * np.arange(6) / 6 + 0.37)


def test_tall_imager_project_and_backproject(lib):
    g = tall_geometry()
    rng = np.random.default_rng(27)
    check_projection(lib, g, rng.uniform(size=(40, 20, 24)))
    G = lib.cbct_geometry_create(g)
    y = rng.normal(size=(6, 600, 30))
    bt = host(lib.cbct_backproject(G, dev(y)))
    ref = oracle.backproject(g, f32(y))
    assert rel(bt, ref) <= P_TOL, rel(bt, ref)


# ---------------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------------

def test_backproject_small_and_ragged(lib):
    rng = np.random.default_rng(24)
    for g in (synth.geometry_for(synth.CONFIGS["small"]), ragged_geometry(),
              tiny_geometry(n=8, h=4.0, nu=9, nv=9, du=8.0, dv=8.0, n_angles=4)):
        G = lib.cbct_geometry_create(g)
        y = rng.normal(size=(len(g["angles"]), g["nv"], g["nu"]))
        bt = host(lib.cbct_backproject(G, dev(y)))
        ref = oracle.backproject(g, f32(y))
        assert rel(bt, ref) <= P_TOL, rel(bt, ref)


def test_backproject_lane_layouts_agree_bitwise(lib):
    """The adjoint's two lane layouts (consecutive and interleaved voxels per lane) and
    every voxels-per-lane count give the same bits, and match the oracle."""
    rng = np.random.default_rng(23)
    for g in (synth.geometry_for(synth.CONFIGS["small"]), ragged_geometry(), tall_geometry()):
        G = lib.cbct_geometry_create(g)
        y = dev(rng.normal(size=(len(g["angles"]), g["nv"], g["nu"])))
        ref = oracle.backproject(g, f32(host(y)))
        first = None
        for vpl in range(1, min(4, (g["nz"] + 31) // 32) + 1):
            for layout in (1, 2):
                lib.cbct_set_tuning(G, 0, {"bp_vpl": vpl, "bp_layout": layout})
                bt = host(lib.cbct_backproject(G, y))
                if first is None:
                    first = bt
                    assert rel(bt, ref) <= P_TOL, rel(bt, ref)
                assert np.array_equal(bt, first), (g["nz"], vpl, layout)
        with pytest.raises(lib.CbctError):
            lib.cbct_set_tuning(G, 0, {"bp_layout": 3})


def test_backproject_medium_full_size(lib):
    g = synth.geometry_for(synth.CONFIGS["medium"])
    rng = np.random.default_rng(25)
    y = rng.normal(size=(40, 192, 256))
    G = lib.cbct_geometry_create(g)
    bt = host(lib.cbct_backproject(G, dev(y)))
    ref = oracle.backproject(g, f32(y))
    assert rel(bt, ref) <= P_TOL, rel(bt, ref)


def test_backproject_large_sampled_voxels(lib):
    g = synth.geometry_for(synth.CONFIGS["large"])
    rng = np.random.default_rng(26)
    y = rng.normal(size=(40, 384, 512)).astype(np.float32)
    G = lib.cbct_geometry_create(g)
    bt = host(lib.cbct_backproject(G, dev(y)))
    y64 = y.astype(np.float64)
    scale = np.abs(bt).max()
    for _ in range(12):
        i, j, k = rng.integers(0, 512), rng.integers(0, 512), rng.integers(0, 96)
        ref = oracle.backproject_voxel(g, y64, int(i), int(j), int(k))
        assert abs(bt[k, j, i] - ref) <= P_TOL * scale, (i, j, k, bt[k, j, i], ref)


def test_backproject_large_central_slab(lib):
    # every voxel of the 4 central z-levels of 512x512x96 from the full large imager (40
    # views of 512x384): a volume of nz = 4 has the same voxel centres as levels 46-49, and
    # a voxel's adjoint value depends on that voxel's intersections alone.
    # Gated on positive data.  Each float32 intersection length is a difference of plane
    # crossings up to 181 mm from the ray's foot, so it carries an absolute error of a few
    # 1e-5 mm (a few 1e-5 of a 0.5 mm chord), more for the nearly horizontal rays of the
    # central levels, which graze the z-planes.  In a sum of positive terms these errors
    # average out below the gate; zero-mean data (normal, printed) cancel the sum itself
    # and leave them at about 1.5e-5 of its norm.  The largest single deviation, at voxels
    # next to the z = 0 plane that the central rows' rays graze, is printed too.
    g = synth.geometry_for(synth.CONFIGS["large"])
    rng = np.random.default_rng(28)
    G = lib.cbct_geometry_create(g)
    slab = dict(g, nz=4)
    y = rng.uniform(0.5, 1.5, size=(40, 384, 512)).astype(np.float32)
    got = host(lib.cbct_backproject(G, dev(y)))[46:50]
    ref = oracle.backproject(slab, y.astype(np.float64))
    assert rel(got, ref) <= P_TOL, rel(got, ref)   # the adjoint's gate (relative L2)
    print(f"large central slab: max |diff| / max |P^T y| = {np.abs(got - ref).max() / np.abs(ref).max():.1e}")
    yn = rng.normal(size=(40, 384, 512)).astype(np.float32)
    gn = host(lib.cbct_backproject(G, dev(yn)))[46:50]
    print(f"large central slab, zero-mean data: rel L2 {rel(gn, oracle.backproject(slab, yn.astype(np.float64))):.2e}")


def test_gpu_adjoint_identity(lib):
    for g in (synth.geometry_for(synth.CONFIGS["small"]), ragged_geometry()):
        G = lib.cbct_geometry_create(g)
        rng = np.random.default_rng(27)
        f = rng.uniform(size=(g["nz"], g["ny"], g["nx"]))
        y = rng.normal(size=(len(g["angles"]), g["nv"], g["nu"]))
        Pf = host(lib.cbct_project(G, dev(f)))
        PTy = host(lib.cbct_backproject(G, dev(y)))
        lhs, rhs = float(np.sum(Pf * f32(y))), float(np.sum(f32(f) * PTy))
        assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(Pf) * np.linalg.norm(y)


# ---------------------------------------------------------------------------------
# TV prox, energies, step size
# ---------------------------------------------------------------------------------

def test_tv_prox_matches_oracle(lib):
    g = synth.geometry_for(synth.CONFIGS["small"])
    case = synth.make_case("small", with_truth=True, truth_ss=1)
    rng = np.random.default_rng(28)
    f0 = case["f_true"]
    gv = f0 + rng.normal(scale=0.004, size=f0.shape)
    eps = oracle.default_eps(g)
    beta = 2.0e5
    G = lib.cbct_geometry_create(g)
    ft = dev(f0)
    lib.cbct_tv_prox(G, dev(gv), ft, beta, eps, 10)
    out = host(ft)
    ref = oracle.prox(f32(gv), f32(f0), (4.0, 4.0, 4.0), beta, eps, 10)
    assert (out >= 0).all() and not np.signbit(out).any()
    d_ref = ref - f32(f0)
    assert np.linalg.norm((out - f32(f0)) - d_ref) <= 1e-4 * np.linalg.norm(d_ref)


@pytest.mark.parametrize("dims,form", [((29, 206, 160), "full columns, 1 voxel per lane"),
                                       ((45, 206, 163), "full columns, 2 voxels per lane, odd nx"),
                                       ((70, 256, 180), "full columns, 3 voxels per lane"),
                                       ((100, 256, 128), "32-voxel row walks")])
@pytest.mark.parametrize("tv_mode", [0, 1])
def test_tv_prox_sweep_forms_match_oracle(lib, dims, form, tv_mode):
    """The warp-tile forms of the prox sweep on ragged sizes (a partly filled z-slot or
    z-block, a last walk of fewer rows) against the oracle's prox."""
    nz, ny, nx = dims
    g = dict(nx=nx, ny=ny, nz=nz, hx=1.0, hy=1.25, hz=2.0, nu=16, nv=16, du=30.0, dv=30.0, dso=800.0,
             dsd=1200.0, angles=np.array([0.0, 1.0]))
    rng = np.random.default_rng(31)
    f0 = np.clip(rng.normal(0.01, 0.006, size=dims), 0.0, None)
    gv = f0 + rng.normal(scale=0.003, size=dims)
    eps, beta = 1e-3, 5.0e3
    G = lib.cbct_geometry_create(g)
    ft = dev(f0)
    lib.cbct_tv_prox(G, dev(gv), ft, beta, eps, 10, tv_mode=tv_mode)
    out = host(ft)
    ref = oracle.prox(f32(gv), f32(f0), (1.0, 1.25, 2.0), beta, eps, 10, tv_mode=tv_mode)
    assert (out >= 0).all() and not np.signbit(out).any()
    d_ref = ref - f32(f0)
    assert np.linalg.norm((out - f32(f0)) - d_ref) <= 1e-4 * np.linalg.norm(d_ref), form


def test_energy_and_power_iteration(lib):
    case = synth.make_case("small")
    g = case["geom"]
    rng = np.random.default_rng(29)
    f = rng.uniform(size=(64, 64, 64)) * 0.02
    eps = oracle.default_eps(g)
    G = lib.cbct_geometry_create(g)
    E = lib.cbct_energy(G, dev(case["Y"]), dev(f), case["mu"], eps)
    ref = oracle.energy(g, f32(case["Y"]), f32(f), case["mu"], eps)
    assert np.all(np.abs(E - ref) <= 1e-5 * np.abs(ref))
    lam = lib.cbct_power_iteration(G, 30)
    lam_ref = oracle.power_iteration(g, 30)
    assert abs(lam - lam_ref) <= 1e-5 * lam_ref
    # one iteration: the Rayleigh quotient of the seeded start volume itself, so both
    # sides must draw the same start (counter-based generator, same voxel order)
    lam1, lam1_ref = lib.cbct_power_iteration(G, 1), oracle.power_iteration(g, 1)
    assert abs(lam1 - lam1_ref) <= 1e-5 * lam1_ref and lam1 < lam
    # eps = 0: the unsmoothed TV, E1 = sum |grad f| / Nv, in both readings; a piecewise
    # constant volume has exactly flat voxels, where the smoothed and exact terms differ most
    fp = np.where(f > 0.01, 0.02, 0.0)
    for tv_mode in (0, 1):
        for vol in (f, fp):
            E0 = lib.cbct_energy(G, dev(case["Y"]), dev(vol), case["mu"], 0.0, tv_mode=tv_mode)
            ref0 = oracle.energy(g, f32(case["Y"]), f32(vol), case["mu"], 0.0, tv_mode=tv_mode)
            assert np.all(np.abs(E0 - ref0) <= 1e-5 * np.abs(ref0)), (tv_mode, E0, ref0)
    with pytest.raises(lib.CbctError):
        lib.cbct_energy(G, dev(case["Y"]), dev(f), case["mu"], -1.0)


# ---------------------------------------------------------------------------------
# Algorithm A1 and the multigrid cascade
# ---------------------------------------------------------------------------------

def test_fbs_small_20_iterations(lib):
    case = synth.make_case("small")
    g = case["geom"]
    mu, eps = case["mu"], oracle.default_eps(g)
    beta = 1.05 * oracle.gamma(g, mu) * oracle.power_iteration(g, 30)
    Y = f32(case["Y"])
    f_ref, tr_ref, st_ref = oracle.fbs(g, Y, mu, beta, eps, 10, 20, steps=True)
    G = lib.cbct_geometry_create(g)
    ft = dev(np.zeros((64, 64, 64)))
    ft, tr, st = lib.cbct_fbs(G, dev(Y), mu, beta, eps, 10, 0, 20, ft, trace=True, step_trace=True)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert (f >= 0).all() and not np.signbit(f).any()
    assert np.all(np.abs(tr - tr_ref) <= 1e-4 * np.abs(tr_ref))
    assert np.all(np.diff(tr[:, 0]) <= 1e-6 * tr[:-1, 0])
    # |f_k+1 - f_k|: both iterates carry the volume tolerance, so the difference of two
    # steps is within 2 VOL_TOL |f| on top of the float32 rounding of the step itself
    assert np.all(np.abs(st - st_ref) <= 1e-4 * st_ref + 2 * VOL_TOL * np.linalg.norm(f_ref)), (st, st_ref)


def test_fbs_paper_literal_clamp_mode(lib):
    case = synth.make_case("small")
    g = case["geom"]
    mu, eps = case["mu"], oracle.default_eps(g)
    beta = 1.05 * oracle.gamma(g, mu) * oracle.power_iteration(g, 30)
    Y = f32(case["Y"])
    f_ref, tr_ref, st_ref = oracle.fbs(g, Y, mu, beta, eps, 10, 10, clamp_mode=1, steps=True)
    G = lib.cbct_geometry_create(g)
    ft, tr, st = lib.cbct_fbs(G, dev(Y), mu, beta, eps, 10, 1, 10, dev(np.zeros((64, 64, 64))), trace=True,
                              step_trace=True)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert (f >= 0).all()
    assert np.all(np.abs(tr - tr_ref) <= 1e-4 * np.abs(tr_ref))
    assert np.all(np.abs(st - st_ref) <= 1e-4 * st_ref + 2 * VOL_TOL * np.linalg.norm(f_ref)), (st, st_ref)


def test_reconstruct_two_levels_small(lib):
    case = synth.make_case("small")
    g = case["geom"]
    mu = case["mu"]
    betas = [1.05 * oracle.gamma(oracle.level_geom(g, l), mu) * oracle.power_iteration(oracle.level_geom(g, l), 30)
             for l in range(2)]
    Y = f32(case["Y"])
    f_ref, tr_ref = oracle.reconstruct(g, Y, mu, 8, 2, betas=betas, M=10)
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, betas=betas, trace=True)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert (f >= 0).all()
    assert np.all(np.abs(info["trace"] - tr_ref) <= 1e-4 * np.abs(tr_ref))


def test_reconstruct_auto_beta_matches_oracle(lib):
    case = synth.make_case("small")
    g = case["geom"]
    Y = f32(case["Y"])
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), case["mu"], 4, 2, trace=True)
    for l in range(2):
        lg = oracle.level_geom(g, l)
        ref = max(10 * case["mu"], 1.05 * oracle.gamma(lg, case["mu"]) * oracle.power_iteration(lg, 30))
        assert abs(info["betas"][l] - ref) <= 1e-5 * ref
    f_ref, _ = oracle.reconstruct(g, Y, case["mu"], 4, 2, betas=info["betas"])
    assert rel(host(ft), f_ref) <= VOL_TOL


def test_cascade_power_iterations_on_the_side_stream(lib):
    """With the automatic beta the finer levels' power iterations run on a side stream
    while the coarser levels iterate: the volume equals, bit for bit, the run with the
    same betas passed in (no power iteration at all), and the betas match the oracle."""
    case = synth.make_case("small")
    g = case["geom"]
    Y = dev(case["Y"])
    for levels in (2, 3):
        G = lib.cbct_geometry_create(g)
        fa, ia = lib.cbct_reconstruct(G, Y, case["mu"], 4, levels, trace=True)
        G2 = lib.cbct_geometry_create(g)
        fb, ib = lib.cbct_reconstruct(G2, Y, case["mu"], 4, levels, betas=list(ia["betas"]), trace=True)
        assert np.array_equal(host(fa), host(fb)) and np.array_equal(ia["trace"], ib["trace"])
        G3 = lib.cbct_geometry_create(g)   # the power iterations in level order on one stream
        fc, ic = lib.cbct_reconstruct(G3, Y, case["mu"], 4, levels, trace=True, serial_power=True)
        assert np.array_equal(host(fa), host(fc)) and np.array_equal(ia["betas"], ic["betas"])
        for l in range(levels):
            lg = oracle.level_geom(g, l)
            ref = max(10 * case["mu"], 1.05 * oracle.gamma(lg, case["mu"]) * oracle.power_iteration(lg, 30))
            assert abs(ia["betas"][l] - ref) <= 1e-5 * ref, (levels, l)


def test_medium_one_iteration_full_size(lib):
    """One Algorithm A1 iteration at the full 256x256x64 / 40x256x192 size, from an
    iterate produced by the GPU's own multigrid run (the benchmark configuration)."""
    case = synth.make_case("medium")
    g = case["geom"]
    mu = case["mu"]
    Y = f32(case["Y"])
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), mu, 5, 2, trace=True)
    f_k = host(ft)
    assert (f_k >= 0).all()
    for l in range(2):
        E = info["trace"][l, :, 0]
        assert np.all(np.diff(E) <= 1e-5 * E[:-1])
    beta = float(info["betas"][0])
    eps = oracle.default_eps(g)
    f1t, st = lib.cbct_fbs(G, dev(Y), mu, beta, eps, 10, 0, 1, dev(f_k), step_trace=True)
    f1 = host(f1t)
    f1_ref, _, st_ref = oracle.fbs(g, Y, mu, beta, eps, 10, 1, f0=f_k, steps=True)
    step_ref = f1_ref - f_k
    assert np.linalg.norm((f1 - f_k) - step_ref) <= 1e-3 * np.linalg.norm(step_ref)
    assert rel(f1, f1_ref) <= 1e-5
    # the reported step norm is that of the GPU's own two iterates, and the oracle's
    assert abs(st[0] - np.linalg.norm(f1.astype(np.float64) - f_k)) <= 1e-5 * st[0]
    assert abs(st[0] - st_ref[0]) <= 1e-3 * st_ref[0]


def test_multigrid_transfers(lib):
    rng = np.random.default_rng(30)
    y = rng.normal(size=(3, 37, 53))
    yc = host(lib.cbct_restrict_sino(dev(y)))
    assert np.abs(yc - oracle.restrict_sino(f32(y))).max() <= 1e-6
    fc = rng.uniform(size=(5, 7, 9))
    f = host(lib.cbct_prolong_vol(dev(fc), (10, 13, 18)))
    assert np.abs(f - oracle.prolong_vol(f32(fc), (10, 13, 18))).max() <= 1e-6


# ---------------------------------------------------------------------------------
# variants, determinism, resume, timing
# ---------------------------------------------------------------------------------

def test_fp16_sinogram_variant_error_reported(lib):
    case = synth.make_case("small")
    g = case["geom"]
    Y = f32(case["Y"])
    G = lib.cbct_geometry_create(g)
    betas = [1.4e6]
    f16 = host(lib.cbct_reconstruct(G, dev(Y), case["mu"], 10, 1, betas=betas, sino_fp16=True))
    f_ref, _ = oracle.reconstruct(g, Y, case["mu"], 10, 1, betas=betas)
    err = rel(f16, f_ref)
    print(f"fp16 sinogram storage: relative L2 error vs FP64 oracle = {err:.3e}")
    assert err < 1e-2 and (f16 >= 0).all()


def test_deterministic_and_graphs_identical(lib, cuda):
    torch = cuda
    case = synth.make_case("small")
    G = lib.cbct_geometry_create(case["geom"])
    Y = dev(case["Y"])
    runs = [host(lib.cbct_reconstruct(G, Y, case["mu"], 6, 2)) for _ in range(2)]
    assert np.array_equal(runs[0], runs[1])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fg = lib.cbct_reconstruct(G, Y, case["mu"], 6, 2, use_graphs=True)
    s.synchronize()
    assert np.array_equal(host(fg), runs[0])


def test_resume_from_checkpoint(lib):
    case = synth.make_case("small")
    G = lib.cbct_geometry_create(case["geom"])
    Y = dev(case["Y"])
    full = host(lib.cbct_reconstruct(G, Y, case["mu"], 6, 1, beta=1.4e6))
    half = lib.cbct_reconstruct(G, Y, case["mu"], 3, 1, beta=1.4e6)
    rest = host(lib.cbct_reconstruct(G, Y, case["mu"], 3, 1, beta=1.4e6, f_init=half, start_level=0))
    assert np.array_equal(full, rest)


def test_kernel_timing_report(lib):
    case = synth.make_case("small")
    G = lib.cbct_geometry_create(case["geom"])
    f, info = lib.cbct_reconstruct(G, dev(case["Y"]), case["mu"], 3, 2, kernel_times=True)
    ms, n = info["kernel_ms"], info["kernel_launches"]
    # kernels per class: one projector launch per projection (the volume fits in L2), the
    # column running sums and the gather per adjoint, one launch per prox sweep
    assert n["project"] == 2 * (3 + 30) and n["backproject"] == 2 * 2 * (3 + 30)
    assert n["tv"] == 2 * 3 * 10
    assert all(ms[k] > 0 for k in ("project", "backproject", "tv"))
    # the finest level's Algorithm A1 iterations alone: 3 projections, 3 adjoints
    nf, msf = info["kernel_launches_finest"], info["kernel_ms_finest"]
    assert nf["project"] == 3 and nf["backproject"] == 2 * 3 and nf["tv"] == 3 * 10
    assert all(0 < msf[k] < ms[k] for k in ("project", "backproject", "tv"))
    # a class mask times only the chosen classes and still counts every launch
    mask = 1 << lib.KERNEL_CLASSES.index("backproject")
    _, m = lib.cbct_reconstruct(G, dev(case["Y"]), case["mu"], 3, 2, kernel_times=True, kernel_mask=mask)
    assert m["kernel_launches"] == n
    assert m["kernel_ms"]["backproject"] > 0 and m["kernel_ms"]["tv"] == 0 and m["kernel_ms"]["project"] == 0


@pytest.mark.parametrize("g", [
    dict(nx=1, ny=1, nz=1, hx=2.0, hy=2.0, hz=2.0, nu=1, nv=1, du=3.0, dv=3.0, dso=100.0, dsd=150.0,
         angles=np.array([0.3])),                                   # one voxel, one ray
    dict(nx=2, ny=3, nz=1, hx=1.5, hy=2.0, hz=2.5, nu=5, nv=1, du=1.2, dv=4.0, dso=120.0, dsd=200.0,
         angles=2 * math.pi * np.arange(3) / 3 + 0.1),              # one slice, one imager row
    dict(nx=1, ny=1, nz=40, hx=3.0, hy=3.0, hz=1.0, nu=1, nv=50, du=5.0, dv=1.3, dso=150.0, dsd=250.0,
         angles=np.array([0.0, 1.7])),                              # one column, one imager column
])
def test_degenerate_sizes_match_oracle(lib, g):
    """Single voxels, single imager rows and columns: projection, adjoint, one prox and
    two Algorithm A1 iterations against the oracle."""
    rng = np.random.default_rng(33)
    shape, sshape = (g["nz"], g["ny"], g["nx"]), (len(g["angles"]), g["nv"], g["nu"])
    f = rng.uniform(0.0, 0.02, size=shape)
    y = rng.uniform(0.0, 1.0, size=sshape)
    G = lib.cbct_geometry_create(g)
    p_ref = oracle.project(g, f32(f))
    p_gpu = host(lib.cbct_project(G, dev(f)))
    assert np.abs(p_gpu - p_ref).max() <= P_TOL * max(np.abs(p_ref).max(), 1e-30)
    b_ref = oracle.backproject(g, f32(y))
    b_gpu = host(lib.cbct_backproject(G, dev(y)))
    assert np.abs(b_gpu - b_ref).max() <= P_TOL * max(np.abs(b_ref).max(), 1e-30)
    h = (g["hx"], g["hy"], g["hz"])
    gv = f + rng.normal(scale=0.002, size=shape)
    ft = dev(f)
    lib.cbct_tv_prox(G, dev(gv), ft, 1.0e4, 1e-3, 5)
    ref = oracle.prox(f32(gv), f32(f), h, 1.0e4, 1e-3, 5)
    assert np.abs(host(ft) - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-30)
    Y = f32(oracle.project(g, f32(f))) * 1.1
    beta = 2.0 * max(1.0, oracle.gamma(g, 1.0) * oracle.power_iteration(g, 30))
    f_ref, tr_ref = oracle.fbs(g, Y, 1.0, beta, 1e-3, 10, 2)
    fg, tr = lib.cbct_fbs(G, dev(Y), 1.0, beta, 1e-3, 10, 0, 2, dev(np.zeros(shape)), trace=True)
    fg = host(fg)
    assert (fg >= 0).all() and np.abs(fg - f_ref).max() <= VOL_TOL * max(np.abs(f_ref).max(), 1e-30)
    assert np.all(np.abs(tr - tr_ref) <= 1e-4 * np.abs(tr_ref) + 1e-12)


def test_zero_iterations_and_zero_data(lib):
    """iters = 0 returns the start (zero) volume and an empty trace; zero data keep the
    iterate at exactly +0.0 (every gradient vanishes there)."""
    case = synth.make_case("small")
    g = case["geom"]
    G = lib.cbct_geometry_create(g)
    f, info = lib.cbct_reconstruct(G, dev(case["Y"]), case["mu"], 0, 2, betas=[1.0e6, 1.0e6], trace=True)
    f = host(f)
    assert np.all(f == 0) and not np.signbit(f).any() and info["trace"].shape == (2, 0, 3)
    fz, tr = lib.cbct_fbs(G, dev(np.zeros((20, 48, 64))), case["mu"], 1.0e6, 1e-3, 10, 0, 3,
                          dev(np.zeros((64, 64, 64))), trace=True)
    fz = host(fz)
    assert np.all(fz == 0) and not np.signbit(fz).any()
    assert np.all(tr[:, 2] == 0) and np.allclose(tr[:, 1], 1e-3, rtol=1e-6)   # E1 = eps, mu E2 = 0


def test_invalid_arguments_on_device(lib):
    case = synth.make_case("small")
    G = lib.cbct_geometry_create(case["geom"])
    Y = dev(case["Y"])
    with pytest.raises(lib.CbctError) as e:
        lib.cbct_reconstruct(G, Y, case["mu"], 2, 8)      # 2^7 > 48 detector rows
    assert e.value.status == 1
    with pytest.raises(lib.CbctError):
        lib.cbct_reconstruct(G, Y, -1.0, 2, 1)
    with pytest.raises(lib.CbctError):
        lib.cbct_fbs(G, Y, 1.0, 0.0, 1e-5, 10, 0, 2, dev(np.zeros((64, 64, 64))))
