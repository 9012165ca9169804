"""Parity of the paper-literal variants of Algorithm A1 with the FP64 oracle.

* anisotropic reading of E1 (tv_mode 1): sum_j sum_d sqrt((D_d f)_j^2 + eps^2);
* the beta ~ 10 mu regime of step 1, reached where the Lipschitz bound
  1.05 gamma lambda_max(P^T P) falls below 10 mu (a geometry with every length
  scaled by 1e-3);
* the Eq. 2 adjoint (adjoint_mode 1): the residual bilinearly interpolated at the
  imager point of each voxel centre, weighted by L^3/(L0 l^2), in place of P^T;
* the paper-literal clamp (clamp_mode 1) is covered with the other parity tests.

Same gates as the main parity tests: volumes after a fixed number of iterations
within 1e-4 relative L2, energies within 1e-4 (1e-5 for a single evaluation),
f >= 0 exactly.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

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


@pytest.fixture(scope="module")
def small():
    return synth.make_case("small", with_truth=True, truth_ss=1)


def test_aniso_tv_prox_matches_oracle(lib, small):
    g = small["geom"]
    rng = np.random.default_rng(61)
    f0 = small["f_true"]
    gv = f0 + rng.normal(scale=0.004, size=f0.shape)
    eps = oracle.default_eps(g)
    beta = 2.0e5
    G = lib.cbct_geometry_create(g)
    ft = dev(f0)
    lib.cbct_tv_prox(G, dev(gv), ft, beta, eps, 10, tv_mode=1)
    out = host(ft)
    ref = oracle.prox(f32(gv), f32(f0), (4.0, 4.0, 4.0), beta, eps, 10, tv_mode=1)
    assert (out >= 0).all() and not np.signbit(out).any()
    d_ref = ref - f32(f0)
    assert np.linalg.norm((out - f32(f0)) - d_ref) <= 1e-4 * np.linalg.norm(d_ref)
    # the isotropic prox of the same input differs: the mode is really switched
    iso = oracle.prox(f32(gv), f32(f0), (4.0, 4.0, 4.0), beta, eps, 10)
    assert np.linalg.norm(iso - ref) > 10 * np.linalg.norm(out - ref)


def test_aniso_energy_matches_oracle(lib, small):
    g = small["geom"]
    rng = np.random.default_rng(62)
    f = rng.uniform(size=(64, 64, 64)) * 0.02
    eps = oracle.default_eps(g)
    G = lib.cbct_geometry_create(g)
    E = lib.cbct_energy(G, dev(small["Y"]), dev(f), small["mu"], eps, tv_mode=1)
    ref = oracle.energy(g, f32(small["Y"]), f32(f), small["mu"], eps, tv_mode=1)
    assert np.all(np.abs(E - ref) <= 1e-5 * np.abs(ref))


def test_aniso_fbs_small_20_iterations(lib, small):
    g = small["geom"]
    mu, eps = small["mu"], oracle.default_eps(g)
    beta = 1.05 * oracle.gamma(g, mu) * oracle.power_iteration(g, 30)
    Y = f32(small["Y"])
    f_ref, tr_ref = oracle.fbs(g, Y, mu, beta, eps, 10, 20, tv_mode=1)
    G = lib.cbct_geometry_create(g)
    ft, tr = lib.cbct_fbs(G, dev(Y), mu, beta, eps, 10, 0, 20, dev(np.zeros((64, 64, 64))), trace=True, tv_mode=1)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert (f >= 0).all() and not np.signbit(f).any()
    assert np.all(np.abs(tr - tr_ref) <= 1e-4 * np.abs(tr_ref))


def test_aniso_reconstruct_and_batch(lib, small):
    g = small["geom"]
    mu = small["mu"]
    betas = [1.05 * oracle.gamma(oracle.level_geom(g, l), mu) * oracle.power_iteration(oracle.level_geom(g, l), 30)
             for l in range(2)]
    Y = f32(small["Y"])
    f_ref, tr_ref = oracle.reconstruct(g, Y, mu, 8, 2, betas=betas, M=10, tv_mode=1)
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, betas=betas, trace=True, tv_mode=1)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert np.all(np.abs(info["trace"] - tr_ref) <= 1e-4 * np.abs(tr_ref))
    # in a batch next to an isotropic request, each comes out as it does alone
    fi = host(lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, betas=betas))
    reqs = [dict(geom=lib.cbct_geometry_create(g), Y=dev(Y), mu=mu, iters=8, levels=2, betas=betas, tv_mode=m)
            for m in (1, 0)]
    outs, _ = lib.cbct_reconstruct_batch(reqs, use_graphs=True)
    assert np.array_equal(host(outs[0]), f) and np.array_equal(host(outs[1]), fi)


def test_beta_ten_mu_regime(lib, small):
    """Every length x 1e-3: the automatic beta is exactly 10 mu and the GPU iterates
    match the oracle's at that beta."""
    g = small["geom"]
    s = 1e-3
    gs = dict(g, **{k: g[k] * s for k in ("hx", "hy", "hz", "du", "dv", "dso", "dsd")})
    mu = small["mu"]
    Ys = f32(small["Y"] * s)
    f_ref, tr_ref = oracle.reconstruct(gs, Ys, mu, 10, 1, betas=[10.0 * mu], M=10)
    G = lib.cbct_geometry_create(gs)
    ft, info = lib.cbct_reconstruct(G, dev(Ys), mu, 10, 1, trace=True)
    assert info["betas"][0] == 10.0 * mu
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert np.all(np.abs(info["trace"] - tr_ref) <= 1e-4 * np.abs(tr_ref))
    assert np.all(np.diff(info["trace"][0, :, 0]) <= 1e-6 * info["trace"][0, :-1, 0])


def _ragged():
    import math
    return dict(nx=45, ny=38, nz=37, hx=2.0, hy=2.5, hz=3.0, nu=53, nv=41, du=4.0, dv=4.5, dso=400.0, dsd=650.0,
                angles=2 * math.pi * np.arange(13) / 13 + 0.2)


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_eq2_backproject_matches_oracle(lib, small, which):
    g = small["geom"] if which == "small" else _ragged()
    rng = np.random.default_rng(63)
    shape = (len(g["angles"]), g["nv"], g["nu"])
    G = lib.cbct_geometry_create(g)
    for y in (rng.uniform(-1, 1, size=shape), f32(small["Y"]) if which == "small" else rng.uniform(0, 2, size=shape)):
        out = host(lib.cbct_backproject_eq2(G, dev(y)))
        ref = oracle.backproject_eq2(g, f32(y))
        assert rel(out, ref) <= 1e-5, rel(out, ref)
        assert np.abs(out - ref).max() <= 1e-5 * np.abs(ref).max()


def test_eq2_fbs_matches_oracle(lib, small):
    g = small["geom"]
    mu, eps = small["mu"], oracle.default_eps(g)
    beta = 1.05 * oracle.gamma(g, mu) * oracle.power_iteration(g, 30)
    Y = f32(small["Y"])
    f_ref, tr_ref = oracle.fbs(g, Y, mu, beta, eps, 10, 20, adjoint_mode=1)
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), mu, 20, 1, betas=[beta], trace=True, adjoint_mode=1)
    f = host(ft)
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    assert (f >= 0).all() and not np.signbit(f).any()
    assert np.all(np.abs(info["trace"][0] - tr_ref) <= 1e-4 * np.abs(tr_ref))


def test_eq2_two_levels_and_batch(lib, small):
    g = small["geom"]
    mu = small["mu"]
    betas = [1.05 * oracle.gamma(oracle.level_geom(g, l), mu) * oracle.power_iteration(oracle.level_geom(g, l), 30)
             for l in range(2)]
    Y = f32(small["Y"])
    f_ref, _ = oracle.reconstruct(g, Y, mu, 8, 2, betas=betas, M=10, adjoint_mode=1)
    G = lib.cbct_geometry_create(g)
    f = host(lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, betas=betas, adjoint_mode=1))
    assert rel(f, f_ref) <= VOL_TOL, rel(f, f_ref)
    # automatic beta, then the same request alone, in a batch next to a matched one, and
    # in the fp16-data variant (reported, not gated)
    fa = host(lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, adjoint_mode=1))
    fm = host(lib.cbct_reconstruct(G, dev(Y), mu, 8, 2))
    reqs = [dict(geom=lib.cbct_geometry_create(g), Y=dev(Y), mu=mu, iters=8, levels=2, adjoint_mode=m) for m in (1, 0)]
    outs, _ = lib.cbct_reconstruct_batch(reqs, use_graphs=True)
    assert np.array_equal(host(outs[0]), fa) and np.array_equal(host(outs[1]), fm)
    fh = host(lib.cbct_reconstruct(G, dev(Y), mu, 8, 2, adjoint_mode=1, sino_fp16=True))
    assert rel(fh, fa) <= 1e-2
