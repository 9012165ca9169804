"""Parity of the V-cycle (mg_cycle 1) with the FP64 oracle: the finest volume after a
fixed number of cycles within 1e-4 relative L2, the energy after each cycle within
1e-4, and the same coarse corrections kept (a decision both sides take from their
own energies)."""
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


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def small():
    return synth.make_case("small")


@pytest.mark.parametrize("levels,tv_mode", [(2, 0), (3, 0), (2, 1)])
def test_vcycle_matches_oracle(lib, small, levels, tv_mode):
    g = small["geom"]
    mu = small["mu"]
    betas = [1.05 * oracle.gamma(oracle.level_geom(g, l), mu) * oracle.power_iteration(oracle.level_geom(g, l), 30)
             for l in range(levels)]
    Y = f32(small["Y"])
    f_ref, tr_ref, acc_ref = oracle.vcycle(g, Y, mu, 3, levels, betas=betas, pre=2, post=2, coarse=10,
                                           tv_mode=tv_mode)
    G = lib.cbct_geometry_create(g)
    ft, info = lib.cbct_reconstruct(G, dev(Y), mu, 3, levels, betas=betas, trace=True, mg_cycle=1, mg_pre=2,
                                    mg_post=2, mg_coarse=10, tv_mode=tv_mode, use_graphs=True)
    f = host(ft)
    assert rel(f, f_ref) <= 1e-4, rel(f, f_ref)
    assert (f >= 0).all() and not np.signbit(f).any()
    assert np.all(np.abs(info["trace"] - tr_ref) <= 1e-4 * np.abs(tr_ref))
    assert list(info["accepted"]) == list(acc_ref) and acc_ref[0] >= 1


def test_vcycle_energy_falls_every_cycle(lib, small):
    g = small["geom"]
    G = lib.cbct_geometry_create(g)
    _, iv = lib.cbct_reconstruct(G, dev(small["Y"]), small["mu"], 5, 2, trace=True, mg_cycle=1)
    assert np.all(np.diff(iv["trace"][:, 0]) < 0) and iv["accepted"][0] >= 1
    # step_trace: the change of the iterate over each cycle; the first is |f_1| (f_0 = 0)
    f1 = host(lib.cbct_reconstruct(lib.cbct_geometry_create(g), dev(small["Y"]), small["mu"], 1, 2, mg_cycle=1))
    st = iv["step_trace"]
    assert st.shape == (5,) and np.all(st > 0)
    assert abs(st[0] - np.linalg.norm(f1.astype(np.float64))) <= 1e-5 * st[0]


def test_vcycle_is_rejected_where_unsupported(lib, small):
    g = small["geom"]
    G = lib.cbct_geometry_create(g)
    Y = dev(small["Y"])
    with pytest.raises(lib.CbctError) as e:
        lib.cbct_reconstruct(G, Y, 1.0, 1, 2, mg_cycle=1, adjoint_mode=1)
    assert e.value.status == 5
    with pytest.raises(lib.CbctError) as e:
        lib.cbct_reconstruct_batch([dict(geom=G, Y=Y, mu=1.0, iters=1, levels=2, mg_cycle=1)])
    assert e.value.status == 5
