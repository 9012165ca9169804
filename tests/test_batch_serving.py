"""Batched persistent kernels, the autotuner and the continuous-batching server.

Every request must come out bitwise identical to its own single cbct_reconstruct
call: alone, in a batch, in any server mix, with or without CUDA graphs, and with any
launch shapes the autotuner picks.
"""
import math
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _geom(nx, ny, nz, h, na, nu, nv, du, theta0=0.0):
    return dict(nx=nx, ny=ny, nz=nz, hx=h[0], hy=h[1], hz=h[2], nu=nu, nv=nv, du=du, dv=du, dso=1000.0, dsd=1500.0,
                angles=theta0 + 2 * math.pi * np.arange(na) / na)


def _cases():
    """Heterogeneous requests (sizes, views, start angles, levels, iterations)."""
    rng = np.random.default_rng(50)
    specs = [
        (_geom(64, 64, 64, (4, 4, 4), 20, 64, 48, 8.0), 2, 4),
        (_geom(48, 56, 32, (5, 4, 6), 24, 60, 44, 8.5, 0.11), 1, 5),
        (_geom(80, 64, 40, (3, 3.5, 5), 30, 72, 52, 7.0, 0.05), 2, 3),
        (_geom(40, 40, 70, (6, 6, 3), 17, 50, 70, 8.0, 0.3), 2, 4),
    ]
    out = []
    for g, levels, iters in specs:
        Y = rng.uniform(0.0, 3.0, size=(len(g["angles"]), g["nv"], g["nu"])).astype(np.float32)
        out.append(dict(geom=g, Y=Y, mu=float(rng.uniform(2, 10)), levels=levels, iters=iters))
    return out


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
    return t.detach().cpu().numpy()


def _alone(lib, c, **kw):
    G = lib.cbct_geometry_create(c["geom"])
    f, info = lib.cbct_reconstruct(G, dev(c["Y"]), c["mu"], c["iters"], c["levels"], trace=True, **kw)
    return host(f), info


def test_batch_equals_single_requests(lib, cuda):
    torch = cuda
    cases = _cases()
    alone = [_alone(lib, c) for c in cases]
    for graphs in (False, True):
        reqs = [dict(geom=lib.cbct_geometry_create(c["geom"]), Y=dev(c["Y"]), mu=c["mu"], iters=c["iters"],
                     levels=c["levels"], trace=True) for c in cases]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            outs, infos = lib.cbct_reconstruct_batch(reqs, use_graphs=graphs)
        s.synchronize()
        for (fa, ia), fb, ib in zip(alone, outs, infos):
            assert np.array_equal(fa, host(fb))
            assert np.array_equal(ia["trace"], ib["trace"])
            assert np.array_equal(ia["step_trace"], ib["step_trace"])
            assert np.array_equal(ia["betas"], ib["betas"])


def test_batch_mixes_single_request_and_persistent_launches(lib, cuda):
    """A request large enough to fill the GPU runs its stages as single-request
    launches, the small ones share persistent launches; each stays bitwise equal to
    its own cbct_reconstruct call."""
    rng = np.random.default_rng(52)
    big = _geom(256, 256, 64, (1, 1, 2.5), 40, 256, 192, 1.6)
    cases = [dict(geom=big, Y=rng.uniform(0.0, 3.0, size=(40, 192, 256)).astype(np.float32), mu=5.0, levels=2,
                  iters=3)] + _cases()[:2]
    alone = [_alone(lib, c) for c in cases]
    reqs = [dict(geom=lib.cbct_geometry_create(c["geom"]), Y=dev(c["Y"]), mu=c["mu"], iters=c["iters"],
                 levels=c["levels"], trace=True) for c in cases]
    outs, infos = lib.cbct_reconstruct_batch(reqs, use_graphs=True)
    for (fa, ia), fb, ib in zip(alone, outs, infos):
        assert np.array_equal(fa, host(fb))
        assert np.array_equal(ia["trace"], ib["trace"])
        assert np.array_equal(ia["step_trace"], ib["step_trace"])
        assert np.all(ib["step_trace"] > 0)


def test_batch_rejects_shared_geometry(lib):
    c = _cases()[0]
    G = lib.cbct_geometry_create(c["geom"])
    reqs = [dict(geom=G, Y=dev(c["Y"]), mu=1.0, iters=1, levels=1)] * 2
    with pytest.raises(lib.CbctError) as e:
        lib.cbct_reconstruct_batch(reqs)
    assert e.value.status == 1


def test_autotune_keeps_results_and_caches(lib, tmp_path):
    from paper_1002_3675_b300 import autotune

    c = _cases()[2]
    f0, i0 = _alone(lib, c)
    G = lib.cbct_geometry_create(c["geom"])
    path = str(tmp_path / "tune.json")
    shapes = autotune.tune(G, c["levels"], path)
    assert len(shapes) == c["levels"] and os.path.exists(path)
    for s in shapes.values():
        assert s["proj_threads"] % 32 == 0 and 1 <= s["bp_vpl"] <= 4 and s["bp_threads"] in (64, 128, 256)
        assert s["bp_layout"] in (1, 2)
    f1, i1 = lib.cbct_reconstruct(G, dev(c["Y"]), c["mu"], c["iters"], c["levels"], trace=True)
    assert np.array_equal(f0, host(f1)) and np.array_equal(i0["trace"], i1["trace"])
    # a second geometry of the same size class takes the cached shapes without timing
    G2 = lib.cbct_geometry_create(c["geom"])
    assert autotune.tune(G2, c["levels"], path) == shapes


def _serve(lib, cases, budget, slots, gaps, graphs=False, reuse=False):
    srv = lib.Server(budget, slots, use_graphs=graphs)
    outs, tickets = [], []
    for c, gap in zip(cases, gaps):
        f = dev(np.zeros((c["geom"]["nz"], c["geom"]["ny"], c["geom"]["nx"])))
        Y = dev(c["Y"])
        tickets.append(srv.submit(c["geom"], Y, c["mu"], c["iters"], c["levels"], f, reuse_lambda=reuse))
        outs.append((f, Y))
        time.sleep(gap)
    res = [srv.wait(t, 60000) for t in tickets]
    stats = srv.stats()
    srv.close()
    return [host(f) for f, _ in outs], res, stats


def test_server_results_equal_alone_in_any_mix(lib):
    cases = _cases()
    mix = cases + cases[:2] + cases[2:]          # repeats reuse resident geometries
    alone = [_alone(lib, c)[0] for c in cases]
    expect = alone + alone[:2] + alone[2:]
    rng = np.random.default_rng(51)
    gaps = rng.exponential(0.002, size=len(mix))  # Poisson arrivals while others run
    for graphs, reuse in ((False, False), (True, True)):
        vols, res, stats = _serve(lib, mix, 8 << 30, 3, gaps, graphs=graphs, reuse=reuse)
        for v, e, r in zip(vols, expect, res):
            assert r["status"] == 0
            assert np.array_equal(v, e)
        assert stats["completed"] == len(mix)


def test_server_small_budget_admits_in_order(lib):
    cases = _cases()
    alone = [_alone(lib, c)[0] for c in cases]
    # room for one or two of these geometries at a time: requests wait for memory
    budget = 9 << 20
    vols, res, stats = _serve(lib, cases, budget, 4, [0.0] * len(cases))
    for v, e, r in zip(vols, alone, res):
        assert np.array_equal(v, e)
    assert stats["hbm_in_use"] <= budget
    assert sorted(r["queue_s"] for r in res)[-1] > 0.5 * min(r["latency_s"] - r["queue_s"] for r in res)


def test_server_timeout_cancel_and_injected_failure(lib):
    cases = _cases()
    srv = lib.Server(8 << 30, 1)
    big = dict(cases[0], iters=60)
    f1, Y1 = dev(np.zeros((64, 64, 64))), dev(big["Y"])
    t1 = srv.submit(big["geom"], Y1, big["mu"], big["iters"], big["levels"], f1)
    f2, Y2 = dev(np.zeros((64, 64, 64))), dev(big["Y"])
    t2 = srv.submit(big["geom"], Y2, big["mu"], 1, 1, f2)
    with pytest.raises(lib.CbctError) as e:            # one slot: t2 waits behind t1
        srv.wait(t2, 1)
    assert e.value.status == 4
    srv.cancel(t2)
    with pytest.raises(lib.CbctError) as e:
        srv.wait(t2, 1000)
    assert e.value.status == 7
    assert srv.wait(t1, 60000)["status"] == 0
    # an injected set-up failure ends that request only
    lib.cbct_debug_fail_next_allocations(1)
    c = cases[1]
    f3, Y3 = dev(np.zeros((c["geom"]["nz"], c["geom"]["ny"], c["geom"]["nx"]))), dev(c["Y"])
    t3 = srv.submit(c["geom"], Y3, c["mu"], 2, 1, f3)
    with pytest.raises(lib.CbctError) as e:
        srv.wait(t3, 60000)
    assert e.value.status == 2
    f4 = dev(np.zeros((c["geom"]["nz"], c["geom"]["ny"], c["geom"]["nx"])))
    t4 = srv.submit(c["geom"], Y3, c["mu"], 2, 1, f4)
    assert srv.wait(t4, 60000)["status"] == 0
    srv.close()


def test_server_rejects_malformed_and_oversized(lib):
    c = _cases()[0]
    srv = lib.Server(64 << 20, 2)
    f, Y = dev(np.zeros((64, 64, 64))), dev(c["Y"])
    bad = dict(c["geom"], nx=0)
    with pytest.raises(lib.CbctError) as e:
        srv.submit(bad, Y, 1.0, 1, 1, f)
    assert e.value.status == 1
    with pytest.raises(lib.CbctError) as e:
        srv.submit(c["geom"], Y, -1.0, 1, 1, f)
    assert e.value.status == 1
    huge = _geom(512, 512, 256, (0.5, 0.5, 0.5), 40, 512, 384, 0.8)
    with pytest.raises(lib.CbctError) as e:
        srv.submit(huge, Y, 1.0, 1, 1, f)
    assert e.value.status == 6
    srv.close()
