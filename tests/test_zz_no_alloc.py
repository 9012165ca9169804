"""The allocation-free E1 entry point (cbct_tv_energy_noalloc) through the C ABI.

It serves callers that cannot call cudaMalloc: real-time hosts that forbid allocation
after start-up, plug-ins that must leave the device heap alone.  Its only scratch is a static array
inside the library, shared by all calls.  Here two calls in a row -- a large volume,
then a smaller one, so stale partial sums of the first call would show up in the
second -- must each give the E1 that the allocating entry point (cbct_energy)
reports for the same volume, within the tolerance of the other energy tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

E_TOL = 1e-5  # relative, as in the energy parity test


def _noalloc_e1(cbct, torch, geom, f_dev, eps):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = cbct.lib.cbct_tv_energy_noalloc(geom["nx"], geom["ny"], geom["nz"], geom["hx"], geom["hy"], geom["hz"],
                                         eps, C.c_void_p(f_dev.data_ptr()), C.c_void_p(out.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, cbct.cbct_last_error()
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_e1_matches_allocating_entry_point(cuda):
    torch = cuda
    from paper_1002_3675_b300 import cbct

    rng = np.random.default_rng(40)
    for name in ("medium", "small"):          # larger first, then smaller
        case = synth.make_case(name)
        g = case["geom"]
        f = torch.tensor((rng.uniform(size=(g["nz"], g["ny"], g["nx"])) * 0.02).astype(np.float32), device="cuda")
        Y = torch.tensor(np.asarray(case["Y"], dtype=np.float32), device="cuda")
        eps = 2e-5 / min(g["hx"], g["hy"], g["hz"])
        G = cbct.cbct_geometry_create(g)
        ref = cbct.cbct_energy(G, Y, f, case["mu"], eps)[1]
        got = _noalloc_e1(cbct, torch, g, f, eps)
        assert abs(got - ref) <= E_TOL * abs(ref), (name, got, ref)
    # eps = 0 (the unsmoothed TV) and a volume starting 4 bytes into its buffer, as for
    # a view into a larger tensor
    g = synth.make_case("small")["geom"]
    buf = torch.tensor((rng.uniform(size=g["nz"] * g["ny"] * g["nx"] + 1) * 0.02).astype(np.float32), device="cuda")
    f = buf[1:].view(g["nz"], g["ny"], g["nx"])
    G = cbct.cbct_geometry_create(g)
    ref0 = cbct.cbct_energy(G, torch.zeros((len(g["angles"]), g["nv"], g["nu"]), device="cuda"), f.clone(),
                            1.0, 0.0)[1]
    got0 = _noalloc_e1(cbct, torch, g, f, 0.0)
    assert abs(got0 - ref0) <= E_TOL * abs(ref0), (got0, ref0)


def test_noalloc_rejects_volumes_beyond_the_static_scratch(cuda):
    torch = cuda
    from paper_1002_3675_b300 import cbct

    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = cbct.lib.cbct_tv_energy_noalloc(512, 512, 256, 1.0, 1.0, 1.0, 1e-5, C.c_void_p(f.data_ptr()),
                                         C.c_void_p(out.data_ptr()), None)
    assert st == 1 and "CBCT_NOALLOC_MAX_VOXELS" in cbct.cbct_last_error()
