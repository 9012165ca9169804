"""The C ABI library loads on a machine without a GPU, exports every function the
header declares, and rejects invalid arguments before touching the device."""
import ctypes as C

import numpy as np

from paper_1002_3675_b300 import cbct


def test_library_exports_every_declared_function():
    names = cbct.header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(cbct.lib, n)]
    assert not missing, missing


def test_version_and_error_strings():
    assert "sm_103a" in cbct.cbct_version()
    assert isinstance(cbct.cbct_last_error(), str)


def _desc(**kw):
    base = dict(nx=8, ny=8, nz=8, hx=1.0, hy=1.0, hz=1.0, nu=8, nv=8, du=1.0, dv=1.0, dso=100.0, dsd=150.0)
    base.update(kw)
    return cbct.make_desc(base)


def _create(desc, angles):
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    h = C.c_void_p()
    st = cbct.lib.cbct_geometry_create(C.byref(desc), ang.ctypes.data_as(C.POINTER(C.c_double)), len(ang),
                                       C.byref(h))
    return st, h


def test_invalid_geometry_rejected_without_device():
    for bad in (dict(nx=0), dict(nv=-3), dict(hx=0.0), dict(dso=-1.0), dict(du=float("nan"))):
        st, h = _create(_desc(**bad), [0.0, 1.0])
        assert st == 1 and not h.value, bad
        assert cbct.cbct_last_error()
    st, h = _create(_desc(), [])
    assert st == 1
    st, h = _create(_desc(), [0.0, float("inf")])
    assert st == 1
    # 2^31 voxels
    st, h = _create(_desc(nx=2048, ny=2048, nz=512), [0.0])
    assert st == 1


def test_null_and_misaligned_pointers_rejected():
    assert cbct.lib.cbct_project(None, None, None, None) == 1
    assert cbct.lib.cbct_restrict_sino(2, 4, 4, C.c_void_p(8), C.c_void_p(32), None) == 1   # misaligned
    assert cbct.lib.cbct_restrict_sino(0, 4, 4, C.c_void_p(16), C.c_void_p(32), None) == 1  # empty
    assert cbct.lib.cbct_prolong_vol(1, 1, 1, None, 2, 2, 2, C.c_void_p(16), None) == 1
    out = (C.c_int * 5)()
    assert cbct.lib.cbct_level_dims(None, 0, out) == 1
