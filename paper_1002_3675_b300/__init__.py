"""B300 (sm_103a) TV-regularised cone-beam CT reconstruction (Jia et al. 2010).

The compute path is the shared library built from ``csrc/`` (hand-written CUDA
kernels behind the C ABI of ``include/cbct.h``); ``cbct`` is its ctypes binding.
PyTorch only supplies device memory and the current stream.
"""
from .cbct import (  # noqa: F401
    CbctError,
    Geometry,
    cbct_backproject,
    cbct_energy,
    cbct_fbs,
    cbct_geometry_create,
    cbct_last_error,
    cbct_level_dims,
    cbct_power_iteration,
    cbct_project,
    cbct_prolong_vol,
    cbct_reconstruct,
    cbct_restrict_sino,
    cbct_tv_prox,
    cbct_version,
)
