"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This package generates *inputs only*: scan geometries, ellipsoid phantoms, their
analytic line integrals and Poisson/log noise.  It contains none of the
reconstruction method's arithmetic (no projector, adjoint, TV or solver), so the
FP64 oracle and the CUDA path can both consume it without sharing code.
"""
from .phantom import (  # noqa: F401
    BATCH_SIZES,
    CONFIGS,
    Ellipsoid,
    analytic_sinogram,
    geometry_for,
    make_case,
    make_ellipsoids,
    make_request,
    make_request_set,
    pixel_rays,
    poisson_log,
    voxelize,
)
