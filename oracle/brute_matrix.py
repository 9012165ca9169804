"""Dense system matrix by brute force -- TEST INFRASTRUCTURE ONLY.

A third, independent statement of the projector of Eq. 1 for tiny problems: every
ray is intersected with every voxel box by the slab method, vectorised in NumPy.
A[ray, voxel] is the intersection length in mm, rays ordered [na][nv][nu], voxels
[nz][ny][nx].  Shares no code with ``cbct_oracle.c`` or the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np


def ray_endpoints(geom):
    """Sources (na,3) and pixel centres (na, nv, nu, 3)."""
    th = np.asarray(geom["angles"], dtype=np.float64)
    c, s = np.cos(th), np.sin(th)
    S = np.stack([geom["dso"] * c, geom["dso"] * s, np.zeros_like(c)], axis=-1)
    u = (np.arange(geom["nu"]) - (geom["nu"] - 1) / 2.0) * geom["du"]
    v = (np.arange(geom["nv"]) - (geom["nv"] - 1) / 2.0) * geom["dv"]
    Cx = S[:, 0] - geom["dsd"] * c
    Cy = S[:, 1] - geom["dsd"] * s
    Px = Cx[:, None, None] - u[None, None, :] * s[:, None, None] + 0 * v[None, :, None]
    Py = Cy[:, None, None] + u[None, None, :] * c[:, None, None] + 0 * v[None, :, None]
    Pz = np.broadcast_to(v[None, :, None], Px.shape)
    return S, np.stack([Px, Py, Pz], axis=-1)


def system_matrix(geom) -> np.ndarray:
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    h = np.array([geom["hx"], geom["hy"], geom["hz"]])
    S, P = ray_endpoints(geom)
    na = len(geom["angles"])
    Sr = np.broadcast_to(S[:, None, None, :], P.shape).reshape(-1, 3)
    D = P.reshape(-1, 3) - Sr                                   # (R, 3)
    # voxel boxes
    lo_x = (np.arange(nx) - nx / 2.0) * h[0]
    lo_y = (np.arange(ny) - ny / 2.0) * h[1]
    lo_z = (np.arange(nz) - nz / 2.0) * h[2]
    LZ, LY, LX = np.meshgrid(lo_z, lo_y, lo_x, indexing="ij")
    lo = np.stack([LX.ravel(), LY.ravel(), LZ.ravel()], axis=-1)  # (V, 3)
    hi = lo + h
    R, V = D.shape[0], lo.shape[0]
    t0 = np.zeros((R, V))
    t1 = np.ones((R, V))
    for ax in range(3):
        d = D[:, ax][:, None]
        s0 = Sr[:, ax][:, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            a = (lo[None, :, ax] - s0) / d
            b = (hi[None, :, ax] - s0) / d
        lo_t = np.minimum(a, b)
        hi_t = np.maximum(a, b)
        par = (d == 0.0)
        inside = (s0 >= lo[None, :, ax]) & (s0 < hi[None, :, ax])
        lo_t = np.where(par, np.where(inside, -np.inf, np.inf), lo_t)
        hi_t = np.where(par, np.where(inside, np.inf, -np.inf), hi_t)
        t0 = np.maximum(t0, lo_t)
        t1 = np.minimum(t1, hi_t)
    L = np.linalg.norm(D, axis=1)[:, None]
    A = np.where(t1 > t0, (t1 - t0) * L, 0.0)
    assert A.shape == (na * geom["nv"] * geom["nu"], nz * ny * nx)
    return A


def tiny_geometry(n=8, h=4.0, nu=8, nv=8, du=8.0, dv=8.0, n_angles=6, dso=200.0, dsd=300.0,
                  theta0=0.0):
    """A small cone-beam geometry that sees the whole volume."""
    return dict(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, nu=nu, nv=nv, du=du, dv=dv, dso=dso, dsd=dsd,
                angles=theta0 + 2 * math.pi * np.arange(n_angles) / n_angles)
