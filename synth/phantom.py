"""Scan geometries, ellipsoid phantoms, analytic line integrals and noise.

Geometry convention (the paper fixes none; the text introducing Eq. 1 defines P^theta
only as the cone-beam projection onto the imager at angle theta):

* millimetres throughout; the rotation axis is z and the volume is centred on the
  origin.  Voxel (i, j, k) has centre ((i - (nx-1)/2) hx, (j - (ny-1)/2) hy,
  (k - (nz-1)/2) hz) and occupies the half-open box centre +- h/2.
* source  S(theta) = (dso cos theta, dso sin theta, 0)
* imager centre C(theta) = S + dsd (-cos theta, -sin theta, 0), with in-plane
  axes u = (-sin theta, cos theta, 0) and v = (0, 0, 1).
* pixel (a, b) centre = C + (a - (nu-1)/2) du u + (b - (nv-1)/2) dv v; one ray per
  pixel centre, from S to that centre.
* volumes are stored [nz][ny][nx] (x fastest); projection stacks [n_angles][nv][nu]
  (u fastest).

Workloads follow the experiments of the paper (a thorax-sized 512x512 volume with a
512x384 imager and 20-40 views over 360 degrees; a low-dose scan) with seeded
synthetic ellipsoid phantoms standing in for the NCAT and CatPhan data, which are
not available.  Everything is float64 NumPy with a PCG64 generator seeded per case.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CONFIGS",
    "BATCH_SIZES",
    "make_request",
    "make_request_set",
    "Ellipsoid",
    "geometry_for",
    "pixel_rays",
    "make_ellipsoids",
    "voxelize",
    "analytic_sinogram",
    "poisson_log",
    "make_case",
]


# ----------------------------------------------------------------------------------
# Workload definitions.  mu weighs E2 against E1 in Eq. 1; the paper sets it by hand
# for image quality, so each workload freezes one value.
# ----------------------------------------------------------------------------------
CONFIGS = {
    # 64^3 at 4 mm, 20 views of 64x48 at 8 mm, noise-free, single grid, 20 iterations
    "small": dict(
        vol=(64, 64, 64), h=(4.0, 4.0, 4.0), det=(64, 48), pitch=(8.0, 8.0),
        n_angles=20, dso=1000.0, dsd=1500.0, I0=None, levels=1, iters=20,
        mu=10.0, seed=1000, inserts=0,
    ),
    # 256x256x64 at 1x1x2.5 mm, 40 views of 256x192 at 1.6 mm, I0 = 1e5,
    # 2-level multigrid, 50 iterations per level
    "medium": dict(
        vol=(256, 256, 64), h=(1.0, 1.0, 2.5), det=(256, 192), pitch=(1.6, 1.6),
        n_angles=40, dso=1000.0, dsd=1500.0, I0=1e5, levels=2, iters=50,
        mu=5.0, seed=1001, inserts=0,
    ),
    # 512x512x96 at 0.5x0.5x2.5 mm, 40 views of 512x384 at 0.8 mm, I0 = 2.5e4,
    # 3-level multigrid, 50 iterations per level, small high-contrast inserts
    "large": dict(
        vol=(512, 512, 96), h=(0.5, 0.5, 2.5), det=(512, 384), pitch=(0.8, 0.8),
        n_angles=40, dso=1000.0, dsd=1500.0, I0=2.5e4, levels=3, iters=50,
        mu=2.0, seed=1002, inserts=5,
    ),
}
for _n in (20, 30):
    CONFIGS[f"large{_n}"] = dict(CONFIGS["large"], n_angles=_n)


@dataclasses.dataclass
class Ellipsoid:
    centre: np.ndarray   # (3,) mm
    axes: np.ndarray     # (3,) semi-axes, mm
    rot: np.ndarray      # (3,3) columns = ellipsoid axes in world coordinates
    density: float       # mm^-1 (added to the background)

    def quadric(self):
        """Matrix M with (p-c)^T M (p-c) <= 1 inside."""
        return self.rot @ np.diag(1.0 / self.axes ** 2) @ self.rot.T


def geometry_for(cfg: dict, theta0: float = 0.0) -> dict:
    """Plain-dict scan geometry for a configuration (angles evenly over 360 deg)."""
    nx, ny, nz = cfg["vol"]
    hx, hy, hz = cfg["h"]
    nu, nv = cfg["det"]
    du, dv = cfg["pitch"]
    na = cfg["n_angles"]
    angles = theta0 + 2.0 * math.pi * np.arange(na, dtype=np.float64) / na
    return dict(nx=nx, ny=ny, nz=nz, hx=hx, hy=hy, hz=hz, nu=nu, nv=nv, du=du, dv=dv,
                dso=float(cfg["dso"]), dsd=float(cfg["dsd"]), angles=angles)


def pixel_rays(geom: dict, theta: float):
    """Source position (3,) and pixel centres (nv, nu, 3) at one angle."""
    c, s = math.cos(theta), math.sin(theta)
    S = np.array([geom["dso"] * c, geom["dso"] * s, 0.0])
    C = S + geom["dsd"] * np.array([-c, -s, 0.0])
    u_hat = np.array([-s, c, 0.0])
    v_hat = np.array([0.0, 0.0, 1.0])
    ua = (np.arange(geom["nu"]) - (geom["nu"] - 1) / 2.0) * geom["du"]
    vb = (np.arange(geom["nv"]) - (geom["nv"] - 1) / 2.0) * geom["dv"]
    P = C[None, None, :] + ua[None, :, None] * u_hat + vb[:, None, None] * v_hat
    return S, P


def _rotation(rng) -> np.ndarray:
    """Rotation from three random Euler angles (z-x-z)."""
    a, b, g = rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)

    def rz(t):
        return np.array([[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1.0]])

    def rx(t):
        return np.array([[1.0, 0, 0], [0, math.cos(t), -math.sin(t)], [0, math.sin(t), math.cos(t)]])

    return rz(a) @ rx(b) @ rz(g)


def _region(geom: dict):
    """Radius and half-height of the region that every view samples."""
    half_w = 0.5 * min(geom["nx"] * geom["hx"], geom["ny"] * geom["hy"])
    half_h = 0.5 * geom["nz"] * geom["hz"]
    fov = geom["dso"] * math.sin(math.atan(0.5 * geom["nu"] * geom["du"] / geom["dsd"]))
    cone = 0.5 * geom["nv"] * geom["dv"] * (geom["dso"] - half_w) / geom["dsd"]
    return min(half_w, fov), min(half_h, cone)


def make_ellipsoids(geom: dict, rng, n: int = 10, inserts: int = 0):
    """Ten additive ellipsoids (semi-axes 8-100 mm, densities 0.002-0.02 /mm), each
    with its bounding sphere inside the sampled region, plus optional small
    high-contrast spheres (radius 1.5-4 mm, +0.02 /mm)."""
    rmax, zmax = _region(geom)
    out = []
    for _ in range(n):
        axes = rng.uniform(8.0, 100.0, size=3)
        rot = _rotation(rng)
        dens = rng.uniform(0.002, 0.02)
        R = float(axes.max())
        lim = 0.95 * min(rmax, zmax)
        if R > lim:
            axes = axes * (lim / R)
            R = lim
        rr = (rmax - R) * math.sqrt(rng.uniform())
        ph = rng.uniform(0, 2 * math.pi)
        zc = rng.uniform(-(zmax - R), zmax - R)
        out.append(Ellipsoid(np.array([rr * math.cos(ph), rr * math.sin(ph), zc]), axes, rot, dens))
    for _ in range(inserts):
        r = rng.uniform(1.5, 4.0)
        rr = (0.6 * rmax) * math.sqrt(rng.uniform())
        ph = rng.uniform(0, 2 * math.pi)
        zc = rng.uniform(-(zmax - r) * 0.6, (zmax - r) * 0.6)
        out.append(Ellipsoid(np.array([rr * math.cos(ph), rr * math.sin(ph), zc]),
                             np.array([r, r, r]), np.eye(3), 0.02))
    return out


def voxelize(ells, geom: dict, ss: int = 4) -> np.ndarray:
    """Ground-truth volume [nz][ny][nx]: mean density over ss^3 sub-samples per voxel."""
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    hx, hy, hz = geom["hx"], geom["hy"], geom["hz"]
    f = np.zeros((nz, ny, nx))
    off = (np.arange(ss) + 0.5) / ss - 0.5
    xs = ((np.arange(nx) - (nx - 1) / 2.0)[:, None] + off[None, :]).ravel() * hx
    ys = ((np.arange(ny) - (ny - 1) / 2.0)[:, None] + off[None, :]).ravel() * hy
    zs = ((np.arange(nz) - (nz - 1) / 2.0)[:, None] + off[None, :]).ravel() * hz
    for e in ells:
        M = e.quadric()
        R = float(e.axes.max())
        ix = np.nonzero(np.abs(xs - e.centre[0]) <= R)[0]
        iy = np.nonzero(np.abs(ys - e.centre[1]) <= R)[0]
        iz = np.nonzero(np.abs(zs - e.centre[2]) <= R)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        X = xs[ix] - e.centre[0]
        Y = ys[iy] - e.centre[1]
        for kz in iz:
            Z = zs[kz] - e.centre[2]
            q = (M[0, 0] * X[None, :] ** 2 + M[1, 1] * Y[:, None] ** 2 + M[2, 2] * Z * Z
                 + 2 * M[0, 1] * X[None, :] * Y[:, None] + 2 * M[0, 2] * X[None, :] * Z
                 + 2 * M[1, 2] * Y[:, None] * Z)
            inside = (q <= 1.0).astype(np.float64)
            # accumulate sub-samples into voxels
            vy, vx = iy // ss, ix // ss
            acc = np.zeros((ny, nx))
            np.add.at(acc, (vy[:, None], vx[None, :]), inside)
            f[kz // ss] += e.density * acc
    return f / float(ss ** 3)


def analytic_sinogram(ells, geom: dict) -> np.ndarray:
    """Exact line integrals sum_k density_k * chord_k for every pixel ray, [na][nv][nu].

    Along the unit ray S + s d, ellipsoid (p - c)^T M (p - c) <= 1 gives the quadratic
    A s^2 + 2 B s + C = 0 with A = d^T M d, B = d^T M q, C = q^T M q - 1, q = S - c, and
    the chord is 2 sqrt(B^2 - A C) / A (the whole ellipsoid lies between source and
    imager)."""
    out = np.zeros((len(geom["angles"]), geom["nv"], geom["nu"]))
    quads = [(e, e.quadric()) for e in ells]
    for ia, th in enumerate(geom["angles"]):
        S, P = pixel_rays(geom, float(th))
        d = (P - S).reshape(-1, 3)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        dx, dy, dz = d[:, 0].copy(), d[:, 1].copy(), d[:, 2].copy()
        xx, yy, zz, xy, xz, yz = dx * dx, dy * dy, dz * dz, dx * dy, dx * dz, dy * dz
        acc = np.zeros(d.shape[0])
        for e, M in quads:
            q = S - e.centre
            mq = M @ q
            A = M[0, 0] * xx + M[1, 1] * yy + M[2, 2] * zz + 2.0 * (M[0, 1] * xy + M[0, 2] * xz + M[1, 2] * yz)
            B = mq[0] * dx + mq[1] * dy + mq[2] * dz
            disc = B * B - A * (float(q @ mq) - 1.0)
            pos = disc > 0
            acc[pos] += e.density * 2.0 * np.sqrt(disc[pos]) / A[pos]
        out[ia] = acc.reshape(geom["nv"], geom["nu"])
    return out


def poisson_log(Y: np.ndarray, I0: float, rng) -> np.ndarray:
    """Poisson counts N ~ Poisson(I0 exp(-Y)); returns -ln(max(N, 0.5) / I0).

    The counts are drawn by torch's CPU Poisson sampler (fast for every mean) from a
    generator seeded by the case's PCG64 stream, so the data stay seeded."""
    import torch

    gen = torch.Generator().manual_seed(int(rng.integers(0, 2 ** 62)))
    lam = torch.from_numpy(np.ascontiguousarray(I0 * np.exp(-Y), dtype=np.float64))
    N = torch.poisson(lam, generator=gen).numpy()
    return -np.log(np.maximum(N, 0.5) / I0)


def make_case(name: str, *, with_truth: bool = False, truth_ss: int = 2, theta0: float = 0.0):
    """Seeded case: geometry, measured data Y [na][nv][nu] (float64), solver settings."""
    cfg = CONFIGS[name]
    rng = np.random.Generator(np.random.PCG64(cfg["seed"]))
    geom = geometry_for(cfg, theta0)
    ells = make_ellipsoids(geom, rng, 10, cfg["inserts"])
    Y = analytic_sinogram(ells, geom)
    if cfg["I0"] is not None:
        Y = poisson_log(Y, cfg["I0"], rng)
    case = dict(name=name, geom=geom, Y=Y, mu=cfg["mu"], iters=cfg["iters"],
                levels=cfg["levels"], ellipsoids=ells)
    if with_truth:
        case["f_true"] = voxelize(ells, geom, truth_ss)
    return case


# Heterogeneous requests of a batch (volume 128^3 to 384x384x64, 20-60 views with a
# random start offset, 128x96 to 384x288 imagers, Poisson I0 log-uniform in
# 1e4..1e5).  The transverse extent is 256 mm and the axial one 160 mm; the imager
# pitch makes the imager cover the volume's field of view x 1.1 at dsd/dso = 1.5.
BATCH_SIZES = [((128, 128, 128), (128, 96)), ((192, 192, 96), (192, 144)), ((256, 256, 64), (256, 192)),
               ((256, 256, 96), (256, 192)), ((320, 320, 64), (320, 240)), ((384, 384, 64), (384, 288))]


def make_request(rng, size_index=None, levels=2, iters=30):
    """One seeded request of the heterogeneous batch workload."""
    if size_index is None:
        size_index = int(rng.integers(0, len(BATCH_SIZES)))
    (nx, ny, nz), (nu, nv) = BATCH_SIZES[size_index]
    hx = 256.0 / nx
    hz = 160.0 / nz
    na = int(rng.integers(20, 61))
    du = 1.1 * 256.0 * 1.5 / nu
    dv = 1.1 * 160.0 * 1.5 / nv
    cfg = dict(vol=(nx, ny, nz), h=(hx, hx, hz), det=(nu, nv), pitch=(du, dv), n_angles=na, dso=1000.0, dsd=1500.0)
    geom = geometry_for(cfg, theta0=float(rng.uniform(0.0, 2.0 * math.pi / na)))
    ells = make_ellipsoids(geom, rng, 10, 0)
    I0 = float(10 ** rng.uniform(4.0, 5.0))
    Y = poisson_log(analytic_sinogram(ells, geom), I0, rng)
    return dict(geom=geom, Y=Y, mu=5.0, levels=levels, iters=iters, I0=I0, size_index=size_index)


def make_request_set(seed, n, levels=2, iters=30):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [make_request(rng, q % len(BATCH_SIZES), levels, iters) for q in range(n)]
