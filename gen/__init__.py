"""Seeded synthetic inputs for Voronoi-grid ray traversal.

This module only draws random numbers: site positions, per-cell densities,
ray origins and directions, detector pixels. It holds none of the traversal
method's arithmetic, so both the CPU oracle and the GPU library can consume
its outputs without sharing any code with each other.

Workload shapes follow the paper's test models (Sect. 3.2-3.3): uniformly
placed sites like the torus grid, density-weighted sites like the spiral
grid, about one million cells. The paper's own models are not reproducible
(their geometry parameters are not printed), so these stand in for them:

* ``uniform_cube``   - sites i.i.d. uniform in [-1, 1]^3 (torus-like placement)
* ``exp_disk``       - sites drawn from rho ~ exp(-R - |z|/0.1) in
                       [-4, 4]^2 x [-0.5, 0.5] (spiral-like, density-weighted)
* ``clumpy``         - 70 % uniform, 30 % in Gaussian clumps
* ``batched``        - many independent grids of uneven size

All sites are rounded to float32 and returned as float64 holding those exact
float32 values (the traversal stores sites as float4, so the float32 values
are the canonical geometry). Exact duplicates after rounding are redrawn.
Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1310_1854

CUBE_BOX = np.array([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0])
DISK_BOX = np.array([-4.0, -4.0, -0.5, 4.0, 4.0, 0.5])
UNIT_BALL = np.array([0.0, 0.0, 0.0, 1.0])   # (cx, cy, cz, R): the ball inscribed in CUBE_BOX

# exponential disk: rho = exp(-R/H_R - |z|/H_Z)
DISK_HR = 1.0
DISK_HZ = 0.1


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _round_f32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _inside(p: np.ndarray, box: np.ndarray) -> np.ndarray:
    return np.all((p >= box[:3]) & (p <= box[3:]), axis=1)


def _dedupe_f32(p: np.ndarray, redraw, rng) -> np.ndarray:
    """Round to float32 and redraw exact duplicates until none remain."""
    p = _round_f32(p)
    for _ in range(100):
        _, first = np.unique(p, axis=0, return_index=True)
        if first.size == p.shape[0]:
            return p
        dup = np.setdiff1d(np.arange(p.shape[0]), first)
        p[dup] = _round_f32(redraw(dup.size, rng))
    raise RuntimeError("could not remove duplicate sites")


def uniform_points(n: int, rng, box=CUBE_BOX) -> np.ndarray:
    lo, hi = box[:3], box[3:]
    return lo + (hi - lo) * rng.random((n, 3))


def in_ball(p: np.ndarray, sphere) -> np.ndarray:
    """Closed ball test for generating sites inside a spherical domain:
    ((dx dx + dy dy) + dz dz) <= R R in float64."""
    c = np.asarray(sphere, np.float64)
    d = np.asarray(p, np.float64) - c[:3]
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= c[3] * c[3]


def ball_points(n: int, rng, sphere=UNIT_BALL) -> np.ndarray:
    """Uniform points in the ball (cx, cy, cz, R), by rejection from its
    bounding cube; the points stay inside after rounding to float32."""
    c = np.asarray(sphere, np.float64)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        q = c[:3] + c[3] * (2.0 * rng.random((2 * (n - out.shape[0]) + 16, 3)) - 1.0)
        q = q[in_ball(_round_f32(q), c)]
        out = np.concatenate([out, q])
    return out[:n]


def disk_points(n: int, rng, box=DISK_BOX) -> np.ndarray:
    """Points with density exp(-R - |z|/0.1), rejected outside ``box``.

    The cylindrical radius has marginal R exp(-R), i.e. Gamma(2, 1); the
    height is Laplace(0, 0.1); the azimuth is uniform.
    """
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.2) + 16
        R = rng.gamma(2.0, DISK_HR, m)
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        z = rng.laplace(0.0, DISK_HZ, m)
        p = np.stack([R * np.cos(phi), R * np.sin(phi), z], axis=1)
        out = np.concatenate([out, p[_inside(p, box)]])
    return out[:n]


def disk_density(p: np.ndarray) -> np.ndarray:
    R = np.hypot(p[:, 0], p[:, 1])
    return np.exp(-R / DISK_HR - np.abs(p[:, 2]) / DISK_HZ)


def isotropic_dirs(n: int, rng) -> np.ndarray:
    """Unit vectors from normalised 3D Gaussians (float64)."""
    while True:
        k = rng.standard_normal((n, 3))
        nrm = np.linalg.norm(k, axis=1)
        bad = nrm < 1e-8
        if not bad.any():
            return k / nrm[:, None]
        k[bad] = rng.standard_normal((int(bad.sum()), 3))


def clumpy_points(n: int, rng, n_clumps=2000, frac_clump=0.3,
                  sigma_lo=0.01, sigma_hi=0.05, box=CUBE_BOX):
    """70 % uniform sites, 30 % split equally over Gaussian clumps.

    Returns (points, in_clump flag). Gaussian draws that land outside the box
    are redrawn from the same clump.
    """
    n_c = int(round(n * frac_clump))
    n_u = n - n_c
    centres = uniform_points(n_clumps, rng, box)
    sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_clumps))
    per = np.full(n_clumps, n_c // n_clumps)
    per[: n_c - per.sum()] += 1
    owner = np.repeat(np.arange(n_clumps), per)
    pts = centres[owner] + sig[owner, None] * rng.standard_normal((n_c, 3))
    for _ in range(1000):
        bad = ~_inside(pts, box)
        if not bad.any():
            break
        o = owner[bad]
        pts[bad] = centres[o] + sig[o, None] * rng.standard_normal((o.size, 3))
    p = np.concatenate([uniform_points(n_u, rng, box), pts])
    flag = np.concatenate([np.zeros(n_u, bool), np.ones(n_c, bool)])
    return p, flag


@dataclasses.dataclass
class Grid:
    """One Voronoi grid: float32-exact sites (as float64), box, density."""
    sites: np.ndarray          # (M, 3) float64 holding float32 values
    box: np.ndarray            # (6,) xmin, ymin, zmin, xmax, ymax, zmax
    rho: np.ndarray            # (M,) float32 per-cell density
    kappa: float = 1.0
    name: str = ""


@dataclasses.dataclass
class Rays:
    origin: np.ndarray         # (N, 3) float64
    dir: np.ndarray            # (N, 3) float64 unit vectors


def make_uniform_grid(M: int, seed: int, box=CUBE_BOX, rho_lo=0.5, rho_hi=1.5):
    rng = rng_for(seed)
    p = _dedupe_f32(uniform_points(M, rng, box), lambda k, r: uniform_points(k, r, box), rng)
    rho = rng.uniform(rho_lo, rho_hi, M).astype(np.float32)
    return Grid(p, np.array(box, dtype=np.float64), rho, 1.0, f"uniform{M}")


def make_disk_grid(M: int, seed: int, box=DISK_BOX):
    rng = rng_for(seed)
    p = _dedupe_f32(disk_points(M, rng, box), lambda k, r: disk_points(k, r, box), rng)
    rho = disk_density(p).astype(np.float32)
    return Grid(p, np.array(box, dtype=np.float64), rho, 1.0, f"disk{M}")


def make_clumpy_grid(M: int, seed: int, box=CUBE_BOX, n_clumps=2000):
    rng = rng_for(seed)
    p, flag = clumpy_points(M, rng, n_clumps=n_clumps, box=box)
    p = _dedupe_f32(p, lambda k, r: uniform_points(k, r, box), rng)
    rho = np.where(flag, 100.0, 1.0).astype(np.float32)
    return Grid(p, np.array(box, dtype=np.float64), rho, 1.0, f"clumpy{M}")


def make_ball_grid(M: int, seed: int, sphere=UNIT_BALL, box=CUBE_BOX):
    """Sites uniform in a ball inside the box (a spherical domain), density
    falling off from the centre: rho = exp(-|r - c| / (R / 3))."""
    rng = rng_for(seed)
    p = _dedupe_f32(ball_points(M, rng, sphere), lambda k, r: ball_points(k, r, sphere), rng)
    c = np.asarray(sphere, np.float64)
    rho = np.exp(-np.linalg.norm(p - c[:3], axis=1) / (c[3] / 3.0)).astype(np.float32)
    return Grid(p, np.array(box, dtype=np.float64), rho, 1.0, f"ball{M}")


def ball_rays(N: int, seed: int, sphere=UNIT_BALL) -> Rays:
    rng = rng_for(seed)
    return Rays(ball_points(N, rng, sphere), isotropic_dirs(N, rng))


def uniform_rays(N: int, seed: int, box=CUBE_BOX) -> Rays:
    rng = rng_for(seed)
    return Rays(uniform_points(N, rng, box), isotropic_dirs(N, rng))


def disk_rays(N: int, seed: int, box=DISK_BOX) -> Rays:
    rng = rng_for(seed)
    return Rays(disk_points(N, rng, box), isotropic_dirs(N, rng))


def detector_rays(npix: int, seed: int, box=DISK_BOX) -> Rays:
    """One +x ray per pixel of an npix x npix detector on the x = xmin face.

    Pixels tile y in [ymin, ymax] and z in [zmin, zmax]; each ray starts at
    its pixel centre plus a uniform jitter within the pixel.
    """
    rng = rng_for(seed)
    iy, iz = np.meshgrid(np.arange(npix), np.arange(npix), indexing="ij")
    iy = iy.ravel()
    iz = iz.ravel()
    dy = (box[4] - box[1]) / npix
    dz = (box[5] - box[2]) / npix
    y = box[1] + (iy + rng.random(iy.size)) * dy
    z = box[2] + (iz + rng.random(iz.size)) * dz
    o = np.stack([np.full(y.size, box[0]), y, z], axis=1)
    d = np.tile(np.array([1.0, 0.0, 0.0]), (y.size, 1))
    return Rays(o, d)


def lognormal_perturb(rho: np.ndarray, seed: int, sigma=0.1) -> np.ndarray:
    rng = rng_for(seed)
    return (rho.astype(np.float64) * np.exp(sigma * rng.standard_normal(rho.size))).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workload configurations.
# ---------------------------------------------------------------------------

def config1(n_rays=10_000):
    """1,000 uniform sites in [-1,1]^3, rho ~ U[0.5,1.5], 10^4 isotropic rays."""
    s = SEED_BASE + 1
    return make_uniform_grid(1000, s), uniform_rays(n_rays, s + 1000)


def config2(M=100_000, n_rays=1_000_000):
    """10^5 exponential-disk sites, rho = analytic disk density, 10^6 rays."""
    s = SEED_BASE + 2
    return make_disk_grid(M, s), disk_rays(n_rays, s + 1000)


def config3(M=1_000_000, n_rays=10_000_000):
    """10^6 clumpy sites (2,000 clumps), rho 1 / 100, 10^7 uniform rays."""
    s = SEED_BASE + 3
    n_clumps = max(1, round(2000 * M / 1_000_000))
    return make_clumpy_grid(M, s, n_clumps=n_clumps), uniform_rays(n_rays, s + 1000)


def config4_plan(G=64, seed=SEED_BASE + 4, site_lo=2_000, site_hi=200_000,
                 ray_lo=10_000, ray_hi=1_000_000):
    """Per-grid (kind, M, N) for the batched workload, log-uniform sizes."""
    rng = rng_for(seed)
    Ms = np.exp(rng.uniform(math.log(site_lo), math.log(site_hi), G)).astype(np.int64)
    Ns = np.exp(rng.uniform(math.log(ray_lo), math.log(ray_hi), G)).astype(np.int64)
    kinds = ["uniform" if g % 2 == 0 else "disk" for g in range(G)]
    return list(zip(kinds, Ms.tolist(), Ns.tolist()))


def config4(G=64, scale=1.0):
    """64 independent grids of uneven size; ``scale`` shrinks sizes for tests."""
    out = []
    for g, (kind, M, N) in enumerate(config4_plan(G)):
        M = max(8, int(M * scale))
        N = max(1, int(N * scale))
        s = SEED_BASE + 4 + 10_000 * (g + 1)
        if kind == "uniform":
            out.append((make_uniform_grid(M, s), uniform_rays(N, s + 1)))
        else:
            out.append((make_disk_grid(M, s), disk_rays(N, s + 1)))
    return out


def config5(M=1_000_000, npix=512, n_interior=1_000_000):
    """10^6-site disk; 512^2 jittered +x detector rays plus interior rays.

    Returns (grid, detector rays, interior rays, perturbed density rho').
    The loss target is exp(-tau) traced through rho'.
    """
    s = SEED_BASE + 5
    g = make_disk_grid(M, s)
    det = detector_rays(npix, s + 1000)
    inner = disk_rays(n_interior, s + 2000)
    rho_t = lognormal_perturb(g.rho, s + 3000)
    return g, det, inner, rho_t


def concat_rays(*rs: Rays) -> Rays:
    return Rays(np.concatenate([r.origin for r in rs]), np.concatenate([r.dir for r in rs]))


# ---------------------------------------------------------------------------
# Structured site sets used by the pins (lattices with known cells).
# ---------------------------------------------------------------------------

def cubic_lattice(n: int, box=CUBE_BOX):
    """n^3 sites at the centres of an n x n x n grid of cubes filling box."""
    lo, hi = box[:3], box[3:]
    h = (hi - lo) / n
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    return _round_f32(lo + (idx + 0.5) * h)


def bcc_lattice(n: int, box=CUBE_BOX):
    """Body-centred cubic lattice: cube centres plus cube corners strictly inside."""
    lo, hi = box[:3], box[3:]
    h = (hi - lo) / n
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    centres = lo + (idx + 0.5) * h
    cidx = np.stack(np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(1, n), indexing="ij"), -1).reshape(-1, 3)
    corners = lo + cidx * h
    return _round_f32(np.concatenate([centres, corners]))
