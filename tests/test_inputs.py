"""The seeded synthetic inputs follow their stated recipes (CPU).

Each generator in gen/ is checked against the distribution it claims:
Kolmogorov-Smirnov tests against the stated marginals (p > 1e-3 with
fixed seeds), exact checks of the densities written with the sites, and
counts of the degenerate starts and directions of the fuzz rays.
"""
import math

import numpy as np
import pytest

import gen
from tests import fuzz_cases

stats = pytest.importorskip("scipy.stats")


def _f32_exact(a):
    return np.array_equal(np.asarray(a, np.float64), np.asarray(a, np.float32).astype(np.float64))


def _inside(p, box):
    return np.all((p >= box[:3]) & (p <= box[3:]))


def test_uniform_grid_and_isotropic_rays():
    """C1: 1,000 uniform float32 sites in [-1,1]^3, rho ~ U[0.5, 1.5], rays
    from uniform points with isotropic directions."""
    g, rays = gen.config1()
    assert g.sites.shape == (1000, 3) and _f32_exact(g.sites) and _inside(g.sites, gen.CUBE_BOX)
    assert np.unique(g.sites, axis=0).shape[0] == 1000
    for c in range(3):
        assert stats.kstest(g.sites[:, c], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert g.rho.dtype == np.float32 and g.rho.min() >= 0.5 and g.rho.max() <= 1.5
    assert stats.kstest(g.rho, stats.uniform(0.5, 1.0).cdf).pvalue > 1e-3
    O, D = rays.origin, rays.dir
    assert O.shape == (10_000, 3) and _inside(O, gen.CUBE_BOX)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, rtol=1e-15)
    # isotropic: each component of a uniform unit vector is U[-1, 1]
    for c in range(3):
        assert stats.kstest(D[:, c], stats.uniform(-1, 2).cdf).pvalue > 1e-3


def _truncated(dist, lo, hi):
    a, b = dist.cdf(lo), dist.cdf(hi)
    return lambda x: (dist.cdf(x) - a) / (b - a)


def test_disk_sites_follow_the_exponential_disk():
    """C2: density exp(-R - |z|/0.1) in [-4,4]^2 x [-0.5,0.5]: R ~ Gamma(2,1)
    (the box cuts it only beyond R = 4), z ~ Laplace(0, 0.1) cut at |z| =
    0.5, azimuth uniform; rho is that density at the site."""
    g = gen.make_disk_grid(20_000, gen.SEED_BASE + 2)
    S = g.sites
    assert _f32_exact(S) and _inside(S, gen.DISK_BOX)
    R = np.hypot(S[:, 0], S[:, 1])
    r_in = R[R < 4.0]
    assert stats.kstest(r_in, _truncated(stats.gamma(2.0), 0.0, 4.0)).pvalue > 1e-3
    assert stats.kstest(S[:, 2], _truncated(stats.laplace(0.0, 0.1), -0.5, 0.5)).pvalue > 1e-3
    phi = np.arctan2(S[:, 1], S[:, 0])[R < 4.0]
    assert stats.kstest(phi, stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3
    want = np.exp(-R - np.abs(S[:, 2]) / 0.1).astype(np.float32)
    np.testing.assert_array_equal(g.rho, want)


def test_disk_rays_start_from_the_same_sampler():
    rays = gen.disk_rays(20_000, gen.SEED_BASE + 1002)
    O = rays.origin
    assert _inside(O, gen.DISK_BOX)
    R = np.hypot(O[:, 0], O[:, 1])
    assert stats.kstest(R[R < 4.0], _truncated(stats.gamma(2.0), 0.0, 4.0)).pvalue > 1e-3
    assert stats.kstest(O[:, 2], _truncated(stats.laplace(0.0, 0.1), -0.5, 0.5)).pvalue > 1e-3


def test_clumpy_sites_are_seventy_percent_uniform():
    """C3: 70 % uniform sites and 30 % in Gaussian clumps (sigma in [0.01,
    0.05]); rho is 1 for the uniform sites and 100 for the clumped ones."""
    rng = gen.rng_for(7)
    p, flag = gen.clumpy_points(20_000, rng, n_clumps=40)
    assert _inside(p, gen.CUBE_BOX)
    assert flag.sum() == 6000
    for c in range(3):
        assert stats.kstest(p[~flag, c], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    # the clumped sites are far denser: their nearest neighbours are much closer
    from scipy.spatial import cKDTree
    t = cKDTree(p)
    d, _ = t.query(p, k=2)
    assert np.median(d[flag, 1]) < 0.3 * np.median(d[~flag, 1])
    g = gen.make_clumpy_grid(20_000, gen.SEED_BASE + 3, n_clumps=40)
    assert set(np.unique(g.rho).tolist()) == {1.0, 100.0}
    assert abs(float(np.mean(g.rho == 100.0)) - 0.3) < 0.01


def test_batch_plan_is_log_uniform_and_alternates():
    """C4: 64 grids, sites log-uniform in [2e3, 2e5], rays in [1e4, 1e6],
    uniform and disk placement alternating."""
    plan = gen.config4_plan()
    assert len(plan) == 64
    kinds = [k for k, _, _ in plan]
    assert kinds == ["uniform" if g % 2 == 0 else "disk" for g in range(64)]
    M = np.array([m for _, m, _ in plan], np.float64)
    N = np.array([n for _, _, n in plan], np.float64)
    assert M.min() >= 2_000 - 1 and M.max() <= 200_000
    assert N.min() >= 10_000 - 1 and N.max() <= 1_000_000
    lo, hi = math.log(2_000), math.log(200_000)
    assert stats.kstest(np.log(M), stats.uniform(lo, hi - lo).cdf).pvalue > 1e-3
    lo, hi = math.log(10_000), math.log(1_000_000)
    assert stats.kstest(np.log(N), stats.uniform(lo, hi - lo).cdf).pvalue > 1e-3


def test_detector_rays_one_per_pixel():
    """C5: one +x ray per pixel of an npix^2 detector on the x = xmin face,
    each inside its own pixel."""
    npix = 32
    r = gen.detector_rays(npix, gen.SEED_BASE + 1005)
    box = gen.DISK_BOX
    assert r.origin.shape == (npix * npix, 3)
    assert np.all(r.origin[:, 0] == box[0])
    np.testing.assert_array_equal(r.dir, np.tile([1.0, 0.0, 0.0], (npix * npix, 1)))
    iy = np.floor((r.origin[:, 1] - box[1]) / ((box[4] - box[1]) / npix)).astype(int)
    iz = np.floor((r.origin[:, 2] - box[2]) / ((box[5] - box[2]) / npix)).astype(int)
    cells = set(zip(iy.tolist(), iz.tolist()))
    assert len(cells) == npix * npix and min(iy) >= 0 and max(iy) < npix and min(iz) >= 0 and max(iz) < npix


def test_perturbed_density_is_lognormal():
    """C5's target density: rho' = rho exp(0.1 xi), xi ~ N(0, 1) per cell."""
    rho = np.full(20_000, 2.0, np.float32)
    rp = gen.lognormal_perturb(rho, 11)
    xi = np.log(rp.astype(np.float64) / 2.0) / 0.1
    assert stats.kstest(xi, stats.norm().cdf).pvalue > 1e-3


def test_ball_grid_recipe():
    """Spherical domain: sites uniform in the unit ball (|r|^3 uniform on
    [0, 1]), rho = exp(-3 |r|)."""
    g = gen.make_ball_grid(20_000, 5)
    r = np.linalg.norm(g.sites, axis=1)
    assert r.max() <= 1.0 and _f32_exact(g.sites)
    assert stats.kstest(r ** 3, stats.uniform(0, 1).cdf).pvalue > 1e-3
    np.testing.assert_array_equal(g.rho, np.exp(-r / (1.0 / 3.0)).astype(np.float32))


def test_fuzz_cases_follow_their_recipe():
    """Degenerate grids: kinds in turn, boxes with edges in [0.125, 8] and
    float32 bounds, sites inside and float32-exact, kappa a float32 value in
    [0.5, 2]; of the 300 rays about a tenth start on a site, a tenth on a
    wall, a fifth run exactly along an axis."""
    on_site = on_wall = along_axis = total = 0
    for i in range(24):
        kind, g, rays = fuzz_cases.case(i)
        assert kind == fuzz_cases.KINDS[i % len(fuzz_cases.KINDS)]
        ext = g.box[3:] - g.box[:3]
        assert np.all(ext >= 0.125 * 0.999) and np.all(ext <= 8.0 * 1.001)
        assert _f32_exact(g.box) and _f32_exact(g.sites) and _inside(g.sites, g.box)
        assert np.unique(g.sites, axis=0).shape[0] == g.sites.shape[0]
        assert 0.5 <= g.kappa <= 2.0 and float(np.float32(g.kappa)) == g.kappa
        O, D = rays.origin, rays.dir
        assert _inside(O, g.box)
        np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, rtol=1e-15)
        site_set = {tuple(s) for s in g.sites.tolist()}
        on_site += sum(tuple(o) in site_set for o in O.tolist())
        on_wall += int(np.sum(np.any((O == g.box[:3]) | (O == g.box[3:]), axis=1)))
        along_axis += int(np.sum(np.sum(D != 0.0, axis=1) == 1))
        total += O.shape[0]
    assert 0.07 < on_site / total < 0.14
    assert 0.07 < on_wall / total < 0.16   # wall starts, plus the few sites on walls
    assert 0.16 < along_axis / total < 0.24
