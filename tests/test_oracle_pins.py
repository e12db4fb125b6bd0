"""Pins of the CPU oracle against facts other than itself.

Each test checks the oracle against a hand-worked example, a textbook or
library routine, a closed form, an invariant or brute force, chosen so that a
dropped term, a sign error, a wrong index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from tests.helpers import dda_voxels, nearest_site, slab_length

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _full(sites, box):
    c = oracle.cells(sites, box)
    off, idx = oracle.csr(c, len(sites))
    return c, off, idx


# --------------------------------------------------------------------------
# hand-worked examples (Sect. 2.2, Eq. 1-5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _load("worked_examples.json")["cases"], ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", ["neighbours", "all_sites"])
def test_worked_examples(case, mode):
    S = np.array(case["sites"], np.float64)
    box = np.array(case["box"], np.float64)
    rho = np.array(case["rho"], np.float64)
    O = np.array([case["origin"]], np.float64)
    D = np.array([case["dir"]], np.float64)
    kw = {}
    if mode == "neighbours":
        _, off, idx = _full(S, box)
        kw = dict(off=off, idx=idx)
    tr = oracle.trace(S, box, rho, O, D, kappa=case["kappa"], **kw)
    cells, lens = tr.segments(0)
    exp = case["segments"]
    assert [int(c) for c in cells] == [e[0] for e in exp]
    np.testing.assert_allclose(lens, [e[1] for e in exp], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr.tau[0], case["tau"], rtol=1e-12)
    assert oracle.STATUS[int(tr.status[0])] == case.get("status", "ok")


@pytest.mark.parametrize("case", _load("fallback_examples.json")["cases"], ids=lambda c: c["name"])
def test_fallback_examples(case):
    """The epsilon nudge of Sect. 2.2, on hand-worked paths: a start on a
    face or at a lattice vertex whose zero-length steps exceed the limit Z,
    and a list without an exit (the branch that finds no candidate)."""
    box = np.array(case["box"], np.float64)
    if "lattice" in case:
        S = gen.cubic_lattice(case["lattice"], box)
        rho = np.full(len(S), case["rho_all"])
    else:
        S = np.array(case["sites"], np.float64)
        rho = np.array(case["rho"], np.float64)
    if "lists" in case:
        lists = case["lists"]
        off = np.concatenate([[0], np.cumsum([len(a) for a in lists])]).astype(np.int64)
        idx = np.concatenate([np.array(a, np.int32) for a in lists])
    else:
        _, off, idx = _full(S, box)
    O = np.array([case["origin"]], np.float64)
    D = np.array([case["dir"]], np.float64)
    tr = oracle.trace(S, box, rho, O, D, off=off, idx=idx, kappa=case["kappa"], zero_run_max=case["zero_run_max"])
    assert tr.status[0] == 0
    assert int(tr.nfallback[0]) == case["nfallback"]
    cells, lens = tr.segments(0)
    assert [int(c) for c in cells] == [e[0] for e in case["segments"]]
    np.testing.assert_allclose(lens, [e[1] for e in case["segments"]], rtol=0, atol=case["len_atol"])
    assert abs(tr.tau[0] - case["tau"]) <= case["len_atol"] * max(1.0, float(rho.max()))
    np.testing.assert_allclose(tr.length[0], sum(e[1] for e in case["segments"]), rtol=0, atol=4 * case["len_atol"])


def test_fallback_all_sites_definition_agrees():
    """The nudge cases through lattice vertices give the same path with every
    site as a candidate (the plain definition of the exit)."""
    for case in _load("fallback_examples.json")["cases"]:
        if "lattice" not in case:
            continue
        box = np.array(case["box"], np.float64)
        S = gen.cubic_lattice(case["lattice"], box)
        rho = np.full(len(S), case["rho_all"])
        O = np.array([case["origin"]], np.float64)
        D = np.array([case["dir"]], np.float64)
        tr = oracle.trace(S, box, rho, O, D, zero_run_max=case["zero_run_max"])
        assert int(tr.nfallback[0]) == case["nfallback"]
        assert [int(c) for c in tr.segments(0)[0]] == [e[0] for e in case["segments"]]
        np.testing.assert_allclose(tr.segments(0)[1], [e[1] for e in case["segments"]], rtol=0,
                                   atol=case["len_atol"])


def test_fallback_lengths_lose_epsilon_per_nudge():
    """Rays that start on lattice faces, edges and vertices (zero-length
    steps) traced with Z = 4 and Z = 0: with Z = 0 every nudge skips exactly
    epsilon of the path, so the summed length is the slab length minus
    epsilon times the nudges, to rounding; with Z = 4 it is the slab length."""
    n = 8
    S = gen.cubic_lattice(n)
    _, off, idx = _full(S, gen.CUBE_BOX)
    rng = gen.rng_for(401)
    m = 300
    # points on lattice planes: one, two or three coordinates on a plane
    P = rng.uniform(-0.95, 0.95, (m, 3))
    planes = np.arange(1, n) * 0.25 - 1.0
    for i in range(m):
        k = 1 + i % 3
        for a in rng.choice(3, k, replace=False):
            P[i, a] = rng.choice(planes)
    D = gen.isotropic_dirs(m, rng)
    L = slab_length(gen.CUBE_BOX, P, D)
    eps = oracle.default_eps(gen.CUBE_BOX)
    t4 = oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), P, D, off=off, idx=idx, zero_run_max=4)
    t0 = oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), P, D, off=off, idx=idx, zero_run_max=0)
    assert np.all(t4.nfallback == 0) and np.all(t0.status == 0)
    assert t0.nfallback.sum() >= m // 2
    np.testing.assert_allclose(t4.length, L, rtol=1e-12)
    err = np.abs(t0.length - (L - eps * t0.nfallback))
    assert np.all(err <= 1e-14 + 1e-15 * t0.nseg), err.max()
    # the cells crossed after each nudge are those of Z = 4 (the nudge is far
    # smaller than the lattice spacing)
    for i in range(m):
        assert np.array_equal(t0.segments(i)[0], t4.segments(i)[0]), i


def test_shell_search_equals_brute_force_disk():
    """The shell-by-shell candidate search (buckets, first shell from the local
    density) against clipping by every site, on a grid whose density spans
    orders of magnitude."""
    g = gen.make_disk_grid(3000, 402)
    ids = np.concatenate([np.arange(0, 3000, 7)])
    a = oracle.cells(g.sites, g.box, ids=ids)
    b = oracle.cells(g.sites, g.box, ids=ids, brute=True)
    for k in range(ids.size):
        assert np.array_equal(a.nbr[k], b.nbr[k]), ids[k]
    np.testing.assert_allclose(a.vol, b.vol, rtol=1e-11)
    np.testing.assert_allclose(a.bbox, b.bbox, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# cells: lattices with known cells, Delaunay adjacency, Monte Carlo volumes
# --------------------------------------------------------------------------

def test_cubic_lattice_cells_are_cubes():
    n = 4  # spacing 0.5: the lattice is exact in float32
    S = gen.cubic_lattice(n)
    c = oracle.cells(S, gen.CUBE_BOX)
    h = 2.0 / n
    np.testing.assert_allclose(c.vol, h ** 3, rtol=1e-12)
    idx = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for m, (i, j, k) in enumerate(idx):
        exp = set()
        for a, (v, lo_wall, hi_wall) in enumerate([(i, -1, -2), (j, -3, -4), (k, -5, -6)]):
            for dv, wall in ((-1, lo_wall), (1, hi_wall)):
                w = v + dv
                if 0 <= w < n:
                    q = [i, j, k]
                    q[a] = w
                    exp.add(q[0] * n * n + q[1] * n + q[2])
                else:
                    exp.add(wall)
        assert set(c.nbr[m].tolist()) == exp, m
        np.testing.assert_allclose(c.bbox[m, :3], S[m] - h / 2, atol=1e-12)
        np.testing.assert_allclose(c.bbox[m, 3:], S[m] + h / 2, atol=1e-12)


def test_bcc_interior_cells_are_truncated_octahedra():
    n = 8  # spacing 0.25: exact in float32
    S = gen.bcc_lattice(n)
    c = oracle.cells(S, gen.CUBE_BOX)
    h = 2.0 / n
    # points whose 14 lattice neighbours all exist (the lattice stops at the walls)
    interior = np.all(np.abs(S) < 1 - 1.2 * h, axis=1)
    assert interior.sum() > 10
    deg = np.array([a.size for a in c.nbr])
    assert np.all(deg[interior] == 14)
    # two lattice points per cube of side h
    np.testing.assert_allclose(c.vol[interior], h ** 3 / 2, rtol=1e-12)
    # 8 hexagonal faces of area (3*sqrt(3)/2) a^2 and 6 squares of area a^2, a = h / (2 sqrt 2)
    a = h / (2 * np.sqrt(2))
    for m in np.nonzero(interior)[0][:5]:
        ar = np.sort(c.area[m])
        np.testing.assert_allclose(ar[:6], a * a, rtol=1e-10)
        np.testing.assert_allclose(ar[6:], 1.5 * np.sqrt(3) * a * a, rtol=1e-10)
    np.testing.assert_allclose(c.vol.sum(), 8.0, rtol=1e-12)


@pytest.fixture(scope="module")
def grid300():
    g = gen.make_uniform_grid(300, 11)
    c, off, idx = _full(g.sites, g.box)
    return g, c, off, idx


def test_symmetry_volume_and_bbox(grid300):
    g, c, off, idx = grid300
    M = len(g.sites)
    pairs = {(m, int(j)) for m in range(M) for j in c.nbr[m] if j >= 0}
    assert all((j, m) in pairs for (m, j) in pairs)
    np.testing.assert_allclose(c.vol.sum(), 8.0, rtol=1e-12)
    assert np.all(c.bbox[:, :3] <= g.sites + 1e-15) and np.all(c.bbox[:, 3:] >= g.sites - 1e-15)
    assert np.all(c.bbox[:, :3] >= g.box[:3] - 1e-12) and np.all(c.bbox[:, 3:] <= g.box[3:] + 1e-12)


def test_security_radius_equals_brute_force(grid300):
    g, c, off, idx = grid300
    b = oracle.cells(g.sites, g.box, brute=True)
    for m in range(len(g.sites)):
        assert np.array_equal(b.nbr[m], c.nbr[m])
    np.testing.assert_allclose(b.vol, c.vol, rtol=1e-11)


def test_neighbours_are_delaunay_edges(grid300):
    spatial = pytest.importorskip("scipy.spatial")
    g, c, off, idx = grid300
    tri = spatial.Delaunay(g.sites)
    edges = set()
    for s in tri.simplices:
        for a in range(4):
            for b in range(a + 1, 4):
                edges.add((min(s[a], s[b]), max(s[a], s[b])))
    ours = {(min(m, int(j)), max(m, int(j))) for m in range(len(g.sites)) for j in c.nbr[m] if j >= 0}
    assert ours <= edges
    # cells far from the walls keep every Delaunay edge (their faces are not clipped)
    far = np.nonzero(np.all(np.abs(g.sites) < 0.5, axis=1) & np.all(np.abs(c.bbox) < 0.95, axis=1))[0]
    assert far.size > 5
    for m in far:
        dl = {b if a == m else a for (a, b) in edges if m in (a, b)}
        assert dl == set(c.nbr[m].tolist())


def test_volumes_match_monte_carlo(grid300):
    g, c, off, idx = grid300
    rng = gen.rng_for(77)
    P = gen.uniform_points(200_000, rng)
    owner = nearest_site(g.sites, P)
    frac = np.bincount(owner, minlength=len(g.sites)) / P.shape[0]
    est = frac * 8.0
    # aggregate check over random groups of 30 cells (binomial error ~ 1.5 %)
    perm = rng.permutation(len(g.sites))[:300].reshape(10, 30)
    for grp in perm:
        v = c.vol[grp].sum()
        sd = np.sqrt(v / 8 * (1 - v / 8) / P.shape[0]) * 8
        assert abs(est[grp].sum() - v) < 5 * sd


def test_mean_degree_uniform_interior():
    """Sect. 2.1: mean neighbour count 15.54 for uniform random sites."""
    const = _load("paper_constants.json")["mean_neighbour_count_uniform"]["value"]
    g = gen.make_uniform_grid(40_000, 12)
    ids = np.nonzero(np.all(np.abs(g.sites) < 0.6, axis=1))[0][:3000]
    c = oracle.cells(g.sites, g.box, ids=ids)
    deg = np.array([a.size for a in c.nbr])
    assert not np.any(np.concatenate(c.nbr) < 0)
    se = deg.std() / np.sqrt(deg.size)
    assert abs(deg.mean() - const) < 4 * se + 0.02, (deg.mean(), se)


# --------------------------------------------------------------------------
# locate
# --------------------------------------------------------------------------

def test_locate_matches_numpy_and_lattice():
    g = gen.make_uniform_grid(500, 13)
    rng = gen.rng_for(5)
    P = gen.uniform_points(3000, rng)
    np.testing.assert_array_equal(oracle.locate(g.sites, g.box, P), nearest_site(g.sites, P))
    out = np.array([[1.5, 0, 0], [0, -1.0001, 0], [0, 0, 2]])
    assert np.all(oracle.locate(g.sites, g.box, out) == -1)
    # boundary points are inside (closed box)
    assert oracle.locate(g.sites, g.box, np.array([[1.0, 1.0, -1.0]]))[0] >= 0
    n = 4
    S = gen.cubic_lattice(n)
    P = gen.uniform_points(2000, rng)
    v = np.minimum(np.floor((P + 1) / 0.5).astype(int), n - 1)
    np.testing.assert_array_equal(oracle.locate(S, gen.CUBE_BOX, P), v[:, 0] * 16 + v[:, 1] * 4 + v[:, 2])


# --------------------------------------------------------------------------
# trace
# --------------------------------------------------------------------------

def test_cubic_lattice_trace_is_dda():
    n = 8  # spacing 0.25: the lattice is exact in float32
    S = gen.cubic_lattice(n)
    box = gen.CUBE_BOX
    c, off, idx = _full(S, box)
    rays = gen.uniform_rays(200, 99)
    rho = np.ones(len(S))
    tr = oracle.trace(S, box, rho, rays.origin, rays.dir, off=off, idx=idx)
    for i in range(200):
        ref = dda_voxels(box, n, rays.origin[i], rays.dir[i])
        cells, lens = tr.segments(i)
        assert [int(c_) for c_ in cells] == [v[0] * n * n + v[1] * n + v[2] for v, _ in ref]
        np.testing.assert_allclose(lens, [l for _, l in ref], rtol=1e-11, atol=1e-13)


@pytest.fixture(scope="module")
def traced300(grid300):
    g, c, off, idx = grid300
    rays = gen.uniform_rays(2000, 21)
    tr = oracle.trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx)
    return g, c, off, idx, rays, tr


def test_lengths_sum_to_slab_length(traced300):
    g, c, off, idx, rays, tr = traced300
    L = slab_length(g.box, rays.origin, rays.dir)
    assert np.all(tr.status == 0)
    np.testing.assert_allclose(tr.length, L, rtol=1e-13, atol=1e-15)


def test_segments_lie_in_their_cells(traced300):
    """Midpoint of each segment is nearest to its cell's site; each exit point
    is equidistant from the two sites it separates (bisector property)."""
    g, c, off, idx, rays, tr = traced300
    S = g.sites
    diag = np.linalg.norm(g.box[3:] - g.box[:3])
    mids, owners, exits, pairs = [], [], [], []
    for i in range(300):
        cells, lens = tr.segments(i)
        t = np.concatenate([[0.0], np.cumsum(lens)])
        for a in range(cells.size):
            mids.append(rays.origin[i] + 0.5 * (t[a] + t[a + 1]) * rays.dir[i])
            owners.append(cells[a])
            if a + 1 < cells.size:
                exits.append(rays.origin[i] + t[a + 1] * rays.dir[i])
                pairs.append((cells[a], cells[a + 1]))
    np.testing.assert_array_equal(nearest_site(S, np.array(mids)), np.array(owners))
    q = np.array(exits)
    pr = np.array(pairs)
    d1 = np.linalg.norm(q - S[pr[:, 0]], axis=1)
    d2 = np.linalg.norm(q - S[pr[:, 1]], axis=1)
    assert np.max(np.abs(d1 - d2)) <= 1e-12 * diag


def test_dense_sampling_reproduces_cell_sequence():
    g = gen.make_uniform_grid(150, 31)
    c, off, idx = _full(g.sites, g.box)
    rays = gen.uniform_rays(60, 32)
    tr = oracle.trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx)
    L = slab_length(g.box, rays.origin, rays.dir)
    checked = 0
    for i in range(60):
        cells, lens = tr.segments(i)
        if lens.min() < 2e-3:
            continue  # a segment shorter than the sampling step cannot be resolved
        ts = np.arange(0.0, L[i], 2.5e-4) + 1.25e-4
        own = nearest_site(g.sites, rays.origin[i] + ts[:, None] * rays.dir[i])
        runs = own[np.concatenate([[True], own[1:] != own[:-1]])]
        assert [int(x) for x in runs] == [int(x) for x in cells]
        checked += 1
    assert checked > 40


def test_neighbour_exit_equals_all_sites_exit(traced300):
    g, c, off, idx, rays, tr = traced300
    tr2 = oracle.trace(g.sites, g.box, g.rho, rays.origin[:400], rays.dir[:400])
    for i in range(400):
        a, la = tr.segments(i)
        b, lb = tr2.segments(i)
        assert np.array_equal(a, b)
        np.testing.assert_array_equal(la, lb)


def test_uniform_density_closed_form(grid300):
    g, c, off, idx = grid300
    rays = gen.uniform_rays(500, 41)
    rho = np.full(len(g.sites), 1.75)
    tr = oracle.trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, kappa=2.0)
    L = slab_length(g.box, rays.origin, rays.dir)
    np.testing.assert_allclose(tr.tau, 2.0 * 1.75 * L, rtol=1e-13)


def test_tau_matches_midpoint_riemann_sum(grid300):
    g, c, off, idx = grid300
    rays = gen.uniform_rays(40, 42)
    tr = oracle.trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx)
    L = slab_length(g.box, rays.origin, rays.dir)
    for i in range(40):
        K = 20000
        h = L[i] / K
        ts = (np.arange(K) + 0.5) * h
        own = nearest_site(g.sites, rays.origin[i] + ts[:, None] * rays.dir[i])
        riemann = h * g.rho[own].astype(np.float64).sum()
        # each cell boundary contributes at most h * max|rho jump|
        assert abs(riemann - tr.tau[i]) <= (tr.nseg[i] + 1) * h * 1.0 + 1e-12


def test_gradient_matches_finite_differences(grid300):
    g, c, off, idx = grid300
    rays = gen.uniform_rays(400, 43)
    rho = g.rho.astype(np.float64)
    tr = oracle.trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3)
    target = np.exp(-tr.tau * 0.9)
    loss, dL = oracle.exp_loss(tr.tau, target)
    grad = oracle.tau_grad(tr, len(g.sites), dL, kappa=1.3)
    rng = gen.rng_for(3)
    hit = np.unique(np.concatenate([tr.segments(i)[0] for i in range(400)]))
    for cidx in rng.choice(hit, 15, replace=False):
        hh = 1e-4 * rho[cidx]
        rp = rho.copy(); rp[cidx] += hh
        rm = rho.copy(); rm[cidx] -= hh
        tp = oracle.trace(g.sites, g.box, rp, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3).tau
        tm = oracle.trace(g.sites, g.box, rm, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3).tau
        fd = (oracle.exp_loss(tp, target)[0] - oracle.exp_loss(tm, target)[0]) / (2 * hh)
        assert abs(fd - grad[cidx]) <= 1e-6 * max(abs(fd), 1e-8), (cidx, fd, grad[cidx])
    miss = np.setdiff1d(np.arange(len(g.sites)), hit)
    assert np.all(grad[miss] == 0.0)


def test_edge_ray_is_flagged_near_tie():
    n = 4
    S = gen.cubic_lattice(n)
    c, off, idx = _full(S, gen.CUBE_BOX)
    # a ray starting on the face plane y = 0: the start is equidistant from two sites
    O = np.array([[-0.9, 0.0, 0.13]])
    D = np.array([[0.8, 0.0, 0.6]])
    tr = oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), O, D, off=off, idx=idx)
    assert tr.near_tie[0] == 1
    L = slab_length(gen.CUBE_BOX, O, D)
    np.testing.assert_allclose(tr.length, L, rtol=1e-12)
    # a ray aimed at the cell edge x = -0.5, y = 0: two exit planes tie
    O = np.array([[-0.9, -0.1, 0.13]])
    D = np.array([[0.4, 0.1, 0.07]])
    D = D / np.linalg.norm(D)
    tr = oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), O, D, off=off, idx=idx)
    assert tr.near_tie[0] == 1 and tr.min_margin[0] <= 1e-9
    np.testing.assert_allclose(tr.length, slab_length(gen.CUBE_BOX, O, D), rtol=1e-12)
    # a generic ray is not
    O = np.array([[-0.9, 0.0123, 0.13]])
    D = np.array([[0.8, 0.1, 0.6]]) / np.linalg.norm([0.8, 0.1, 0.6])
    assert oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), O, D, off=off, idx=idx).near_tie[0] == 0


def test_vertex_ray_zero_length_steps():
    """A ray through a lattice vertex (eight cubes meet) crosses several cells
    at one point; zero-length steps emit nothing and the path still ends at
    the wall."""
    n = 4
    S = gen.cubic_lattice(n)
    c, off, idx = _full(S, gen.CUBE_BOX)
    D = np.array([[1.0, 1.0, 1.0]]) / np.sqrt(3)
    O = np.array([[-0.75, -0.75, -0.75]])
    tr = oracle.trace(S, gen.CUBE_BOX, np.ones(len(S)), O, D, off=off, idx=idx)
    assert tr.status[0] == 0 and tr.near_tie[0] == 1
    np.testing.assert_allclose(tr.length, slab_length(gen.CUBE_BOX, O, D), rtol=1e-12)
    cells, lens = tr.segments(0)
    assert np.all(lens > 0)
    # the diagonal visits the diagonal cubes (i, i, i)
    diag = [i * 16 + i * 4 + i for i in range(n)]
    assert [int(x) for x in cells] == diag


def test_status_codes():
    g = gen.make_uniform_grid(50, 51)
    c, off, idx = _full(g.sites, g.box)
    O = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [3.0, 0.0, 0.0]])
    D = np.array([[1.0, 0, 0], [1.0, 0, 0], [1.0, 0, 0]])
    tr = oracle.trace(g.sites, g.box, g.rho, O, D, off=off, idx=idx, cap=1)
    assert tr.status[2] == 1
    assert tr.status[0] in (0, 3)
    tr = oracle.trace(g.sites, g.box, g.rho, O[:1], D[:1], off=off, idx=idx, max_steps=1)
    assert tr.status[0] == 2 or tr.nseg[0] == 1


# --------------------------------------------------------------------------
# interaction sampling (the Monte Carlo step that consumes the path)
# --------------------------------------------------------------------------

def test_interaction_hand_worked():
    """Two sites at (1,1,1), (3,1,1) in [0,4]^3, rho 2 and 3, ray from
    (0.5,1,1) along +x: tau is 3 at x = 2 (after 1.5 in cell 0), so
    tau_int = 4 is reached 1/3 further, in cell 1; the package loses
    1 - e^-3 in cell 0 and e^-3 - e^-4 in cell 1. tau_int = 10 exceeds the
    total 3 + 3*2 = 9: the ray leaves after 3.5."""
    S = np.array([[1.0, 1, 1], [3.0, 1, 1]])
    box = np.array([0.0, 0, 0, 4, 4, 4])
    rho = np.array([2.0, 3.0])
    c, off, idx = _full(S, box)
    tr = oracle.trace(S, box, rho, np.array([[0.5, 1, 1]] * 2), np.array([[1.0, 0, 0]] * 2), off=off, idx=idx)
    cell, s, ab, amb = oracle.interact(tr, rho, [4.0, 10.0], weight=[1.0, 2.0])
    assert list(cell) == [1, -1]
    np.testing.assert_allclose(s, [1.5 + 1.0 / 3.0, 3.5], rtol=1e-14)
    np.testing.assert_allclose(ab, [(1 - np.exp(-3)) * 3.0, (np.exp(-3) - np.exp(-4)) + 2 * (np.exp(-3) - np.exp(-9))],
                               rtol=1e-13)
    assert not amb.any()


def test_interaction_through_empty_cells():
    """A cell of zero density adds length but no optical depth, and takes
    nothing from the package. Three sites at x = 1, 3, 5 in [0,6] x [0,2]^2
    with rho 0, 3, 0 and kappa 2; a ray from (0.5, 1, 1) along +x crosses
    1.5 of cell 0, 2 of cell 1 (tau 12) and 2 of cell 2. tau_int = 6 is
    reached 1 into cell 1 (s = 2.5); tau_int = 20 is never reached, and
    the ray leaves after 5.5 having lost 1 - e^-12, all in cell 1."""
    S = np.array([[1.0, 1, 1], [3.0, 1, 1], [5.0, 1, 1]])
    box = np.array([0.0, 0, 0, 6, 2, 2])
    rho = np.array([0.0, 3.0, 0.0])
    c, off, idx = _full(S, box)
    tr = oracle.trace(S, box, rho, np.array([[0.5, 1, 1]] * 2), np.array([[1.0, 0, 0]] * 2), off=off, idx=idx,
                      kappa=2.0)
    np.testing.assert_allclose(tr.tau, [12.0, 12.0], rtol=1e-15)
    cell, s, ab, amb = oracle.interact(tr, rho, [6.0, 20.0], kappa=2.0)
    assert list(cell) == [1, -1]
    np.testing.assert_allclose(s, [2.5, 5.5], rtol=1e-14)
    np.testing.assert_allclose(ab, [0.0, (1 - np.exp(-6)) + (1 - np.exp(-12)), 0.0], rtol=1e-14, atol=0)
    assert not amb.any()
    grad = oracle.tau_grad(tr, 3, [1.0, 1.0], kappa=2.0)
    # dtau/drho_c = kappa l_c, whatever rho_c is
    np.testing.assert_allclose(grad, [2 * 2 * 1.5, 2 * 2 * 2.0, 2 * 2 * 2.0], rtol=1e-14)


def test_interaction_uniform_closed_form_and_conservation(grid300):
    g, c, off, idx = grid300
    rays = gen.uniform_rays(400, 61)
    rho = np.full(len(g.sites), 0.8)
    tr = oracle.trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, kappa=1.5)
    rng = gen.rng_for(62)
    tau_int = -np.log(rng.random(400))
    w = rng.uniform(0.5, 2.0, 400)
    cell, s, ab, amb = oracle.interact(tr, rho, tau_int, weight=w, kappa=1.5)
    L = slab_length(g.box, rays.origin, rays.dir)
    inside = tau_int < 1.5 * 0.8 * L
    # uniform medium: the interaction distance is tau_int / (kappa rho)
    np.testing.assert_allclose(s[inside], tau_int[inside] / 1.2, rtol=1e-12)
    np.testing.assert_allclose(s[~inside], L[~inside], rtol=1e-12)
    assert np.all(cell[~inside] == -1) and np.all(cell[inside] >= 0)
    # the interaction point lies in the reported cell
    pts = rays.origin[inside] + s[inside, None] * rays.dir[inside]
    ok = ~amb[inside]
    np.testing.assert_array_equal(nearest_site(g.sites, pts[ok]), cell[inside][ok])
    # what the cells remove is what the package lost
    lost = w * (1 - np.exp(-np.minimum(tau_int, 1.2 * L)))
    np.testing.assert_allclose(ab.sum(), lost.sum(), rtol=1e-12)


def test_enter_points_closed_form():
    box = gen.CUBE_BOX
    O = np.array([[-2.0, 0.1, 0.2], [0.5, 3.0, -0.25], [2.0, 2.0, 2.0], [-3.0, 0.0, 0.0], [0.1, 0.2, 0.3]])
    D = np.array([[1.0, 0, 0], [0.0, -1, 0], [-1.0, -1, -1], [-1.0, 0, 0], [0.6, 0.8, 0.0]])
    D = D / np.linalg.norm(D, axis=1)[:, None]
    E = oracle.enter_points(box, O, D)
    np.testing.assert_allclose(E[0], [-1.0, 0.1, 0.2])
    np.testing.assert_allclose(E[1], [0.5, 1.0, -0.25])
    np.testing.assert_allclose(E[2], [1.0, 1.0, 1.0], rtol=1e-15)      # enters at the corner
    np.testing.assert_array_equal(E[3], O[3])                            # points away: misses
    np.testing.assert_array_equal(E[4], O[4])                            # already inside
    # random rays: an entry point is on the boundary and continues into the box
    rng = gen.rng_for(71)
    O = gen.uniform_points(2000, rng, np.array([-3.0, -3, -3, 3, 3, 3]))
    D = gen.isotropic_dirs(2000, rng)
    E = oracle.enter_points(box, O, D)
    outside = ~np.all((O >= -1) & (O <= 1), axis=1)
    moved = outside & np.any(E != O, axis=1)
    assert moved.sum() > 100
    on_face = np.any(np.isclose(np.abs(E[moved]), 1.0, rtol=0, atol=1e-14), axis=1)
    assert np.all(on_face)
    ahead = E[moved] + 1e-9 * D[moved]
    assert np.all(np.abs(ahead) <= 1 + 1e-12)
    # the missed rays never reach the box (checked by dense sampling)
    missed = outside & ~np.any(E != O, axis=1)
    ts = np.linspace(0, 12, 4001)
    for i in np.nonzero(missed)[0][:100]:
        p = O[i] + ts[:, None] * D[i]
        assert not np.any(np.all(np.abs(p) <= 1 - 1e-9, axis=1))


# --------------------------------------------------------------------------
# a spherical domain (Sect. 2.2: the method carries over to other domain
# geometries): cells keep the box's lists, the path ends on the sphere
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _load("sphere_examples.json")["cases"], ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", ["neighbours", "all_sites"])
def test_sphere_examples(case, mode):
    S = np.array(case["sites"], np.float64)
    box = np.array(case["box"], np.float64)
    rho = np.array(case["rho"], np.float64)
    kw = {}
    if mode == "neighbours":
        _, off, idx = _full(S, box)
        kw = dict(off=off, idx=idx)
    tr = oracle.trace(S, box, rho, np.array([case["origin"]], np.float64), np.array([case["dir"]], np.float64),
                      sphere=case["sphere"], **kw)
    assert oracle.STATUS[int(tr.status[0])] == case.get("status", "ok")
    cells, lens = tr.segments(0)
    assert [int(c) for c in cells] == [e[0] for e in case["segments"]]
    np.testing.assert_allclose(lens, [e[1] for e in case["segments"]], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr.tau[0], case["tau"], rtol=1e-12, atol=0)


def test_sphere_locate_example():
    L = _load("sphere_examples.json")["locate"]
    got = oracle.locate(np.array(L["sites"], np.float64), L["box"], np.array(L["points"], np.float64),
                        sphere=L["sphere"])
    assert [int(x) for x in got] == L["cells"]


def test_sphere_enter_example():
    E = _load("sphere_examples.json")["enter"]
    S = np.array(E["sites"], np.float64)
    O = np.array([E["origin"]], np.float64)
    D = np.array([E["dir"]], np.float64)
    P = oracle.enter_points(E["box"], O, D, sphere=E["sphere"])
    np.testing.assert_allclose(P[0], E["entry"], rtol=0, atol=1e-15)
    _, off, idx = _full(S, np.array(E["box"], np.float64))
    tr = oracle.trace(S, E["box"], np.array(E["rho"]), P, D, off=off, idx=idx, sphere=E["sphere"])
    cells, lens = tr.segments(0)
    assert [int(c) for c in cells] == [e[0] for e in E["segments"]]
    np.testing.assert_allclose(lens, [e[1] for e in E["segments"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(tr.tau[0], E["tau"], rtol=0, atol=4e-15)


@pytest.fixture(scope="module")
def ball300():
    g = gen.make_ball_grid(300, 41)
    c, off, idx = _full(g.sites, g.box)
    rays = gen.ball_rays(500, 42)
    tr = oracle.trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx, sphere=gen.UNIT_BALL)
    return g, off, idx, rays, tr


def test_sphere_paths_end_on_the_sphere(ball300):
    """Every path ends on the sphere: |r0 + L k - c| = R, with L the summed
    length and the end point's distance taken by numpy's norm; and L is the
    positive root of s^2 + 2 b s + q (numpy.roots)."""
    g, off, idx, rays, tr = ball300
    assert np.all(tr.status == 0)
    end = rays.origin + tr.length[:, None] * rays.dir
    np.testing.assert_allclose(np.linalg.norm(end, axis=1), 1.0, rtol=0, atol=1e-13)
    for i in range(0, 500, 25):
        o, k = rays.origin[i], rays.dir[i]
        roots = np.roots([k @ k, 2 * (k @ o), o @ o - 1.0])
        np.testing.assert_allclose(tr.length[i], roots.real.max(), rtol=1e-12)


def test_sphere_neighbour_exit_equals_all_sites_exit(ball300):
    g, off, idx, rays, tr = ball300
    tr2 = oracle.trace(g.sites, g.box, g.rho, rays.origin[:200], rays.dir[:200], sphere=gen.UNIT_BALL)
    for i in range(200):
        a, b = tr.segments(i), tr2.segments(i)
        assert np.array_equal(a[0], b[0])
        np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-15)


def test_sphere_uniform_density_closed_form(ball300):
    g, off, idx, rays, tr = ball300
    t = oracle.trace(g.sites, g.box, np.full(len(g.sites), 2.5), rays.origin, rays.dir, off=off, idx=idx,
                     kappa=0.8, sphere=gen.UNIT_BALL)
    np.testing.assert_allclose(t.tau, 0.8 * 2.5 * tr.length, rtol=1e-13)


def test_sphere_dense_sampling_reproduces_cell_sequence():
    """Brute force: points sampled along the path, inside the ball, owned by
    their nearest site, give the oracle's cell sequence; just past the end the
    path is outside the ball."""
    g = gen.make_ball_grid(120, 43)
    _, off, idx = _full(g.sites, g.box)
    rays = gen.ball_rays(60, 44)
    tr = oracle.trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx, sphere=gen.UNIT_BALL)
    checked = 0
    for i in range(60):
        cells, lens = tr.segments(i)
        if lens.min() < 2e-3:
            continue
        ts = np.arange(0.0, tr.length[i], 2.5e-4) + 1.25e-4
        ts = ts[ts < tr.length[i]]
        P = rays.origin[i] + ts[:, None] * rays.dir[i]
        assert np.all(np.linalg.norm(P, axis=1) < 1.0 + 1e-12)
        own = nearest_site(g.sites, P)
        runs = own[np.concatenate([[True], own[1:] != own[:-1]])]
        assert [int(x) for x in runs] == [int(x) for x in cells]
        beyond = rays.origin[i] + (tr.length[i] + 1e-9) * rays.dir[i]
        assert np.linalg.norm(beyond) > 1.0
        checked += 1
    assert checked > 40


def test_sphere_locate_matches_brute_force():
    g = gen.make_ball_grid(200, 45)
    rng = gen.rng_for(46)
    P = gen.uniform_points(3000, rng, g.box)
    got = oracle.locate(g.sites, g.box, P, sphere=gen.UNIT_BALL)
    inside = np.linalg.norm(P, axis=1) <= 1.0
    assert (~inside).sum() > 1000 and inside.sum() > 1000
    assert np.all(got[~inside] == -1)
    np.testing.assert_array_equal(got[inside], nearest_site(g.sites, P[inside]))


def test_sphere_enter_points():
    """Rays from outside the ball: the start lies epsilon past the sphere
    along k (so |E - c| is R to within epsilon), and a ray that misses keeps
    its origin (dense sampling never comes within the ball)."""
    rng = gen.rng_for(47)
    box = np.array([-2.0, -2, -2, 2, 2, 2])
    O = gen.uniform_points(2000, rng, box)
    D = gen.isotropic_dirs(2000, rng)
    E = oracle.enter_points(box, O, D, sphere=gen.UNIT_BALL)
    out = np.linalg.norm(O, axis=1) > 1.0
    moved = out & np.any(E != O, axis=1)
    assert moved.sum() > 100
    eps = oracle.default_eps(box)
    rad = np.linalg.norm(E[moved], axis=1)
    assert np.all(rad < 1.0) and np.all(rad > 1.0 - 1.01 * eps)
    back = E[moved] - 1.5 * eps * D[moved]
    assert np.all(np.linalg.norm(back, axis=1) > 1.0 - 1e-15)
    ts = np.linspace(0, 8, 8001)
    for i in np.nonzero(out & ~moved)[0][:100]:
        p = O[i] + ts[:, None] * D[i]
        assert not np.any(np.linalg.norm(p, axis=1) < 1.0 - 1e-3)


@pytest.mark.parametrize("case", _load("tie_examples.json")["cases"], ids=lambda c: c["name"])
def test_tie_examples(case):
    """R4 on a path where the tie-break shows: with every site a candidate, a
    ray through the edge where four cells meet goes straight into the
    diagonal cell, whose id is the lowest of the three tied planes."""
    S = np.array(case["sites"], np.float64)
    tr = oracle.trace(S, np.array(case["box"], np.float64), np.array(case["rho"]), np.array([case["origin"]]),
                      np.array([case["dir"]]), zero_run_max=case["zero_run_max"])
    assert int(tr.nfallback[0]) == case["nfallback"]
    cells, lens = tr.segments(0)
    assert [int(c) for c in cells] == [e[0] for e in case["segments"]]
    np.testing.assert_allclose(lens, [e[1] for e in case["segments"]], rtol=1e-12)


def test_degenerate_fuzz_cases_hold_the_invariants():
    """The oracle on the seeded degenerate grids of the GPU fuzz test
    (lattices, coplanar sites, near-duplicate pairs, sites on the walls,
    odd boxes; rays from sites, from walls and along the axes): every path
    ends on the box (summed length = slab length, numpy ray-box test), and
    away from near ties every segment's midpoint is nearest (numpy brute
    force) to the site of its cell, with the cells summing to the box's
    volume."""
    from tests import fuzz_cases
    for i in range(0, 120, 3):
        kind, g, rays = fuzz_cases.case(i)
        c = oracle.cells(g.sites, g.box)
        np.testing.assert_allclose(c.vol.sum(), np.prod(g.box[3:] - g.box[:3]), rtol=1e-10)
        off, idx = oracle.csr(c, len(g.sites))
        tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin, rays.dir, off=off, idx=idx)
        assert np.all(tr.status == 0), (i, kind)
        diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
        np.testing.assert_allclose(tr.length, slab_length(g.box, rays.origin, rays.dir), rtol=0, atol=1e-12 * diag,
                                   err_msg=f"case {i} ({kind})")
        mids, owners = [], []
        for r in np.nonzero(tr.near_tie == 0)[0]:
            cells, lens = tr.segments(r)
            t = np.concatenate([[0.0], np.cumsum(lens)])
            for a in range(cells.size):
                if lens[a] > 1e-9 * diag:
                    mids.append(rays.origin[r] + 0.5 * (t[a] + t[a + 1]) * rays.dir[r])
                    owners.append(cells[a])
        if mids:
            got = nearest_site(g.sites, np.array(mids))
            own = np.array(owners)
            # an equidistant midpoint (a segment along a face) may pick either site
            d_got = np.linalg.norm(np.array(mids) - g.sites[got], axis=1)
            d_own = np.linalg.norm(np.array(mids) - g.sites[own], axis=1)
            assert np.all((got == own) | (d_own - d_got <= 1e-12 * diag)), f"case {i} ({kind})"
