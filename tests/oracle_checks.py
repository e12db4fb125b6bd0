"""A fast selection of the oracle's pins, runnable on its own:
``python -m tests.oracle_checks`` exits 0 when every check holds and 1
otherwise, naming the checks that failed. The mutation test runs it against
copies of the oracle with one planted mistake each (ORACLE_LIB); the same
facts are checked, more widely, in test_oracle_pins.py.

Each check compares the oracle with something other than itself: hand-worked
paths (tests/golden), numpy brute force, closed forms and invariants.
"""
from __future__ import annotations

import json
import os
import sys
import traceback

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# ORACLE_PKG: a folder holding a copy of the oracle package with one planted
# mistake in its Python layer; it is imported in place of the real one
if os.environ.get("ORACLE_PKG"):
    sys.path.insert(0, os.environ["ORACLE_PKG"])

import gen  # noqa: E402
import oracle  # noqa: E402
from tests.helpers import dda_voxels, nearest_site, slab_length  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# every path of these small grids takes well under 100 decisions; a planted
# mistake that walks in circles stops here instead of at the default limit
MAX_STEPS = 10_000


def _trace(*args, **kw):
    kw.setdefault("max_steps", MAX_STEPS)
    return oracle.trace(*args, **kw)


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _full(S, box):
    c = oracle.cells(S, box)
    off, idx = oracle.csr(c, len(S))
    return c, off, idx


def _segments_match(tr, i, exp, rtol=1e-12, atol=0.0):
    cells, lens = tr.segments(i)
    assert [int(c) for c in cells] == [e[0] for e in exp], (list(cells), exp)
    np.testing.assert_allclose(lens, [e[1] for e in exp], rtol=rtol, atol=atol)


def check_worked_examples():
    for case in _load("worked_examples.json")["cases"]:
        S = np.array(case["sites"], np.float64)
        box = np.array(case["box"], np.float64)
        _, off, idx = _full(S, box)
        for kw in ({}, {"off": off, "idx": idx}):
            tr = _trace(S, box, np.array(case["rho"]), np.array([case["origin"]], np.float64),
                              np.array([case["dir"]], np.float64), kappa=case["kappa"], **kw)
            _segments_match(tr, 0, case["segments"])
            np.testing.assert_allclose(tr.tau[0], case["tau"], rtol=1e-12)


def check_fallback_examples():
    for case in _load("fallback_examples.json")["cases"]:
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
        tr = _trace(S, box, rho, np.array([case["origin"]], np.float64), np.array([case["dir"]], np.float64),
                          off=off, idx=idx, kappa=case["kappa"], zero_run_max=case["zero_run_max"])
        assert int(tr.nfallback[0]) == case["nfallback"]
        _segments_match(tr, 0, case["segments"], rtol=0, atol=case["len_atol"])


def check_sphere_examples():
    data = _load("sphere_examples.json")
    for case in data["cases"]:
        S = np.array(case["sites"], np.float64)
        box = np.array(case["box"], np.float64)
        _, off, idx = _full(S, box)
        tr = _trace(S, box, np.array(case["rho"]), np.array([case["origin"]], np.float64),
                          np.array([case["dir"]], np.float64), off=off, idx=idx, sphere=case["sphere"])
        assert oracle.STATUS[int(tr.status[0])] == case.get("status", "ok")
        _segments_match(tr, 0, case["segments"])
    L = data["locate"]
    got = oracle.locate(np.array(L["sites"], np.float64), L["box"], np.array(L["points"], np.float64),
                        sphere=L["sphere"])
    assert [int(x) for x in got] == L["cells"]


def check_sphere_paths_end_on_sphere():
    g = gen.make_ball_grid(150, 141)
    _, off, idx = _full(g.sites, g.box)
    rays = gen.ball_rays(150, 142)
    tr = _trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx, sphere=gen.UNIT_BALL)
    assert np.all(tr.status == 0)
    end = rays.origin + tr.length[:, None] * rays.dir
    np.testing.assert_allclose(np.linalg.norm(end, axis=1), 1.0, rtol=0, atol=1e-12)


def _grid150():
    g = gen.make_uniform_grid(150, 143)
    c, off, idx = _full(g.sites, g.box)
    return g, c, off, idx


def check_lengths_and_bisectors():
    """Summed lengths equal the slab length (Eq. 5); each segment's midpoint
    is nearest to its cell's site; each exit point is equidistant from the
    two sites it separates."""
    g, c, off, idx = _grid150()
    rays = gen.uniform_rays(120, 144)
    tr = _trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx)
    np.testing.assert_allclose(tr.length, slab_length(g.box, rays.origin, rays.dir), rtol=1e-12, atol=1e-15)
    mids, owners, d = [], [], []
    for i in range(120):
        cells, lens = tr.segments(i)
        t = np.concatenate([[0.0], np.cumsum(lens)])
        for a in range(cells.size):
            mids.append(rays.origin[i] + 0.5 * (t[a] + t[a + 1]) * rays.dir[i])
            owners.append(cells[a])
            if a + 1 < cells.size:
                q = rays.origin[i] + t[a + 1] * rays.dir[i]
                d.append(abs(np.linalg.norm(q - g.sites[cells[a]]) - np.linalg.norm(q - g.sites[cells[a + 1]])))
    np.testing.assert_array_equal(nearest_site(g.sites, np.array(mids)), np.array(owners))
    assert max(d) <= 1e-12 * 2 * np.sqrt(3)


def check_tau_closed_form():
    g, c, off, idx = _grid150()
    rays = gen.uniform_rays(80, 145)
    tr = _trace(g.sites, g.box, np.full(len(g.sites), 2.5), rays.origin, rays.dir, off=off, idx=idx,
                      kappa=0.8)
    np.testing.assert_allclose(tr.tau, 0.8 * 2.5 * slab_length(g.box, rays.origin, rays.dir), rtol=1e-12)
    tr2 = _trace(g.sites, g.box, g.rho, rays.origin, rays.dir, off=off, idx=idx)
    want = np.array([float(np.sum(g.rho[tr2.segments(i)[0]] * tr2.segments(i)[1])) for i in range(80)])
    np.testing.assert_allclose(tr2.tau, want, rtol=1e-12)


def check_locate_brute_force():
    g, _, _, _ = _grid150()
    rng = gen.rng_for(146)
    P = np.concatenate([gen.uniform_points(800, rng, g.box), [[1.5, 0, 0], [0, -1.0000001, 0]]])
    got = oracle.locate(g.sites, g.box, P)
    np.testing.assert_array_equal(got[:800], nearest_site(g.sites, P[:800]))
    assert np.all(got[800:] == -1)


def check_cells_brute_and_volume():
    g, c, _, _ = _grid150()
    b = oracle.cells(g.sites, g.box, brute=True)
    for x, y in zip(c.nbr, b.nbr):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_allclose(c.vol.sum(), np.prod(g.box[3:] - g.box[:3]), rtol=1e-10)
    L = gen.cubic_lattice(4, gen.CUBE_BOX)
    lc = oracle.cells(L, gen.CUBE_BOX)
    np.testing.assert_allclose(lc.vol, (2.0 / 4) ** 3, rtol=1e-10)
    assert all(a.size == 6 for a in lc.nbr)


def check_interior_cells_are_delaunay():
    """Away from the walls a cell's neighbours are exactly its site's
    Delaunay edges (scipy's Delaunay triangulation of the sites)."""
    try:
        from scipy.spatial import Delaunay
    except ImportError:
        return
    g = gen.make_uniform_grid(600, 148)
    c = oracle.cells(g.sites, g.box)
    ptr, nb = Delaunay(g.sites).vertex_neighbor_vertices
    inner = 0
    for i in range(len(g.sites)):
        bb = c.bbox[i]
        if np.any(bb[:3] < g.box[:3] + 0.05) or np.any(bb[3:] > g.box[3:] - 0.05):
            continue
        inner += 1
        np.testing.assert_array_equal(np.sort(nb[ptr[i]:ptr[i + 1]]), c.nbr[i])
    assert inner >= 50


def check_lattice_is_dda():
    """A cubic lattice (spacing 0.5, exact in float32): the cells crossed are
    the voxels of a 3D DDA walk, with the same lengths."""
    n = 4
    S = gen.cubic_lattice(n, gen.CUBE_BOX)
    _, off, idx = _full(S, gen.CUBE_BOX)
    rays = gen.uniform_rays(60, 147)
    tr = _trace(S, gen.CUBE_BOX, np.ones(len(S)), rays.origin, rays.dir, off=off, idx=idx)
    for i in range(60):
        ref = dda_voxels(gen.CUBE_BOX, n, rays.origin[i], rays.dir[i])
        cells, got = tr.segments(i)
        assert [int(x) for x in cells] == [v[0] * n * n + v[1] * n + v[2] for v, _ in ref]
        np.testing.assert_allclose(got, [l for _, l in ref], rtol=1e-11, atol=1e-13)


def check_tie_examples():
    for case in _load("tie_examples.json")["cases"]:
        S = np.array(case["sites"], np.float64)
        tr = _trace(S, np.array(case["box"], np.float64), np.array(case["rho"]), np.array([case["origin"]], np.float64),
                    np.array([case["dir"]], np.float64), zero_run_max=case["zero_run_max"])
        assert int(tr.nfallback[0]) == case["nfallback"]
        _segments_match(tr, 0, case["segments"])


def check_exp_loss():
    """The loss sum (e^-tau - t)^2 and its derivative, against a hand value
    and central differences in tau."""
    tau = np.array([0.0, 0.5, 2.0])
    t = np.array([0.5, 0.25, 0.0])
    loss, dL = oracle.exp_loss(tau, t)
    e = np.exp(-tau)
    np.testing.assert_allclose(loss, (1 - 0.5) ** 2 + (e[1] - 0.25) ** 2 + e[2] ** 2, rtol=1e-15)
    h = 1e-6
    for i in range(3):
        tp = tau.copy(); tp[i] += h
        tm = tau.copy(); tm[i] -= h
        fd = (oracle.exp_loss(tp, t)[0] - oracle.exp_loss(tm, t)[0]) / (2 * h)
        assert abs(fd - dL[i]) <= 1e-8, (i, fd, dL[i])


def check_tau_grad_fd():
    """dL/drho of the loss against central differences of the loss in rho
    (through the traced tau), with kappa != 1; cells no ray crosses get 0."""
    g, c, off, idx = _grid150()
    rays = gen.uniform_rays(60, 149)
    rho = g.rho.astype(np.float64)
    tr = _trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3)
    target = np.exp(-0.9 * tr.tau)
    _, dL = oracle.exp_loss(tr.tau, target)
    grad = oracle.tau_grad(tr, len(g.sites), dL, kappa=1.3)
    hit = np.unique(np.concatenate([tr.segments(i)[0] for i in range(60)]))
    for cidx in gen.rng_for(150).choice(hit, 4, replace=False):
        hh = 1e-4 * rho[cidx]
        rp = rho.copy(); rp[cidx] += hh
        rm = rho.copy(); rm[cidx] -= hh
        tp = _trace(g.sites, g.box, rp, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3).tau
        tm = _trace(g.sites, g.box, rm, rays.origin, rays.dir, off=off, idx=idx, kappa=1.3).tau
        fd = (oracle.exp_loss(tp, target)[0] - oracle.exp_loss(tm, target)[0]) / (2 * hh)
        assert abs(fd - grad[cidx]) <= 1e-6 * max(abs(fd), 1e-8), (cidx, fd, grad[cidx])
    assert np.all(grad[np.setdiff1d(np.arange(len(g.sites)), hit)] == 0.0)


def check_enter_points():
    """Entry points on the box by hand (a face, a corner, a ray pointing
    away, a start inside) and on the unit ball (epsilon past the sphere,
    along the ray; a ray that misses keeps its origin)."""
    box = gen.CUBE_BOX
    O = np.array([[-2.0, 0.1, 0.2], [0.5, 3.0, -0.25], [2.0, 2.0, 2.0], [-3.0, 0.0, 0.0], [0.1, 0.2, 0.3]])
    D = np.array([[1.0, 0, 0], [0.0, -1, 0], [-1.0, -1, -1], [-1.0, 0, 0], [0.6, 0.8, 0.0]])
    D = D / np.linalg.norm(D, axis=1)[:, None]
    E = oracle.enter_points(box, O, D)
    np.testing.assert_allclose(E[:3], [[-1.0, 0.1, 0.2], [0.5, 1.0, -0.25], [1.0, 1.0, 1.0]], rtol=1e-15)
    np.testing.assert_array_equal(E[3:], O[3:])
    big = np.array([-2.0, -2, -2, 2, 2, 2])
    eps = 1e-12 * np.sqrt(48.0)     # 1e-12 |Dmax - Dmin| (R6) for this box
    O = np.array([[-1.5, 0.0, 0.0], [1.5, 1.5, 0.0], [0.0, 0.0, 1.5], [0.2, 0.1, 0.0]])
    D = np.array([[1.0, 0, 0], [1.0, 0, 0], [0.0, 0.6, -0.8], [1.0, 0, 0]])
    E = oracle.enter_points(big, O, D, sphere=gen.UNIT_BALL)
    np.testing.assert_allclose(E[0], [-1.0 + eps, 0, 0], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(E[1], O[1])       # points away from the ball
    # |(0, 0.6 s, 1.5 - 0.8 s)|^2 = 1 is s^2 - 2.4 s + 1.25 = 0; the ray enters at the smaller root
    s = (2.4 - np.sqrt(2.4 ** 2 - 4 * 1.25)) / 2
    np.testing.assert_allclose(E[2], O[2] + (s + eps) * D[2], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(E[3], O[3])       # already inside


def check_interaction():
    """Interaction sampling: the hand-worked two-cell path, the uniform
    medium's closed form s = tau_int / (kappa rho), and conservation (what
    the cells remove is what the packages lose)."""
    S = np.array([[1.0, 1, 1], [3.0, 1, 1]])
    box = np.array([0.0, 0, 0, 4, 4, 4])
    rho = np.array([2.0, 3.0])
    _, off, idx = _full(S, box)
    tr = _trace(S, box, rho, np.array([[0.5, 1, 1]] * 2), np.array([[1.0, 0, 0]] * 2), off=off, idx=idx)
    cell, s, ab, amb = oracle.interact(tr, rho, [4.0, 10.0], weight=[1.0, 2.0])
    assert list(cell) == [1, -1]
    np.testing.assert_allclose(s, [1.5 + 1.0 / 3.0, 3.5], rtol=1e-14)
    np.testing.assert_allclose(ab, [(1 - np.exp(-3)) * 3.0, (np.exp(-3) - np.exp(-4)) + 2 * (np.exp(-3) - np.exp(-9))],
                               rtol=1e-13)
    g, c, off, idx = _grid150()
    rays = gen.uniform_rays(100, 151)
    rho = np.full(len(g.sites), 0.8)
    tr = _trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, kappa=1.5)
    rng = gen.rng_for(152)
    tau_int = -np.log(rng.random(100))
    w = rng.uniform(0.5, 2.0, 100)
    cell, s, ab, amb = oracle.interact(tr, rho, tau_int, weight=w, kappa=1.5)
    L = slab_length(g.box, rays.origin, rays.dir)
    inside = tau_int < 1.2 * L
    np.testing.assert_allclose(s[inside], tau_int[inside] / 1.2, rtol=1e-12)
    np.testing.assert_allclose(s[~inside], L[~inside], rtol=1e-12)
    np.testing.assert_allclose(ab.sum(), (w * (1 - np.exp(-np.minimum(tau_int, 1.2 * L)))).sum(), rtol=1e-12)


CHECKS = [check_worked_examples, check_tie_examples, check_fallback_examples, check_sphere_examples, check_sphere_paths_end_on_sphere,
          check_lengths_and_bisectors, check_tau_closed_form, check_locate_brute_force, check_cells_brute_and_volume,
          check_interior_cells_are_delaunay, check_lattice_is_dda, check_exp_loss, check_tau_grad_fd, check_enter_points,
          check_interaction]


def run() -> list:
    failed = []
    for fn in CHECKS:
        try:
            fn()
        except Exception:  # a planted mistake may also crash a check
            failed.append(fn.__name__)
            if os.environ.get("ORACLE_CHECKS_VERBOSE"):
                traceback.print_exc()
    return failed


if __name__ == "__main__":
    bad = run()
    print("failed:", " ".join(bad) if bad else "none")
    sys.exit(1 if bad else 0)
