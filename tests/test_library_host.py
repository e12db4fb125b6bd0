"""The C-ABI library on the host: it loads, exports every declared entry
point, and its grid builder (an implementation independent of the oracle)
agrees with the oracle's cells. No GPU is used: grids are built with
host_only, which runs the whole construction and copies nothing to a device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import gen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vgrid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(vgrid_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol(libvgrid):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(libvgrid, n), n
    from paper_1310_1854_gb300 import _lib
    assert {s[0] for s in _lib.SIGNATURES} == set(names)


def _grid(sites, box, **kw):
    from paper_1310_1854_gb300 import VoronoiGrid
    return VoronoiGrid(sites, box, host_only=True, **kw)


def _delaunay_neighbours(sites):
    spatial = pytest.importorskip("scipy.spatial")
    tri = spatial.Delaunay(sites)
    ptr, nb = tri.vertex_neighbor_vertices
    return lambda m: set(nb[ptr[m]:ptr[m + 1]].tolist())


def _assert_cells_match(vg, sites, box, ids, area_rel=1e-9):
    off, idx = vg.neighbors()
    vol, bb = vg.cells()
    c = oracle.cells(sites, box, ids=ids)
    delaunay = _delaunay_neighbours(sites)
    for k, m in enumerate(ids):
        ours = set(idx[off[m]:off[m + 1]].tolist())
        faces = c.nbr[k]
        big = set(faces[c.area[k] > area_rel * c.area[k].sum()].tolist())
        # every face of non-negligible area is in our list; ours may add
        # planes that only touch the cell (they never change an exit):
        # those are still Delaunay neighbours (their bisector meets the
        # cell), never walls, and there are at most two of them
        assert big <= ours, (m, big - ours)
        extra = ours - set(faces.tolist())
        assert all(j >= 0 for j in extra), (m, extra)
        assert extra <= delaunay(m), (m, extra - delaunay(m))
        assert len(extra) <= 2, (m, extra)
    np.testing.assert_allclose(vol[ids], c.vol, rtol=1e-10)
    np.testing.assert_allclose(bb[ids], c.bbox, atol=1e-12 * np.linalg.norm(box[3:] - box[:3]))


def test_builder_matches_oracle_uniform_1000(libvgrid):
    g, _ = gen.config1(10)
    vg = _grid(g.sites, g.box)
    off, idx = vg.neighbors()
    c = oracle.cells(g.sites, g.box)
    for m in range(len(g.sites)):
        assert np.array_equal(np.sort(idx[off[m]:off[m + 1]]), c.nbr[m]), m
    vol, _ = vg.cells()
    np.testing.assert_allclose(vol, c.vol, rtol=1e-11)
    np.testing.assert_allclose(vol.sum(), 8.0, rtol=1e-12)


@pytest.mark.parametrize("kind", ["disk", "clumpy"])
def test_builder_matches_oracle_sampled(libvgrid, kind):
    if kind == "disk":
        g = gen.make_disk_grid(20_000, 91)
    else:
        g = gen.make_clumpy_grid(20_000, 92, n_clumps=40)
    vg = _grid(g.sites, g.box)
    ids = gen.rng_for(93).choice(len(g.sites), 300, replace=False)
    _assert_cells_match(vg, g.sites, g.box, ids)
    vol, _ = vg.cells()
    box = g.box
    np.testing.assert_allclose(vol.sum(), np.prod(box[3:] - box[:3]), rtol=1e-11)


def test_builder_symmetric_and_reorder_invariant(libvgrid):
    g = gen.make_uniform_grid(3000, 94)
    a = _grid(g.sites, g.box)
    b = _grid(g.sites, g.box, reorder=False)
    oa, ia = a.neighbors()
    ob, ib = b.neighbors()
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(ia, ib)
    pairs = {(m, int(j)) for m in range(3000) for j in ia[oa[m]:oa[m + 1]] if j >= 0}
    assert all((j, m) in pairs for m, j in pairs)


def test_builder_lattices(libvgrid):
    S = gen.cubic_lattice(8)
    vg = _grid(S, gen.CUBE_BOX)
    off, idx = vg.neighbors()
    deg = np.diff(off)
    interior = np.all(np.abs(S) < 0.8, axis=1)
    assert np.all(deg[interior] >= 6)
    c = oracle.cells(S, gen.CUBE_BOX)
    for m in np.nonzero(interior)[0][:50]:
        assert set(c.nbr[m].tolist()) <= set(idx[off[m]:off[m + 1]].tolist())
    vol, _ = vg.cells()
    np.testing.assert_allclose(vol, 0.25 ** 3, rtol=1e-12)
    S = gen.bcc_lattice(8)
    vg = _grid(S, gen.CUBE_BOX)
    off, idx = vg.neighbors()
    interior = np.all(np.abs(S) < 1 - 1.2 * 0.25, axis=1)
    assert np.all(np.diff(off)[interior] >= 14)
    vol, _ = vg.cells()
    np.testing.assert_allclose(vol[interior], 0.25 ** 3 / 2, rtol=1e-12)


def test_create_rejects_bad_input(libvgrid):
    from paper_1310_1854_gb300 import VGridError, _lib
    box = gen.CUBE_BOX
    with pytest.raises(VGridError) as e:
        _grid(np.array([[0.0, 0, 0], [0.0, 0, 0]]), box)
    assert e.value.code == _lib.ERR_DUP_SITE
    with pytest.raises(VGridError) as e:
        _grid(np.array([[0.0, 0, 0], [1.5, 0, 0]]), box)
    assert e.value.code == _lib.ERR_OUTSIDE
    with pytest.raises(VGridError) as e:
        _grid(np.array([[0.1, 0, 0]]), box)  # 0.1 is not a float32 value
    assert e.value.code == _lib.ERR_ARG
    _grid(np.array([[0.1, 0, 0]]), box, round_sites=True)
    with pytest.raises(VGridError) as e:
        _grid(np.zeros((0, 3)), box)
    assert e.value.code == _lib.ERR_ARG
    with pytest.raises(VGridError) as e:
        _grid(np.array([[0.0, 0, 0]]), np.array([1, -1, -1, -1, 1, 1.0]))
    assert e.value.code == _lib.ERR_ARG
    with pytest.raises(VGridError) as e:
        _grid(np.array([[np.nan, 0, 0]]), box)
    assert e.value.code == _lib.ERR_ARG


def test_single_site_grid_is_the_box(libvgrid):
    vg = _grid(np.array([[0.25, -0.5, 0.125]]), gen.CUBE_BOX)
    off, idx = vg.neighbors()
    assert sorted(idx.tolist()) == [-6, -5, -4, -3, -2, -1]
    vol, bb = vg.cells()
    assert vol[0] == pytest.approx(8.0, rel=1e-14)


def test_host_only_grid_refuses_device_calls(libvgrid):
    from paper_1310_1854_gb300 import _lib
    vg = _grid(gen.cubic_lattice(2), gen.CUBE_BOX)
    lib = _lib.load()
    dummy = ctypes.c_void_p(16)
    rc = lib.vgrid_trace(vg._h, dummy, dummy, 1, _lib.FP32_RECHECK, _lib.TAU, dummy, None, None, None, 0, None,
                         None, None)
    assert rc == _lib.ERR_ARG
    assert b"host_only" in lib.vgrid_last_error()
    assert lib.vgrid_locate(vg._h, dummy, 1, 0, dummy, None) == _lib.ERR_ARG
    assert lib.vgrid_trace_grad(vg._h, dummy, dummy, 1, dummy, dummy, None) == _lib.ERR_ARG
    assert lib.vgrid_segments_grad(vg._h, dummy, dummy, dummy, 1, dummy, 1.0, dummy, None) == _lib.ERR_ARG
    assert lib.vgrid_enable_timing(vg._h, 1) == _lib.ERR_ARG


def test_segments_grad_argument_checks(libvgrid):
    """VoronoiGrid.segments_grad wants the float32 segment lists of a trace
    and one dL/dtau per ray (checked before any device work)."""
    import torch
    from paper_1310_1854_gb300 import TraceResult
    vg = _grid(gen.cubic_lattice(2), gen.CUBE_BOX)
    off = torch.tensor([0, 2, 3], dtype=torch.int64)
    cells = torch.tensor([0, 1, 1], dtype=torch.int32)
    tau = torch.zeros(2)
    with pytest.raises(TypeError):
        vg.segments_grad(TraceResult(tau), torch.ones(2))
    with pytest.raises(TypeError):
        vg.segments_grad(TraceResult(tau, off, cells, torch.ones(3, dtype=torch.float64)), torch.ones(2))
    with pytest.raises(ValueError):
        vg.segments_grad(TraceResult(tau, off, cells, torch.ones(3)), torch.ones(3))


def test_launch_shape_validation(libvgrid):
    """vgrid_set_launch checks every field (host-only grid: no GPU needed)."""
    from paper_1310_1854_gb300 import _lib
    vg = _grid(gen.cubic_lattice(2), gen.CUBE_BOX)
    assert vg.get_launch() == {"lanes_per_ray": 1, "block": 128, "blocks_per_sm": 0, "fp64_lanes_per_ray": 1,
                               "order": 0}
    vg.set_launch(lanes_per_ray=2, block=256, blocks_per_sm=3, fp64_lanes_per_ray=8, order=1)
    assert vg.get_launch() == {"lanes_per_ray": 2, "block": 256, "blocks_per_sm": 3, "fp64_lanes_per_ray": 8,
                               "order": 1}
    for bad in ({"order": 2}, {"order": -2}, {"lanes_per_ray": 3}, {"block": 48}, {"block": 512},
                {"blocks_per_sm": -1}, {"fp64_lanes_per_ray": 5}):
        with pytest.raises(_lib.VGridError):
            vg.set_launch(**bad)
    assert vg.get_launch()["order"] == 1  # a refused shape leaves the last one
    lib = _lib.load()
    assert lib.vgrid_set_launch(vg._h, None) == 0
    assert vg.get_launch()["order"] == 0


def test_probe_rejects_bad_arguments(libvgrid):
    """vgrid_probe_l2 checks its arguments before touching a device."""
    from paper_1310_1854_gb300 import _lib
    lib = _lib.load()
    out = ctypes.c_double(-1.0)
    assert lib.vgrid_probe_l2(1 << 24, 2, ctypes.byref(out), None) == _lib.ERR_ARG
    assert lib.vgrid_probe_l2(1000, 0, ctypes.byref(out), None) == _lib.ERR_ARG
    assert lib.vgrid_probe_l2((1 << 32) + 1, 1, ctypes.byref(out), None) == _lib.ERR_ARG
    assert lib.vgrid_probe_l2(1 << 24, 0, None, None) == _lib.ERR_ARG
    assert out.value == -1.0


def test_zero_run_limit_option(libvgrid):
    """opts.zero_run_max: 4 by default, 0 allowed, negative refused."""
    from paper_1310_1854_gb300 import _lib
    lib = _lib.load()
    o = _lib.Opts()
    lib.vgrid_default_opts(ctypes.byref(o))
    assert o.zero_run_max == 4
    _grid(gen.cubic_lattice(2), gen.CUBE_BOX, zero_run_max=0)
    with pytest.raises(_lib.VGridError) as e:
        _grid(gen.cubic_lattice(2), gen.CUBE_BOX, zero_run_max=-1)
    assert e.value.code == _lib.ERR_ARG


def test_sphere_domain_options(libvgrid):
    """opts.domain / opts.sphere: box by default; a ball must lie inside the
    box with a positive radius and hold every site; its grid keeps the box's
    neighbour lists (the cells are the box's clipping)."""
    from paper_1310_1854_gb300 import _lib
    lib = _lib.load()
    o = _lib.Opts()
    lib.vgrid_default_opts(ctypes.byref(o))
    assert o.domain == _lib.DOMAIN_BOX and list(o.sphere) == [0.0] * 4
    g = gen.make_ball_grid(400, 61)
    a = _grid(g.sites, g.box, sphere=gen.UNIT_BALL)
    b = _grid(g.sites, g.box)
    for x, y in zip(a.neighbors(), b.neighbors()):
        np.testing.assert_array_equal(x, y)
    for bad in ((0.0, 0, 0, 1.5), (0.5, 0, 0, 0.6), (0.0, 0, 0, 0.0), (0.0, 0, 0, -1.0), (0.0, np.nan, 0, 0.5)):
        with pytest.raises(_lib.VGridError) as e:
            _grid(g.sites, g.box, sphere=bad)
        assert e.value.code == _lib.ERR_ARG
    # a site outside the ball (but inside the box)
    S = np.concatenate([g.sites, [[0.875, 0.875, 0.0]]])  # float32 values, 1.53125 > 1
    with pytest.raises(_lib.VGridError) as e:
        _grid(S, g.box, sphere=gen.UNIT_BALL)
    assert e.value.code == _lib.ERR_OUTSIDE
    o.domain = 2
    M = len(g.sites)
    h = ctypes.c_void_p()
    S = np.ascontiguousarray(g.sites, np.float64)
    B = np.ascontiguousarray(g.box, np.float64)
    assert lib.vgrid_create(S.ctypes.data_as(ctypes.c_void_p), M, B.ctypes.data_as(ctypes.c_void_p),
                            ctypes.byref(o), ctypes.byref(h)) == _lib.ERR_ARG


def test_quality_samples_cover_the_domain():
    """grid_quality's points: uniform in the box, or in the ball of a
    spherical domain (every point inside it; the share within half the
    radius is 1/8, the ratio of the volumes)."""
    from paper_1310_1854_gb300.quality import sample_points
    P = sample_points(gen.CUBE_BOX, 20_000, 3)
    assert np.all((P >= -1) & (P <= 1))
    B = sample_points(gen.CUBE_BOX, 40_000, 4, gen.UNIT_BALL)
    r = np.linalg.norm(B, axis=1)
    assert B.shape == (40_000, 3) and np.all(r <= 1.0)
    assert abs(np.mean(r < 0.5) - 0.125) < 0.01
