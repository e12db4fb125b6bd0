"""GPU traversal against the CPU oracle, through the C-ABI.

Acceptance (float64 form): cell sequences identical on rays whose exit
decisions are not near ties (decision margin > 1e-9, start not equidistant),
segment lengths within 1e-12 relative (1e-12 * diagonal absolute for
lengths below 1e-6 * diagonal), tau within 1e-12 relative.
Acceptance (float32 form with float64 recheck): the same cell sequences, and
tau within 1e-5 relative of the oracle's float64 tau.
Small cases compare every ray; full-size workloads compare a seeded sample
of rays traced by the oracle with every site as a candidate.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

TAU32_REL = 1e-5
LEN64_REL = 1e-12
# float32 adjoint: per cell within this fraction of the sum of |contributions|
# (float32 products plus atomic summation in arbitrary order)
GRAD32_REL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(g, **kw):
    from paper_1310_1854_gb300 import VoronoiGrid
    vg = VoronoiGrid(g.sites, g.box, **kw)
    vg.set_density(dev(g.rho), float(g.kappa))
    return vg


def oracle_full(g, rays, **kw):
    c = oracle.cells(g.sites, g.box)
    off, idx = oracle.csr(c, len(g.sites))
    kw.setdefault("kappa", float(g.kappa))
    return oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin, rays.dir, off=off, idx=idx, **kw)


def check_segments(ref, sel, seg_off, seg_cell, seg_len, diag, len_rel):
    """Cell sequences equal and lengths within tolerance on rays `sel`."""
    so = seg_off.cpu().numpy()
    cells = seg_cell.cpu().numpy()
    lens = seg_len.cpu().numpy().astype(np.float64)
    for i in sel:
        rc, rl = ref.segments(i)
        gc = cells[so[i]:so[i + 1]]
        gl = lens[so[i]:so[i + 1]]
        assert np.array_equal(gc, rc), f"ray {i}: cells differ"
        if len_rel is not None:
            tol = np.where(rl < 1e-6 * diag, 1e-12 * diag, len_rel * rl)
            assert np.all(np.abs(gl - rl) <= tol), f"ray {i}: lengths differ by {np.max(np.abs(gl - rl) / rl)}"


def run_case(g, rays, ref, lanes=(1, 4), **mk):
    """Every ray: float64 and float32 segment lists and tau against the
    oracle, for each lanes-per-ray shape; tau identical across shapes."""
    vg = make(g, **mk)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    O, D = dev(rays.origin), dev(rays.dir)
    ok = np.nonzero(ref.near_tie == 0)[0]
    assert ok.size >= 0.9 * len(rays.origin)
    rt = ref.tau[ok]
    taus = []
    for lpr in lanes:
        vg.set_launch(lanes_per_ray=lpr, fp64_lanes_per_ray=lpr)
        r64 = vg.trace(O, D, precision="fp64", segments=True, status=True)
        r32 = vg.trace(O, D, precision="fp32", segments=True, status=True)
        t32 = vg.trace(O, D, precision="fp32", stats=True)
        check_segments(ref, ok, r64.seg_off, r64.seg_cell, r64.seg_len, diag, LEN64_REL)
        check_segments(ref, ok, r32.seg_off, r32.seg_cell, r32.seg_len, diag, None)
        np.testing.assert_allclose(r64.tau.cpu().numpy()[ok], rt, rtol=1e-12, atol=1e-300)
        t = t32.tau.cpu().numpy().astype(np.float64)[ok]
        err = np.abs(t - rt) / np.maximum(rt, 1e-300)
        assert np.all(err[rt > 0] <= TAU32_REL), f"max rel tau error {err.max()}"
        # tau mode writes the tau of segment mode (same decisions)
        np.testing.assert_array_equal(t32.tau.cpu().numpy(), r32.tau.cpu().numpy())
        assert np.all(r64.status.cpu().numpy() == 0) and np.all(r32.status.cpu().numpy() == 0)
        taus.append(t32.tau.cpu().numpy())
    for t in taus[1:]:
        np.testing.assert_array_equal(t, taus[0])
    return vg


def test_config1_full_parity():
    g, rays = gen.config1()
    ref = oracle_full(g, rays)
    run_case(g, rays, ref, lanes=(1, 2, 4, 8))


def test_small_disk_parity():
    g = gen.make_disk_grid(20_000, 101)
    rays = gen.disk_rays(3000, 102)
    ref = oracle_full(g, rays)
    run_case(g, rays, ref)


def test_small_clumpy_parity():
    g = gen.make_clumpy_grid(20_000, 103, n_clumps=40)
    rays = gen.uniform_rays(3000, 104)
    ref = oracle_full(g, rays)
    run_case(g, rays, ref)


def test_cubic_lattice_parity():
    """Degenerate geometry (eight cells per vertex): the float32 form must
    fall back to float64 near the ties and still match the oracle."""
    S = gen.cubic_lattice(8)
    g = gen.Grid(S, gen.CUBE_BOX.copy(), gen.rng_for(5).uniform(0.5, 1.5, len(S)).astype(np.float32))
    rays = gen.uniform_rays(2000, 106)
    ref = oracle_full(g, rays)
    run_case(g, rays, ref)


def test_near_perpendicular_planes_parity():
    """Rays along the axes of a cubic lattice, exactly and tilted by 1e-9 to
    1e-3: many planes are perpendicular to the ray or nearly so (n.k = 0 or
    tiny), where the float64 form's float32 pre-test must never drop a plane
    that faces ahead. Both forms against the oracle."""
    S = gen.cubic_lattice(8)
    rng = gen.rng_for(109)
    g = gen.Grid(S, gen.CUBE_BOX.copy(), rng.uniform(0.5, 1.5, len(S)).astype(np.float32))
    n = 1500
    o = rng.uniform(-0.95, 0.95, (n, 3))
    axis = rng.integers(0, 3, n)
    d = np.zeros((n, 3))
    d[np.arange(n), axis] = rng.choice([-1.0, 1.0], n)
    tilt = 10.0 ** rng.uniform(-9, -3, (n, 3)) * rng.choice([-1.0, 0.0, 1.0], (n, 3))
    tilt[: n // 4] = 0.0  # exactly along an axis
    d = d + tilt
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = gen.Rays(o, d)
    ref = oracle_full(g, rays)
    vg = make(g)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    ok = np.nonzero(ref.near_tie == 0)[0]
    assert ok.size >= n // 3
    O, D = dev(o), dev(d)
    for lpr in (1, 4):
        vg.set_launch(fp64_lanes_per_ray=lpr)
        r64 = vg.trace(O, D, precision="fp64", segments=True)
        check_segments(ref, ok, r64.seg_off, r64.seg_cell, r64.seg_len, diag, LEN64_REL)
        np.testing.assert_allclose(r64.tau.cpu().numpy()[ok], ref.tau[ok], rtol=1e-12, atol=1e-300)
    r32 = vg.trace(O, D, precision="fp32", segments=True)
    check_segments(ref, ok, r32.seg_off, r32.seg_cell, r32.seg_len, diag, None)
    vg.set_launch()


def lattice_plane_starts(n, m, seed):
    """m rays of a cubic lattice of n^3 cells in [-1,1]^3 whose start lies on
    one, two or three lattice planes (a face, an edge or a vertex of several
    cells), the other coordinates at least 1e-4 from any plane, isotropic
    directions. The plane coordinates and the sites are dyadic, so a plane
    through the start has a numerator of exactly zero in every form."""
    rng = gen.rng_for(seed)
    h = 2.0 / n
    P = rng.uniform(-1 + h, 1 - h, (m, 3))
    frac = (P + 1) / h - np.round((P + 1) / h)
    P = np.where(np.abs(frac) * h < 1e-4, P + 2e-4, P)
    planes = np.arange(1, n) * h - 1.0
    for i in range(m):
        for a in rng.choice(3, 1 + i % 3, replace=False):
            P[i, a] = rng.choice(planes)
    return gen.Rays(P, gen.isotropic_dirs(m, rng))


def test_epsilon_fallback_matches_oracle():
    """The epsilon nudge of Sect. 2.2 (zero_run_max = 0: every zero-length step
    nudges the point by epsilon and locates it again) on rays that start on
    lattice faces, edges and vertices, against the oracle with the same limit.
    float64 form: the same nudges, cells and lengths as the oracle (same
    epsilon, 1e-12 |D|). float32 form: the same cells and the same number of
    nudges; it nudges by 1e-6 |D| (reading R6), so its path misses up to that
    much more per nudge than the oracle's, and tau may differ by
    kappa rho_max 1e-6 |D| per nudge beyond the usual 1e-5 relative."""
    n = 8
    S = gen.cubic_lattice(n)
    rng = gen.rng_for(410)
    g = gen.Grid(S, gen.CUBE_BOX.copy(), rng.uniform(0.5, 1.5, len(S)).astype(np.float32))
    rays = lattice_plane_starts(n, 3000, 411)
    c = oracle.cells(g.sites, g.box)
    off, idx = oracle.csr(c, len(g.sites))
    rho = g.rho.astype(np.float64)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    O, D = dev(rays.origin), dev(rays.dir)
    from paper_1310_1854_gb300 import Batch, VoronoiGrid
    for zmax in (0, 4):
        ref = oracle.trace(g.sites, g.box, rho, rays.origin, rays.dir, off=off, idx=idx, zero_run_max=zmax)
        assert np.all(ref.status == 0)
        nfb = int(ref.nfallback.sum())
        if zmax == 0:
            # a start on a plane gives a zero-length step unless the ray heads
            # into the cell that holds the start (lowest index of the tie)
            assert nfb >= 1500
        else:
            assert nfb == 0
        vg = VoronoiGrid(g.sites, g.box, zero_run_max=zmax)
        vg.set_density(dev(g.rho), 1.0)
        for lpr in (1, 4):
            vg.set_launch(lanes_per_ray=lpr, fp64_lanes_per_ray=lpr)
            r64 = vg.trace(O, D, precision="fp64", segments=True, stats=True)
            r32 = vg.trace(O, D, precision="fp32", segments=True, stats=True)
            assert r64.stats["fallbacks"] == nfb and r32.stats["fallbacks"] == nfb, (zmax, r64.stats, r32.stats)
            check_segments(ref, range(rays.origin.shape[0]), r64.seg_off, r64.seg_cell, r64.seg_len,
                           diag, LEN64_REL)
            check_segments(ref, range(rays.origin.shape[0]), r32.seg_off, r32.seg_cell, r32.seg_len, diag, None)
            np.testing.assert_allclose(r64.tau.cpu().numpy(), ref.tau, rtol=1e-12, atol=0)
            t32 = r32.tau.cpu().numpy().astype(np.float64)
            bound = 1e-5 * ref.tau + ref.nfallback * float(g.kappa) * rho.max() * 1e-6 * diag
            assert np.all(np.abs(t32 - ref.tau) <= bound), np.max(np.abs(t32 - ref.tau) - bound)
            # tau mode and the batch launch take the same decisions
            t = vg.trace(O, D, precision="fp32", stats=True)
            np.testing.assert_array_equal(t.tau.cpu().numpy(), r32.tau.cpu().numpy())
            assert t.stats["fallbacks"] == nfb
        vg.set_launch()
        b = Batch([(vg, O, D)])
        st = b.run(stats=True)
        np.testing.assert_array_equal(b.tau[0].cpu().numpy(), vg.trace(O, D, precision="fp32").tau.cpu().numpy())
        assert st["fallbacks"] == nfb


def test_zero_run_limit_does_not_touch_generic_rays():
    """On a random grid with random rays no step has length zero, so the
    zero-run limit changes nothing: tau is the same bits with limit 0 and 4,
    and no ray is nudged."""
    from paper_1310_1854_gb300 import VoronoiGrid
    g, rays = gen.config1(5000)
    O, D = dev(rays.origin), dev(rays.dir)
    out = []
    for zmax in (0, 4):
        vg = VoronoiGrid(g.sites, g.box, zero_run_max=zmax)
        vg.set_density(dev(g.rho), 1.0)
        for prec in ("fp32", "fp64"):
            r = vg.trace(O, D, precision=prec, stats=True)
            assert r.stats["fallbacks"] == 0 and r.stats["zero_steps"] == 0
            out.append(r.tau.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[2])
    np.testing.assert_array_equal(out[1], out[3])


def test_tiny_coordinates_parity():
    """Sites with tiny nonzero coordinates next to ordinary ones: their float
    differences and sums round in float64, so the float64 form takes those
    records from the float coordinates instead of its table of exact
    differences; it must still match the oracle bit for bit."""
    rng = gen.rng_for(107)
    S = rng.uniform(-1.0, 1.0, (1500, 3))
    pick = rng.choice(len(S), 200, replace=False)
    axis = rng.integers(0, 3, 200)
    S[pick, axis] = rng.choice([-1.0, 1.0], 200) * 10.0 ** rng.uniform(-30, -9, 200)
    S = S.astype(np.float32).astype(np.float64)
    S = np.unique(S, axis=0)
    g = gen.Grid(S, gen.CUBE_BOX.copy(), rng.uniform(0.5, 1.5, len(S)).astype(np.float32))
    rays = gen.uniform_rays(3000, 108)
    ref = oracle_full(g, rays)
    run_case(g, rays, ref)


@pytest.mark.parametrize("box", [(1000.0, 1000.0, 1000.0, 1002.0, 1002.0, 1002.0),
                                 (-1e-3, -1e-3, -1e-3, 1e-3, 1e-3, 1e-3),
                                 (0.0, 0.0, 0.0, 4.0, 4.0, 0.02)],
                         ids=["far_from_origin", "millimetre", "thin_slab"])
def test_offset_scaled_and_thin_boxes_parity(box):
    """The error bounds of the float32 form carry the coordinates' size (the
    float pairs of r0 and k, C(r)'s 4uX term): a box far from the origin
    (coordinates 1000 times the cell size), a tiny box (cells of 1e-4) and a
    thin slab (cells wider than the slab is thick) give the oracle's cells
    and lengths in both forms."""
    B = np.array(box, np.float64)
    rng = gen.rng_for(109)
    S = gen.uniform_points(1500, rng, B).astype(np.float32).astype(np.float64)
    S = np.unique(S[np.all((S >= B[:3]) & (S <= B[3:]), axis=1)], axis=0)
    g = gen.Grid(S, B, rng.uniform(0.5, 1.5, len(S)).astype(np.float32))
    rays = gen.uniform_rays(3000, 110, B)
    ref = oracle_full(g, rays)
    run_case(g, rays, ref)


def test_locate_parity():
    g = gen.make_disk_grid(20_000, 107)
    vg = make(g)
    rng = gen.rng_for(108)
    P = np.concatenate([gen.disk_points(4000, rng), gen.uniform_points(1000, rng, g.box),
                        np.array([[5.0, 0, 0], [0, 0, -0.6], [4.0, 4.0, 0.5], [-4.0, -4.0, -0.5]])])
    ref = oracle.locate(g.sites, g.box, P)
    for prec in ("fp32", "fp64"):
        out = vg.locate(dev(P), precision=prec).cpu().numpy()
        np.testing.assert_array_equal(out, ref)


def test_locate_on_block_faces():
    """C(r) for points on and next to the faces of the block grid: the
    block index comes from float32 pairs, and the block lists are padded to
    cover its rounding, so the nearest site must still be found."""
    g = gen.make_disk_grid(20_000, 111)
    vg = make(g)
    info = vg.info()
    lo, hi = np.asarray(g.box[:3]), np.asarray(g.box[3:])
    dim = np.asarray(info["block_dim"])
    rng = gen.rng_for(112)
    n = 3000
    P = lo + rng.random((n, 3)) * (hi - lo)
    axis = rng.integers(0, 3, n)
    k = rng.integers(1, dim[axis])
    face = lo[axis] + k * (hi[axis] - lo[axis]) / dim[axis]
    ext = (hi - lo)[axis]
    delta = rng.choice(np.array([0.0, 1e-7, -1e-7, 3e-8, -3e-8, 1e-9, -1e-9]), n) * ext
    P[np.arange(n), axis] = np.clip(face + delta, lo[axis], hi[axis])
    P = np.concatenate([P, np.nextafter(P, np.inf), np.nextafter(P, -np.inf)])
    P = np.clip(P, lo, hi)
    ref = oracle.locate(g.sites, g.box, P)
    for prec in ("fp32", "fp64"):
        out = vg.locate(dev(P), precision=prec).cpu().numpy()
        np.testing.assert_array_equal(out, ref)


def oracle_slab(box, O, D):
    from tests.helpers import slab_length
    return slab_length(box, O, D)


def test_edge_cases():
    from paper_1310_1854_gb300 import VGridError, _lib
    g, rays = gen.config1(64)
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    # empty input
    e = vg.trace(O[:0], D[:0], precision="fp32", segments=True)
    assert e.seg_off.shape[0] == 1 and int(e.seg_off[0]) == 0
    # a ray starting outside, one on the boundary going out, one with a bad direction
    o = np.array([[2.0, 0, 0], [1.0, 0.1, 0.2], [0.0, 0.0, 0.0], [0.1, 0.1, 0.1]])
    d = np.array([[1.0, 0, 0], [1.0, 0, 0], [0.5, 0.5, 0.0], [0.0, 0.0, 1.0]])
    for prec in ("fp32", "fp64"):
        r = vg.trace(dev(o), dev(d), precision=prec, status=True)
        st = r.status.cpu().numpy()
        assert st[0] == _lib.RAY_OUTSIDE and st[2] == _lib.RAY_BAD_DIR and st[3] == _lib.RAY_OK
        assert float(r.tau[0]) == 0.0 and float(r.tau[1]) == 0.0
        with pytest.raises(VGridError) as ex:
            vg.trace(dev(o), dev(d), precision=prec, stats=True)
        assert ex.value.code == _lib.ERR_ARG
    # capacity: too small a buffer reports the sizes
    with pytest.raises(VGridError) as ex:
        vg.trace(O, D, precision="fp32", segments=True, seg_capacity=3)
    assert ex.value.code == _lib.ERR_CAPACITY
    # step limit
    from paper_1310_1854_gb300 import VoronoiGrid
    v1 = VoronoiGrid(g.sites, g.box, max_steps=2)
    with pytest.raises(VGridError) as ex:
        v1.trace(O, D, precision="fp32", stats=True)
    assert ex.value.code == _lib.ERR_STEP_LIMIT
    r = v1.trace(O, D, precision="fp32", status=True)
    assert np.any(r.status.cpu().numpy() == _lib.RAY_STEP_LIMIT)


def test_gradient_matches_oracle():
    g, rays = gen.config1(3000)
    ref = oracle_full(g, rays)
    target = np.exp(-0.9 * ref.tau)
    _, dL = oracle.exp_loss(ref.tau, target)
    want = oracle.tau_grad(ref, len(g.sites), dL, kappa=float(g.kappa))
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    wabs = oracle.tau_grad(ref, len(g.sites), np.abs(dL), kappa=float(g.kappa))
    got = vg.trace_grad(O, D, dev(dL.astype(np.float32))).cpu().numpy().astype(np.float64)
    ok = np.all(ref.near_tie == 0)
    assert ok or ref.near_tie.sum() < 5
    assert np.all(np.abs(got - want) <= GRAD32_REL * wabs + 1e-30)
    assert np.all(got[wabs == 0] == 0)
    # the same adjoint from the segment lists of a float32 trace (no second
    # traversal): same terms, other summation order
    seg = vg.trace(O, D, precision="fp32", segments=True)
    got2 = vg.segments_grad(seg, dev(dL.astype(np.float32))).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got2 - want) <= GRAD32_REL * wabs + 1e-30)
    assert np.all(got2[wabs == 0] == 0)
    assert np.all(np.abs(got2 - got) <= 2 * GRAD32_REL * wabs + 1e-30)
    acc = vg.segments_grad(seg, dev(dL.astype(np.float32)), out=torch.from_numpy(got2.astype(np.float32)).cuda())
    np.testing.assert_allclose(acc.cpu().numpy(), 2 * got2, rtol=1e-5, atol=1e-30 + 1e-6 * np.abs(got2).max())
    # autograd wrapper gives the same gradient
    from paper_1310_1854_gb300 import optical_depth
    rho = dev(g.rho).requires_grad_(True)
    tau = optical_depth(vg, rho, O, D, float(g.kappa))
    t = dev(target.astype(np.float32))
    loss = ((torch.exp(-tau) - t) ** 2).sum()
    loss.backward()
    gg = rho.grad.cpu().numpy().astype(np.float64)
    # torch evaluates the loss in float32 from float32 tau; dL/dtau carries
    # that rounding (about 1e-7 relative to exp(-tau))
    assert np.all(np.abs(gg - want) <= 1e-3 * wabs + 1e-30)
    # backward by a second traversal instead of the kept segment lists
    rho2 = dev(g.rho).requires_grad_(True)
    tau2 = optical_depth(vg, rho2, O, D, float(g.kappa), keep_segments=False)
    np.testing.assert_array_equal(tau2.detach().cpu().numpy(), tau.detach().cpu().numpy())
    ((torch.exp(-tau2) - t) ** 2).sum().backward()
    gg2 = rho2.grad.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gg2 - want) <= 1e-3 * wabs + 1e-30)
    # with exact lengths: the oracle's tau to 1e-6 and the same gradient, the
    # lists kept or traced again
    for keep in (True, False):
        rho3 = dev(g.rho).requires_grad_(True)
        tau3 = optical_depth(vg, rho3, O, D, float(g.kappa), keep_segments=keep, precision="fp32_exact")
        ok = ref.near_tie == 0
        t3 = tau3.detach().cpu().numpy().astype(np.float64)
        assert np.all(np.abs(t3[ok] - ref.tau[ok]) <= 1e-6 * ref.tau[ok])
        ((torch.exp(-tau3) - t) ** 2).sum().backward()
        gg3 = rho3.grad.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gg3 - want) <= 1e-3 * wabs + 1e-30)
    with pytest.raises(ValueError):
        optical_depth(vg, rho3, O, D, 1.0, precision="fp64")


def test_gradient_uses_the_forward_kappa():
    """Two forward calls with different kappa on one grid before backward:
    the gradient of the first call uses its own kappa (the grid holds the
    second one by then), on both backward routes (kept segment lists,
    second traversal) and when the grid's kappa has been set to 0."""
    from paper_1310_1854_gb300 import optical_depth
    g, rays = gen.config1(2000)
    ref = oracle_full(g, rays, kappa=2.0)
    target = np.exp(-0.9 * ref.tau)
    _, dL = oracle.exp_loss(ref.tau, target)
    want = oracle.tau_grad(ref, len(g.sites), dL, kappa=2.0)
    wabs = oracle.tau_grad(ref, len(g.sites), np.abs(dL), kappa=2.0)
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    t = dev(target.astype(np.float32))
    for keep in (True, False):
        for later_kappa in (1.0, 0.0):
            rho = dev(g.rho).requires_grad_(True)
            tau = optical_depth(vg, rho, O, D, 2.0, keep_segments=keep)
            other = dev(g.rho).requires_grad_(True)
            optical_depth(vg, other, O, D, later_kappa, keep_segments=keep)
            assert vg.kappa == later_kappa
            ok = ref.near_tie == 0
            tt = tau.detach().cpu().numpy().astype(np.float64)
            assert np.all(np.abs(tt[ok] - ref.tau[ok]) <= TAU32_REL * ref.tau[ok])
            ((torch.exp(-tau) - t) ** 2).sum().backward()
            gg = rho.grad.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(gg - want) <= 1e-3 * wabs + 1e-30), (keep, later_kappa)


def test_batched_matches_single():
    from paper_1310_1854_gb300 import Batch
    sets = gen.config4(G=12, scale=0.02)
    grids, single = [], []
    for g, r in sets:
        vg = make(g)
        grids.append((vg, dev(r.origin), dev(r.dir)))
        single.append(vg.trace(grids[-1][1], grids[-1][2], precision="fp32").tau.cpu().numpy())
    b = Batch(grids)
    st = b.run(stats=True)
    for k in range(len(sets)):
        np.testing.assert_array_equal(b.tau[k].cpu().numpy(), single[k])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(graph=True, stream=s)
        b.run(graph=True, stream=s)
    s.synchronize()
    for k in range(len(sets)):
        np.testing.assert_array_equal(b.tau[k].cpu().numpy(), single[k])
    assert st["rays"] == sum(len(r.origin) for _, r in sets)
    # one grid against the oracle
    g, r = sets[3]
    ref = oracle_full(g, r)
    ok = ref.near_tie == 0
    t = b.tau[3].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(t[ok] - ref.tau[ok]) <= TAU32_REL * ref.tau[ok])


def test_autotuned_batch_matches_single(tmp_path):
    """The batch autotuner times its candidate shapes (lanes per ray, block,
    ray order) on a seeded sample of every set's rays, applies the fastest to
    the batch and caches it; a tuned batch, every shape of the space, and the
    graph replay after a change of shape give the single-grid tau to the bit."""
    from paper_1310_1854_gb300 import Batch, tune
    sets = gen.config4(G=10, scale=0.02)
    grids, single = [], []
    for g, r in sets:
        vg = make(g)
        grids.append((vg, dev(r.origin), dev(r.dir)))
        single.append(vg.trace(grids[-1][1], grids[-1][2], precision="fp32").tau.cpu().numpy())
    b = Batch(grids)
    space = ((1, 128, 0, -1), (2, 64, 0, 1), (1, 256, 0, 1), (4, 128, 0, -1))
    path = str(tmp_path / "tune.json")
    r = tune.autotune_batch(b, sample_rays=b.rays // 3, space=space, path=path)
    assert not r["cached"] and r["sample_rays"] < b.rays and len(r["table"]) == len(space)
    L = b.get_launch()
    assert (L["lanes_per_ray"], L["block"], L["blocks_per_sm"], L["order"]) == \
        (r["lanes_per_ray"], r["block"], r["blocks_per_sm"], r["order"])
    s = torch.cuda.Stream()
    for shape in (None,) + space:
        if shape is not None:
            b.set_launch(*shape)
        b.run()
        for k in range(len(sets)):
            np.testing.assert_array_equal(b.tau[k].cpu().numpy(), single[k])
        with torch.cuda.stream(s):
            for k in range(len(sets)):
                b.tau[k].fill_(-1.0)
            b.run(graph=True, stream=s)
        s.synchronize()
        for k in range(len(sets)):
            np.testing.assert_array_equal(b.tau[k].cpu().numpy(), single[k])
    b.set_launch()
    r2 = tune.autotune_batch(b, sample_rays=b.rays // 3, space=space, path=path)
    assert r2["cached"] and b.get_launch()["order"] == r["order"]


# --------------------------------------------------------------------------
# full-size workloads: every ray traced in the benchmark's launch shape, a
# seeded sample of at least 10^4 rays against the oracle (tests/accuracy.py)
# --------------------------------------------------------------------------

def _assert_accuracy(stats, bad):
    assert stats["oracle_status_ok"] if "oracle_status_ok" in stats else True
    assert stats["near_tie_fraction"] < 0.05, stats
    assert stats["sample"] >= 10_000
    for k, v in bad.items():
        assert not v, (k, len(v), v[:10])
    assert stats["fp32_tau_rel_err"]["max"] <= TAU32_REL, stats
    assert stats["fp32_sequence_mismatches"] == 0
    assert stats["gpu_fallbacks"] == 0 and stats["oracle_fallbacks"] == 0


@pytest.mark.slow
def test_full_size_config2_accuracy():
    """10^5-site disk, 10^6 rays: 10^4 sampled rays against the oracle, both
    forms (sequences, float64 lengths, tau); over all rays the float64
    lengths add up to the in-domain distance (Eq. 5)."""
    from tests import accuracy
    g, rays = gen.config2()
    sel = np.sort(gen.rng_for(501).choice(len(rays.origin), 10_000, replace=False))
    stats, bad, ctx = accuracy._single("disk1e5", g, rays, sel)
    _assert_accuracy(stats, bad)
    assert stats["fp64_sequence_mismatches"] == 0 and stats["fp64_tau_rel_err"]["max"] <= 1e-12
    vg, O, D, t32, ref, _ = ctx
    r64 = vg.trace(O, D, precision="fp64", segments=True)
    so64 = r64.seg_off.cpu().numpy()
    l64 = r64.seg_len.cpu().numpy()
    L = oracle_slab(g.box, rays.origin, rays.dir)
    per_ray = np.bincount(np.repeat(np.arange(len(L)), np.diff(so64)), weights=l64, minlength=len(L))
    np.testing.assert_allclose(per_ray, L, rtol=1e-12, atol=1e-12)
    assert t32.stats["rays"] == len(L)


@pytest.mark.slow
def test_full_size_config3_accuracy():
    """10^6 clumpy sites, 10^7 rays: sequences from the full ordered launch
    (segment lists of all 10^7 rays), tau of both forms from their full
    launches, against the oracle on 10^4 sampled rays."""
    from tests import accuracy
    stats, bad = accuracy.clumpy1e6()
    _assert_accuracy(stats, bad)
    assert stats["fp64_tau_rel_err"]["max"] <= 1e-12
    assert stats["launch"]["order"] == 0 and stats["rays"] == 10_000_000


@pytest.mark.slow
def test_full_size_config4_accuracy():
    """64 uneven grids in one autotuned batch launch and its graph replay:
    every set's tau equals its single-grid launch, and 10^4 rays spread over
    the grids agree with the oracle."""
    from tests import accuracy
    stats, bad = accuracy.batched64()
    _assert_accuracy(stats, bad)
    assert stats["gpu_rays"] == stats["rays"]


@pytest.mark.slow
def test_full_size_config5_accuracy_and_gradient():
    """10^6-site disk, 512^2 detector + 10^6 interior rays. (1) 10^4 sampled
    rays (2,000 from the detector) against the oracle. (2) The adjoint:
    dL/drho of the sample's rays against the oracle's float64 gradient, cell
    by cell. (3) Central finite differences of the loss with the GPU's float64
    forward on 100 seeded cells hit by rays (h = 1e-4 rho_c; tau is linear in
    rho, so the difference is exact up to rounding and the exp's third
    derivative) against the float32 gradient of all rays, by the adjoint
    traversal and through optical_depth's backward."""
    from paper_1310_1854_gb300 import optical_depth
    from tests import accuracy
    stats, bad, ctx, g, rays, rho_t = accuracy.grad1e6(keep=True)
    _assert_accuracy(stats, bad)
    assert stats["detector_rays_compared"] >= 1000
    vg, O, D, t32, ref, sel = ctx
    M = len(g.sites)
    vg.set_density(dev(rho_t), 1.0)
    target = torch.exp(-vg.trace(O, D, precision="fp32").tau)
    vg.set_density(dev(g.rho), 1.0)
    tau = t32.tau
    e = torch.exp(-tau)
    dL = (-2.0 * (e - target) * e).float()
    # (2) the sample's adjoint against the oracle's
    keep = ref.near_tie == 0
    ks = sel[keep]
    dls = dL.cpu().numpy().astype(np.float64)[ks]
    sub = oracle.Trace(*(getattr(ref, f)[keep] for f in ("nseg", "seg_cell", "seg_len", "tau", "length",
                                                         "min_margin", "near_tie", "nfallback", "status")))
    want = oracle.tau_grad(sub, M, dls)
    wabs = oracle.tau_grad(sub, M, np.abs(dls))
    got = vg.trace_grad(dev(rays.origin[ks]), dev(rays.dir[ks]), dev(dls.astype(np.float32))).cpu().numpy()
    got = got.astype(np.float64)
    assert np.count_nonzero(want) > 50_000
    # float32 exit points carry an absolute error of a few ulp of the path
    # length per segment, which the per-cell bound includes
    lens = np.repeat(sub.length, sub.nseg)
    cells = np.concatenate([sub.segments(k)[0] for k in range(len(ks))])
    slack = np.bincount(cells, weights=np.repeat(np.abs(dls), sub.nseg) * 2e-6 * lens, minlength=M)
    assert np.all(np.abs(got - want) <= GRAD32_REL * wabs + slack + 1e-30)
    assert np.all(got[wabs == 0] == 0)
    # (3) finite differences with the float64 forward
    full = vg.trace_grad(O, D, dL).cpu().numpy().astype(np.float64)
    fabs = vg.trace_grad(O, D, dL.abs()).cpu().numpy().astype(np.float64)
    rho_a = dev(g.rho).requires_grad_(True)
    tau_a = optical_depth(vg, rho_a, O, D, 1.0)
    ((torch.exp(-tau_a) - target) ** 2).sum().backward()
    auto = rho_a.grad.cpu().numpy().astype(np.float64)
    s64 = vg.trace(O, D, precision="fp64", segments=True)
    ray_of = torch.repeat_interleave(torch.arange(O.shape[0], device="cuda"), s64.seg_off.diff())
    hit = torch.bincount(s64.seg_cell.long(), minlength=M).cpu().numpy() > 0
    # the float32 lengths' absolute error, bounded per segment by 2e-6 of the
    # ray's path length, times |dL/dtau| of its ray, summed per cell
    Lr = torch.zeros(O.shape[0], dtype=torch.float64, device="cuda").index_add_(0, ray_of, s64.seg_len)
    wseg = (dL.abs().double() * 2e-6 * Lr)[ray_of]
    slack = torch.zeros(M, dtype=torch.float64, device="cuda").index_add_(0, s64.seg_cell.long(), wseg).cpu().numpy()
    cells = np.sort(gen.rng_for(505).choice(np.nonzero(hit)[0], 100, replace=False))
    rho64 = g.rho.astype(np.float64)
    tgt = target.double()
    for c in cells:
        rs = torch.unique(ray_of[s64.seg_cell == int(c)])
        Oc, Dc = O[rs].contiguous(), D[rs].contiguous()
        h = 1e-4 * rho64[c]
        losses = []
        for sgn in (1.0, -1.0):
            rp = g.rho.copy()
            rp[c] = np.float32(rho64[c] + sgn * h)
            hh = float(rp[c]) - rho64[c]  # the step the float32 density actually takes
            vg.set_density(dev(rp), 1.0)
            tp = vg.trace(Oc, Dc, precision="fp64").tau
            losses.append((float(((torch.exp(-tp) - tgt[rs]) ** 2).sum()), hh))
        vg.set_density(dev(g.rho), 1.0)
        fd = (losses[0][0] - losses[1][0]) / (losses[0][1] - losses[1][1])
        tol = 1e-4 * fabs[c] + slack[c] + 1e-6 * abs(fd) + 1e-12
        assert abs(full[c] - fd) <= tol, (c, full[c], fd, fabs[c])
        assert abs(auto[c] - fd) <= tol, (c, auto[c], fd, fabs[c])


def test_interaction_matches_oracle():
    g, rays = gen.config1(4000)
    ref = oracle_full(g, rays)
    rng = gen.rng_for(300)
    tau_int = (-np.log(rng.random(len(rays.origin)))).astype(np.float32)
    w = rng.uniform(0.5, 2.0, len(rays.origin)).astype(np.float32)
    cell_o, s_o, ab_o, amb = oracle.interact(ref, g.rho.astype(np.float64), tau_int.astype(np.float64),
                                             weight=w.astype(np.float64))
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    cell, s, ab = vg.interact(O, D, dev(tau_int), dev(w), absorbed=True)
    cell = cell.cpu().numpy()
    s = s.cpu().numpy().astype(np.float64)
    ab = ab.cpu().numpy().astype(np.float64)
    ok = (ref.near_tie == 0) & ~amb
    assert ok.sum() > 0.9 * len(ok)
    np.testing.assert_array_equal(cell[ok], cell_o[ok])
    # float32 tau and lengths: the interaction distance moves by tau error / (kappa rho)
    L = ref.length
    assert np.all(np.abs(s[ok] - s_o[ok]) <= 2e-5 * np.maximum(L[ok], 1e-3) + 1e-6)
    # per cell, within float32 rounding of the sum of what each ray removed
    np.testing.assert_allclose(ab.sum(), ab_o.sum(), rtol=1e-5)
    assert np.all(np.abs(ab - ab_o) <= 2e-4 * np.abs(ab_o) + 1e-6 * ab_o.max())


def test_ray_order_does_not_change_results():
    """The longest-first ray order (vgrid_launch.order) changes which lane
    takes which ray, not what a ray computes: tau (both forms), segment
    lists and interaction cells/distances are bit-identical to the caller's
    order, and the gradient agrees up to the order of its float32 atomic
    sums."""
    g, rays = gen.config2(n_rays=300_000)
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    rng = gen.rng_for(310)
    tau_int = dev((-np.log(rng.random(len(rays.origin)))).astype(np.float32))
    dL = dev(rng.uniform(0.5, 2.0, len(rays.origin)).astype(np.float32))
    out = {}
    for order in (-1, 1):
        vg.set_launch(order=order)
        t = vg.trace(O, D, precision="fp32", stats=True)
        sg = vg.trace(O, D, precision="fp32", segments=True)
        c, s_, _ = vg.interact(O, D, tau_int)
        gr = torch.zeros(len(g.sites), dtype=torch.float32, device="cuda")
        vg.trace_grad(O, D, dL, gr)
        t64 = vg.trace(O, D, precision="fp64")
        out[order] = (t.tau.cpu().numpy(), t.stats, sg.seg_off.cpu().numpy(), sg.seg_cell.cpu().numpy(),
                      sg.seg_len.cpu().numpy(), c.cpu().numpy(), s_.cpu().numpy(), gr.cpu().numpy(),
                      t64.tau.cpu().numpy())
    a, b = out[-1], out[1]
    for k in (0, 2, 3, 4, 5, 6, 8):
        np.testing.assert_array_equal(a[k], b[k])
    for key in ("rays", "crossings", "decisions", "rechecks"):
        assert a[1][key] == b[1][key]
    np.testing.assert_allclose(b[7], a[7], rtol=1e-4, atol=1e-6 * float(np.abs(a[7]).max()))
    vg.set_launch()
    assert vg.get_launch()["order"] == 0


def test_host_pipelined_trace_matches_device_trace():
    """vgrid_trace_host (rays and results in host memory, copies overlapped
    with the traversal) gives the tau, status and counters of vgrid_trace on
    the same rays: one chunk, several with a ragged last one, pageable
    buffers, pinned rays with a pageable result, the float64 form and the
    float32 form with exact lengths, and calls queued back to back."""
    g, rays = gen.config2(n_rays=300_000)
    vg = make(g)
    N = len(rays.origin)
    O, D = dev(rays.origin), dev(rays.dir)
    Oh = torch.from_numpy(rays.origin).pin_memory()
    Dh = torch.from_numpy(rays.dir).pin_memory()
    for prec in ("fp32", "fp64", "fp32_exact"):
        ref = vg.trace(O, D, precision=prec, status=True, stats=True)
        rt, rs = ref.tau.cpu().numpy(), ref.status.cpu().numpy()
        for chunk in (0, 70_001, N):
            r = vg.trace_host(Oh, Dh, precision=prec, status=True, stats=True, chunk=chunk)
            assert not r.tau.is_cuda
            np.testing.assert_array_equal(r.tau.numpy(), rt)
            np.testing.assert_array_equal(r.status.numpy(), rs)
            for key in ("rays", "crossings", "decisions", "outside"):
                assert r.stats[key] == ref.stats[key], (prec, chunk, key)
    r = vg.trace_host(torch.from_numpy(rays.origin), torch.from_numpy(rays.dir), chunk=123_457)
    t32 = vg.trace(O, D).tau.cpu().numpy()
    np.testing.assert_array_equal(r.tau.numpy(), t32)
    # pinned rays, pageable tau: results through the slots and a copy out
    # (pinned tau is written by the traversal directly)
    r = vg.trace_host(Oh, Dh, out_tau=torch.empty(N, dtype=torch.float32), chunk=100_000)
    np.testing.assert_array_equal(r.tau.numpy(), t32)
    assert vg.trace_host(Oh[:0], Dh[:0]).tau.numel() == 0
    # queued calls back to back (the next call's copies overlap this traversal)
    half = N // 2
    outs = [torch.empty(n, dtype=torch.float32).pin_memory() for n in (N, half, N)]
    vg.trace_host(Oh, Dh, out_tau=outs[0], wait=False)
    vg.trace_host(Oh[:half], Dh[:half], out_tau=outs[1], wait=False)
    vg.trace_host(Oh, Dh, out_tau=outs[2], wait=False)
    torch.cuda.current_stream().synchronize()
    np.testing.assert_array_equal(outs[0].numpy(), t32)
    np.testing.assert_array_equal(outs[1].numpy(), t32[:half])
    np.testing.assert_array_equal(outs[2].numpy(), t32)


def test_ray_order_edge_cases():
    """The ray order forced on for inputs it was not built for: one ray, a
    handful, rays outside the box, non-unit directions; statuses, tau and
    segments equal the caller's order (both forms), and the host-resident
    call agrees."""
    from paper_1310_1854_gb300 import _lib
    g, rays = gen.config1(2000)
    vg = make(g)
    rng = gen.rng_for(320)
    o = np.concatenate([rays.origin, rng.uniform(1.5, 3.0, (50, 3)), rays.origin[:30]])
    d = np.concatenate([rays.dir, rays.dir[:50], rays.dir[:30] * 1.5])  # last 30: not unit
    for n in (1, 7, 120, len(o)):
        O, D = dev(o[:n]), dev(d[:n])
        res = {}
        for order in (-1, 1):
            vg.set_launch(order=order)
            t32 = vg.trace(O, D, precision="fp32", status=True)
            t64 = vg.trace(O, D, precision="fp64", status=True)
            m = min(n, 2050)  # segment mode reports non-unit directions as an error
            sg = vg.trace(O[:m], D[:m], precision="fp32", segments=True)
            res[order] = [t32.tau.cpu().numpy(), t32.status.cpu().numpy(), t64.tau.cpu().numpy(),
                          t64.status.cpu().numpy(), sg.seg_off.cpu().numpy(), sg.seg_cell.cpu().numpy(),
                          sg.seg_len.cpu().numpy()]
            if order == 1:
                h = vg.trace_host(torch.from_numpy(o[:n]), torch.from_numpy(d[:n]), status=True)
                np.testing.assert_array_equal(h.tau.numpy(), res[1][0])
                np.testing.assert_array_equal(h.status.numpy(), res[1][1])
        for a, b in zip(res[-1], res[1]):
            np.testing.assert_array_equal(a, b)
        st = res[1][1]
        if n == len(o):
            assert np.all(st[2000:2050] == _lib.RAY_OUTSIDE) and np.all(st[2050:] == _lib.RAY_BAD_DIR)
            assert np.all(res[1][0][2000:] == 0.0)
    vg.set_launch()


def test_segment_lists_single_pass():
    """Segment lists come from one traversal (chunks of 8 per ray, handed out
    in warp pages, then copied into ray order): the lists are the same for
    every launch shape and with or without the ray order, whatever the
    capacity given (exact, generous); a capacity one short, or zero, reports
    the same offsets; per ray the lengths add up to the path length to the
    wall and kappa rho l adds up to tau."""
    from paper_1310_1854_gb300 import VGridError, _lib
    g, rays = gen.config2(M=20_000, n_rays=30_000)
    vg = make(g)
    rng = gen.rng_for(321)
    # a few rays outside the box among them: no segments
    o = rays.origin.copy()
    out = rng.choice(len(o), 100, replace=False)
    o[out] = g.box[3:] + rng.uniform(0.1, 1.0, (100, 3))
    O, D = dev(o), dev(rays.dir)
    N = len(o)
    lo, hi = g.box[:3], g.box[3:]
    with np.errstate(divide="ignore", invalid="ignore"):
        tw = np.where(rays.dir > 0, (hi - o) / rays.dir, np.where(rays.dir < 0, (lo - o) / rays.dir, np.inf))
    tmax = tw.min(axis=1)
    rho = g.rho.astype(np.float64)
    inside = np.ones(N, dtype=bool)
    inside[out] = False
    for prec in ("fp32", "fp64"):
        ref = None
        for lpr in (1, 2, 4, 8):
            for order in (-1, 1):
                vg.set_launch(lanes_per_ray=lpr, fp64_lanes_per_ray=lpr, order=order)
                r = vg.trace(O, D, precision=prec, segments=True, status=True, stats=True)
                cur = [r.seg_off.cpu().numpy(), r.seg_cell.cpu().numpy(), r.seg_len.cpu().numpy(),
                       r.tau.cpu().numpy()]
                if ref is None:
                    ref = cur
                    total = int(cur[0][-1])
                    assert total == r.stats["crossings"] and total > 10 * N
                    st = r.status.cpu().numpy()
                    assert np.all(st[out] == _lib.RAY_OUTSIDE) and np.all(st[inside] == _lib.RAY_OK)
                elif prec == "fp64" and lpr != 1:
                    # the float64 winner does not depend on the lane split
                    for a, b in zip(ref, cur):
                        np.testing.assert_array_equal(a, b)
                else:
                    for a, b in zip(ref[:3], cur[:3]):
                        np.testing.assert_array_equal(a, b)
        so, cells, lens, tau = ref
        cnt = np.diff(so)
        assert np.all(cnt[out] == 0) and np.all(cnt[inside] > 0)
        ray_of = np.repeat(np.arange(N), cnt)
        ltot = np.bincount(ray_of, weights=lens.astype(np.float64), minlength=N)
        ttot = np.bincount(ray_of, weights=float(g.kappa) * rho[cells] * lens.astype(np.float64), minlength=N)
        if prec == "fp64":
            # the point moves by rounded steps r += s k; the last step, to
            # the wall, makes up for their drift only to about n ulp / |k_axis|
            np.testing.assert_allclose(ltot[inside], tmax[inside], rtol=1e-9)
            np.testing.assert_allclose(ttot[inside], tau[inside], rtol=1e-11)
        else:
            np.testing.assert_allclose(ltot[inside], tmax[inside], rtol=1e-4)
            np.testing.assert_allclose(ttot[inside], tau[inside], rtol=1e-5)
        vg.set_launch()
        for cap in (total, 4 * total + 17):
            r = vg.trace(O, D, precision=prec, segments=True, seg_capacity=cap)
            np.testing.assert_array_equal(r.seg_off.cpu().numpy(), so)
            np.testing.assert_array_equal(r.seg_cell.cpu().numpy(), cells)
            np.testing.assert_array_equal(r.seg_len.cpu().numpy(), lens)
        for cap in (total - 1, 0):
            with pytest.raises(VGridError) as ex:
                vg.trace(O, D, precision=prec, segments=True, seg_capacity=cap)
            assert ex.value.code == _lib.ERR_CAPACITY
        # the offsets of a refused call, read through the C ABI
        import ctypes
        lib = _lib.load()
        off = torch.empty(N + 1, dtype=torch.int64, device="cuda")
        tdt = torch.float64 if prec == "fp64" else torch.float32
        tb = torch.empty(N, dtype=tdt, device="cuda")
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        rc = lib.vgrid_trace(vg._h, p(O), p(D), N, _lib.FP64 if prec == "fp64" else _lib.FP32_RECHECK,
                             _lib.SEGMENTS, p(tb), p(off), None, None, 0, None, None, None)
        assert rc == _lib.ERR_CAPACITY
        torch.cuda.synchronize()
        np.testing.assert_array_equal(off.cpu().numpy(), so)


def test_rays_entering_from_outside():
    g, _ = gen.config1(10)
    rng = gen.rng_for(310)
    O = gen.uniform_points(3000, rng, np.array([-2.5, -2.5, -2.5, 2.5, 2.5, 2.5]))
    D = gen.isotropic_dirs(3000, rng)
    E = oracle.enter_points(g.box, O, D)
    c = oracle.cells(g.sites, g.box)
    off, idx = oracle.csr(c, len(g.sites))
    ref = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), E, D, off=off, idx=idx)
    vg = make(g)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    r64 = vg.trace(dev(O), dev(D), precision="fp64", segments=True, status=True, enter=True)
    t32 = vg.trace(dev(O), dev(D), precision="fp32", status=True, enter=True)
    from paper_1310_1854_gb300 import _lib
    st = r64.status.cpu().numpy()
    hit = ref.status == 0
    assert hit.sum() > 500 and (~hit).sum() > 500
    assert np.all(st[~hit] == _lib.RAY_OUTSIDE) and np.all(st[hit] == 0)
    ok = np.nonzero(hit & (ref.near_tie == 0))[0]
    check_segments(ref, ok, r64.seg_off, r64.seg_cell, r64.seg_len, diag, LEN64_REL)
    t = t32.tau.cpu().numpy().astype(np.float64)[ok]
    assert np.all(np.abs(t - ref.tau[ok]) <= TAU32_REL * ref.tau[ok])
    assert np.all(t32.tau.cpu().numpy()[~hit] == 0)
    # exact lengths from the entry points too
    rx = vg.trace(dev(O), dev(D), precision="fp32_exact", segments=True, enter=True)
    check_segments(ref, ok, rx.seg_off, rx.seg_cell, rx.seg_len, diag, 1e-6)
    tx = rx.tau.cpu().numpy().astype(np.float64)[ok]
    assert np.all(np.abs(tx - ref.tau[ok]) <= 1e-6 * ref.tau[ok])


def test_sphere_domain_parity():
    """A spherical domain (the paper notes the method carries over to other
    domain geometries, Sect. 2.2): the ball inscribed in the box, sites and
    rays inside it. Both forms against the oracle on every ray and in two
    lanes-per-ray shapes; every float64 path ends on the sphere."""
    g = gen.make_ball_grid(3000, 51)
    rays = gen.ball_rays(4000, 52)
    ref = oracle_full(g, rays, sphere=gen.UNIT_BALL)
    assert np.all(ref.status == 0)
    vg = run_case(g, rays, ref, sphere=gen.UNIT_BALL)
    r64 = vg.trace(dev(rays.origin), dev(rays.dir), precision="fp64", segments=True)
    so = r64.seg_off.cpu().numpy()
    L = np.add.reduceat(r64.seg_len.cpu().numpy(), so[:-1])
    end = rays.origin + L[:, None] * rays.dir
    np.testing.assert_allclose(np.linalg.norm(end, axis=1), 1.0, rtol=0, atol=1e-12)
    # exact lengths in the ball too (the sphere's exit as the wall candidate)
    rx = vg.trace(dev(rays.origin), dev(rays.dir), precision="fp32_exact", segments=True)
    ok = np.nonzero(ref.near_tie == 0)[0]
    check_segments(ref, ok, rx.seg_off, rx.seg_cell, rx.seg_len, 2.0 * np.sqrt(3.0), 1e-6)
    tx = rx.tau.cpu().numpy().astype(np.float64)[ok]
    assert np.all(np.abs(tx - ref.tau[ok]) <= 1e-6 * ref.tau[ok])


def test_sphere_domain_locate_and_entry():
    """C(r) in a spherical domain (points of the box outside the ball are
    outside the domain), and rays from outside the ball: each starts epsilon
    past its entry point, as the oracle's, and the paths match; rays that
    miss the ball are outside."""
    g = gen.make_ball_grid(2000, 53)
    vg = make(g, sphere=gen.UNIT_BALL)
    rng = gen.rng_for(54)
    P = np.concatenate([gen.uniform_points(4000, rng, g.box),
                        np.array([[0.0, 0, 1.0], [0.6, -0.8, 0], [0.0, 0.8, 0.6000001], [1.0, 1.0, 1.0]])])
    ref = oracle.locate(g.sites, g.box, P, sphere=gen.UNIT_BALL)
    assert (ref == -1).sum() > 1000
    for prec in ("fp32", "fp64"):
        np.testing.assert_array_equal(vg.locate(dev(P), precision=prec).cpu().numpy(), ref)
    O = gen.uniform_points(3000, rng, np.array([-2.5, -2.5, -2.5, 2.5, 2.5, 2.5]))
    D = gen.isotropic_dirs(3000, rng)
    E = oracle.enter_points(g.box, O, D, sphere=gen.UNIT_BALL)
    c = oracle.cells(g.sites, g.box)
    off, idx = oracle.csr(c, len(g.sites))
    tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), E, D, off=off, idx=idx, sphere=gen.UNIT_BALL)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    r64 = vg.trace(dev(O), dev(D), precision="fp64", segments=True, status=True, enter=True)
    t32 = vg.trace(dev(O), dev(D), precision="fp32", status=True, enter=True)
    from paper_1310_1854_gb300 import _lib
    hit = tr.status == 0
    assert hit.sum() > 300 and (~hit).sum() > 300
    assert np.all(r64.status.cpu().numpy()[~hit] == _lib.RAY_OUTSIDE)
    assert np.all(r64.status.cpu().numpy()[hit] == 0) and np.all(t32.status.cpu().numpy()[hit] == 0)
    ok = np.nonzero(hit & (tr.near_tie == 0))[0]
    check_segments(tr, ok, r64.seg_off, r64.seg_cell, r64.seg_len, diag, LEN64_REL)
    t = t32.tau.cpu().numpy().astype(np.float64)[ok]
    assert np.all(np.abs(t - tr.tau[ok]) <= TAU32_REL * tr.tau[ok])


def test_sphere_domain_in_a_batch():
    """A batch that mixes a spherical-domain grid with box grids gives each
    grid's single-grid tau bit for bit."""
    from paper_1310_1854_gb300 import Batch
    gs = gen.make_ball_grid(2000, 55)
    rs = gen.ball_rays(3000, 56)
    gb = gen.make_uniform_grid(1500, 57)
    rb = gen.uniform_rays(2000, 58)
    a = make(gs, sphere=gen.UNIT_BALL)
    b = make(gb)
    want = [a.trace(dev(rs.origin), dev(rs.dir)).tau.cpu().numpy(), b.trace(dev(rb.origin), dev(rb.dir)).tau.cpu().numpy()]
    bt = Batch([(a, dev(rs.origin), dev(rs.dir)), (b, dev(rb.origin), dev(rb.dir))])
    bt.run()
    for k in range(2):
        np.testing.assert_array_equal(bt.tau[k].cpu().numpy(), want[k])
    ref = oracle_full(gs, rs, sphere=gen.UNIT_BALL)
    ok = ref.near_tie == 0
    t = want[0].astype(np.float64)
    assert np.all(np.abs(t[ok] - ref.tau[ok]) <= TAU32_REL * ref.tau[ok])


def test_grid_quality_matches_oracle_locate():
    """Table 1's measure on a small disk grid: the GPU's C(r) gives the same
    cells as the oracle's brute force, hence the same statistic."""
    from paper_1310_1854_gb300.quality import grid_quality, sample_points
    g = gen.make_disk_grid(20_000, 320)
    vg = make(g)
    q = grid_quality(vg, g.rho, gen.disk_density, n_points=20_000, seed=5)
    P = sample_points(g.box, 20_000, 5)
    cell = oracle.locate(g.sites, g.box, P)
    d = gen.disk_density(P) - g.rho.astype(np.float64)[cell]
    assert q["std"] == pytest.approx(float(d.std()), rel=1e-12)
    assert q["mean"] == pytest.approx(float(d.mean()), rel=1e-9, abs=1e-15)


def test_grid_quality_in_a_spherical_domain():
    """The same measure over a ball: the sample points are spread over the
    ball, and the GPU's cells equal the oracle's C(r) there."""
    from paper_1310_1854_gb300.quality import grid_quality, sample_points
    g = gen.make_ball_grid(5000, 321)
    vg = make(g, sphere=gen.UNIT_BALL)

    def rho_true(p):
        return np.exp(-3.0 * np.linalg.norm(p, axis=1))
    q = grid_quality(vg, g.rho, rho_true, n_points=20_000, seed=6)
    P = sample_points(g.box, 20_000, 6, gen.UNIT_BALL)
    cell = oracle.locate(g.sites, g.box, P, sphere=gen.UNIT_BALL)
    assert np.all(cell >= 0)
    d = rho_true(P) - g.rho.astype(np.float64)[cell]
    assert q["std"] == pytest.approx(float(d.std()), rel=1e-12)


def test_gpu_cell_construction_host_fallback():
    """A cell beyond the GPU builder's fixed capacities (a site with 80
    neighbours on a sphere around it: more faces and vertices than one
    thread's polyhedron holds) is rebuilt by the host builder, and the grid
    still matches the host-built one."""
    from paper_1310_1854_gb300 import VoronoiGrid
    n = 80
    k = np.arange(n) + 0.5
    th = np.arccos(1.0 - 2.0 * k / n)
    ph = np.pi * (1.0 + 5.0 ** 0.5) * k
    shell = 0.5 * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    rng = gen.rng_for(335)
    far = rng.uniform(-1.0, 1.0, (3000, 3))
    far = far[np.linalg.norm(far, axis=1) > 0.75][:300]
    S = np.float32(np.concatenate([[[0.0, 0.0, 0.0]], shell, far])).astype(np.float64)
    host = VoronoiGrid(S, gen.CUBE_BOX, host_only=True)
    dev_ = VoronoiGrid(S, gen.CUBE_BOX, gpu_build=True)
    assert dev_.info()["host_fallback_cells"] >= 1
    ho, hi = host.neighbors()
    do, di = dev_.neighbors()
    assert set(di[do[0]:do[1]].tolist()) == set(hi[ho[0]:ho[1]].tolist())
    assert do[1] - do[0] == n
    for m in range(len(S)):
        a, b = set(hi[ho[m]:ho[m + 1]].tolist()), set(di[do[m]:do[m + 1]].tolist())
        assert len(a ^ b) <= 2, m   # at most planes that only touch the cell (R7)
    hv, hb = host.cells()
    dv, db = dev_.cells()
    np.testing.assert_allclose(dv, hv, rtol=1e-10)
    np.testing.assert_allclose(db, hb, rtol=0, atol=1e-12 * np.linalg.norm(gen.CUBE_BOX[3:] - gen.CUBE_BOX[:3]))
    np.testing.assert_allclose(dv.sum(), 8.0, rtol=1e-12)


@pytest.mark.parametrize("kind", ["uniform", "disk", "clumpy", "lattice"])
def test_gpu_cell_construction_matches_host(kind):
    from paper_1310_1854_gb300 import VoronoiGrid
    if kind == "uniform":
        g = gen.make_uniform_grid(20_000, 330)
    elif kind == "disk":
        g = gen.make_disk_grid(20_000, 331)
    elif kind == "clumpy":
        g = gen.make_clumpy_grid(20_000, 332, n_clumps=40)
    else:
        S = gen.bcc_lattice(8)
        g = gen.Grid(S, gen.CUBE_BOX.copy(), np.ones(len(S), np.float32))
    host = VoronoiGrid(g.sites, g.box, host_only=True)
    dev_ = VoronoiGrid(g.sites, g.box, gpu_build=True)
    ho, hi = host.neighbors()
    do, di = dev_.neighbors()
    np.testing.assert_array_equal(ho, do)
    np.testing.assert_array_equal(hi, di)
    hv, hb = host.cells()
    dv, db = dev_.cells()
    np.testing.assert_allclose(dv, hv, rtol=1e-10)
    np.testing.assert_allclose(db, hb, rtol=0, atol=1e-12 * np.linalg.norm(g.box[3:] - g.box[:3]))
    # against the oracle's own clipping on sampled cells: every face of
    # non-negligible area is in the GPU-built list (which may add planes
    # that only touch the cell, R7), volumes and bounding boxes agree
    ids = np.sort(gen.rng_for(334).choice(len(g.sites), min(400, len(g.sites)), replace=False))
    c = oracle.cells(g.sites, g.box, ids=ids)
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    for k, m in enumerate(ids):
        ours = set(di[do[m]:do[m + 1]].tolist())
        faces = c.nbr[k]
        big = set(faces[c.area[k] > 1e-9 * c.area[k].sum()].tolist())
        assert big <= ours, (m, big - ours)
        assert len(ours - set(faces.tolist())) <= 2, m
    np.testing.assert_allclose(dv[ids], c.vol, rtol=1e-10)
    np.testing.assert_allclose(db[ids], c.bbox, rtol=0, atol=1e-12 * diag)
    assert dev_.info()["host_fallback_cells"] < 0.001 * len(g.sites)
    # same lists, same layout: traversal agrees to the bit
    rays = gen.uniform_rays(2000, 333, g.box)
    a = make(g)
    dev_.set_density(dev(g.rho), 1.0)
    O, D = dev(rays.origin), dev(rays.dir)
    np.testing.assert_array_equal(a.trace(O, D, precision="fp32").tau.cpu().numpy(),
                                  dev_.trace(O, D, precision="fp32").tau.cpu().numpy())


def test_autotune_applies_and_caches(tmp_path):
    """The launch-shape tuner times its candidate shapes on the GPU, applies
    the fastest, caches it, and a later call takes it from the cache; tau
    does not depend on the shape."""
    from paper_1310_1854_gb300 import tune
    g, rays = gen.config2(n_rays=100_000)
    vg = make(g)
    O, D = dev(rays.origin), dev(rays.dir)
    ref = vg.trace(O, D).tau.cpu().numpy()
    path = str(tmp_path / "tune.json")
    space = ((1, 128, 0), (2, 128, 0), (1, 64, 0))
    r = tune.autotune(vg, O, D, sample=50_000, space=space, path=path)
    assert not r["cached"] and (r["lanes_per_ray"], r["block"], r["blocks_per_sm"]) in space
    assert len(r["table"]) == len(space) and all(v > 0 for v in r["table"].values())
    L = vg.get_launch()
    assert (L["lanes_per_ray"], L["block"], L["blocks_per_sm"]) == (r["lanes_per_ray"], r["block"], r["blocks_per_sm"])
    np.testing.assert_array_equal(vg.trace(O, D).tau.cpu().numpy(), ref)
    vg.set_launch()
    r2 = tune.autotune(vg, O, D, sample=50_000, space=space, path=path)
    assert r2["cached"] and r2["lanes_per_ray"] == r["lanes_per_ray"]
    assert vg.get_launch()["lanes_per_ray"] == r["lanes_per_ray"]


@pytest.mark.parametrize("chunk", range(4))
def test_fuzz_degenerate_small_grids(chunk):
    """Seeded small grids in random boxes (lattices, jittered lattices,
    coplanar sites, near-duplicate pairs, sites on the walls) with rays from
    sites, from walls and along the axes: both forms against the oracle's
    neighbour-list traversal. Statuses agree on every ray; away from near
    ties the cell sequences are identical, float64 lengths and tau within
    1e-12; on every ray the summed length is the path length (float64
    within 1e-12 of the diagonal). The float32 form decides every exit
    exactly but places the crossing to within about 12 u N^2 / (n.k) (u =
    2^-24, N the cell's largest |n|_1): a grazing exit between cells whose
    densities differ 100-fold, which these grids contain and the workloads
    rarely do, moves tau by more than 1e-5 relative (1.8e-5 here), so its
    tau is held to 1e-4 here and to 1e-5 on the workloads."""
    from tests import fuzz_cases
    for i in range(chunk * 30, chunk * 30 + 30):
        kind, g, rays = fuzz_cases.case(i)
        ref = oracle_full(g, rays)
        vg = make(g)
        diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
        O, D = dev(rays.origin), dev(rays.dir)
        ok = np.nonzero(ref.near_tie == 0)[0]
        r64 = vg.trace(O, D, precision="fp64", segments=True, status=True)
        r32 = vg.trace(O, D, precision="fp32", segments=True, status=True)
        for r in (r64, r32):
            np.testing.assert_array_equal(r.status.cpu().numpy(), ref.status, err_msg=f"case {i} ({kind})")
        try:
            check_segments(ref, ok, r64.seg_off, r64.seg_cell, r64.seg_len, diag, LEN64_REL)
            check_segments(ref, ok, r32.seg_off, r32.seg_cell, r32.seg_len, diag, None)
        except AssertionError as e:
            raise AssertionError(f"case {i} ({kind}): {e}")
        t64 = r64.tau.cpu().numpy()[ok]
        np.testing.assert_allclose(t64, ref.tau[ok], rtol=1e-12, atol=1e-300, err_msg=f"case {i} ({kind})")
        t32 = r32.tau.cpu().numpy().astype(np.float64)[ok]
        rt = ref.tau[ok]
        assert np.all(np.abs(t32 - rt) <= 10 * TAU32_REL * rt), f"case {i} ({kind}): float32 tau"
        so = r64.seg_off.cpu().numpy()
        total = np.add.reduceat(np.concatenate([r64.seg_len.cpu().numpy(), [0.0]]), so[:-1]) * (np.diff(so) > 0)
        np.testing.assert_allclose(total, ref.length, rtol=0, atol=1e-12 * diag, err_msg=f"case {i} ({kind})")


def test_fuzz_gpu_cell_construction():
    """The GPU cell construction on the seeded degenerate grids: every face
    of non-negligible area in the oracle's clipping is in the GPU-built list,
    any extra plane only touches the cell (R7), volumes agree, and the
    float32 traversal over the GPU-built grid matches the oracle away from
    near ties."""
    from tests import fuzz_cases
    from paper_1310_1854_gb300 import VoronoiGrid
    for i in range(0, 120, 2):
        kind, g, rays = fuzz_cases.case(i)
        c = oracle.cells(g.sites, g.box)
        vg = VoronoiGrid(g.sites, g.box, gpu_build=True)
        do, di = vg.neighbors()
        dv, _ = vg.cells()
        for m in range(len(g.sites)):
            ours = set(di[do[m]:do[m + 1]].tolist())
            faces = c.nbr[m]
            big = set(faces[c.area[m] > 1e-9 * c.area[m].sum()].tolist())
            assert big <= ours, (i, kind, m, big - ours)
            assert len(ours - set(faces.tolist())) <= 2, (i, kind, m, ours - set(faces.tolist()))
        # thin cells (near-duplicate pairs) round differently in another cut order
        np.testing.assert_allclose(dv, c.vol, rtol=1e-10, atol=1e-12 * np.prod(g.box[3:] - g.box[:3]),
                                   err_msg=f"case {i} ({kind})")
        vg.set_density(dev(g.rho), float(g.kappa))
        off, idx = oracle.csr(c, len(g.sites))
        ref = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin, rays.dir, off=off, idx=idx,
                           kappa=float(g.kappa))
        ok = np.nonzero(ref.near_tie == 0)[0]
        t32 = vg.trace(dev(rays.origin), dev(rays.dir), precision="fp32").tau.cpu().numpy().astype(np.float64)[ok]
        assert np.all(np.abs(t32 - ref.tau[ok]) <= TAU32_REL * ref.tau[ok]), f"case {i} ({kind})"


def test_fp32_exact_lengths():
    """The float32 form with exact lengths: the float32 form's decisions (the
    same cells) and each crossing's length from the exact site difference in
    float-pair arithmetic, so that tau and every length are within 1e-6 of
    the oracle's (relative; 1e-12 of the diagonal for lengths below 1e-6 of
    it), on the first workload, small disk and clumpy grids and the seeded
    degenerate grids, including the grazing exit that puts the plain float32
    form's tau 1.8e-5 off."""
    from tests import fuzz_cases
    cases = [("config1",) + gen.config1(3000), ("disk", gen.make_disk_grid(20_000, 101), gen.disk_rays(3000, 102)),
             ("clumpy", gen.make_clumpy_grid(20_000, 103, n_clumps=40), gen.uniform_rays(3000, 104))]
    cases += [("fuzz %d" % i,) + fuzz_cases.case(i)[1:] for i in range(0, 120, 4)] + [("fuzz 17",) + fuzz_cases.case(17)[1:]]
    worst = 0.0
    for name, g, rays in cases:
        ref = oracle_full(g, rays)
        vg = make(g)
        diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
        O, D = dev(rays.origin), dev(rays.dir)
        ok = np.nonzero(ref.near_tie == 0)[0]
        rx = vg.trace(O, D, precision="fp32_exact", segments=True, status=True)
        r32 = vg.trace(O, D, precision="fp32", segments=True)
        np.testing.assert_array_equal(rx.status.cpu().numpy(), ref.status, err_msg=name)
        try:
            check_segments(ref, ok, rx.seg_off, rx.seg_cell, rx.seg_len, diag, 1e-6)
        except AssertionError as e:
            raise AssertionError(f"{name}: {e}")
        # the same decisions as the float32 form: the same cells on every ray
        np.testing.assert_array_equal(rx.seg_off.cpu().numpy(), r32.seg_off.cpu().numpy(), err_msg=name)
        np.testing.assert_array_equal(rx.seg_cell.cpu().numpy(), r32.seg_cell.cpu().numpy(), err_msg=name)
        tx = rx.tau.cpu().numpy().astype(np.float64)[ok]
        rt = ref.tau[ok]
        err = np.abs(tx - rt) / np.maximum(rt, 1e-300)
        assert np.all(err[rt > 0] <= 1e-6), f"{name}: max rel tau error {err.max()}"
        worst = max(worst, float(err[rt > 0].max(initial=0.0)))
    assert tx.dtype == np.float64 and worst <= 1e-6
    # only vgrid_trace takes it
    from paper_1310_1854_gb300 import VGridError
    with pytest.raises(VGridError):
        vg.locate(O, precision="fp32_exact")
