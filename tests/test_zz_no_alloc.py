"""vgrid_trace_noalloc: tau per ray with no device allocation.

This entry point is for callers that cannot call cudaMalloc (their device
memory is owned by another allocator under a fixed budget, or they run
latency-bound loops that must not take the implicit synchronisation of
cudaMalloc/cudaFree). Its work buffers live in a fixed device array inside
the library. Called through the C-ABI, it must give what vgrid_trace gives
in tau mode, to the bit, on two calls in a row (the second one sees the
array as the first left it), in every arithmetic form.
"""
import ctypes

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_trace_on_two_calls():
    """Same kernel, same start records: tau and status equal vgrid_trace's to
    the bit, in every form, on two calls in a row (the second sees the array
    as the first left it), once without a status buffer."""
    from paper_1310_1854_gb300 import VoronoiGrid, _lib
    lib = _lib.load()
    g, rays = gen.config1(6000)
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).cuda(), 1.0)
    O = torch.from_numpy(rays.origin).cuda()
    D = torch.from_numpy(rays.dir).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for prec, name, dt in ((_lib.FP32_RECHECK, "fp32", torch.float32), (_lib.FP64, "fp64", torch.float64),
                           (_lib.FP32_EXACT, "fp32_exact", torch.float32)):
        # two calls in a row: all rays, then a shifted subset, so the second
        # call starts from the array the first one left behind; the second
        # passes no status buffer (NULL is allowed)
        for lo, hi, with_status in ((0, 6000, True), (1234, 5000, False)):
            o, d = O[lo:hi].contiguous(), D[lo:hi].contiguous()
            want = vg.trace(o, d, precision=name, status=True)
            got = torch.full((hi - lo,), float("nan"), dtype=dt, device="cuda")
            st = torch.full((hi - lo,), -1, dtype=torch.int32, device="cuda")
            rc = lib.vgrid_trace_noalloc(vg._h, _p(o), _p(d), hi - lo, prec, _p(got),
                                         _p(st) if with_status else None, stream)
            assert rc == 0, lib.vgrid_last_error()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), want.tau.cpu().numpy())
            if with_status:
                np.testing.assert_array_equal(st.cpu().numpy(), want.status.cpu().numpy())
            else:
                assert np.all(st.cpu().numpy() == -1)  # untouched
    # no rays: nothing to do, nothing written
    t0 = torch.full((1,), 7.0, dtype=torch.float32, device="cuda")
    rc = lib.vgrid_trace_noalloc(vg._h, _p(O), _p(D), 0, _lib.FP32_RECHECK, _p(t0), None, stream)
    assert rc == 0, lib.vgrid_last_error()
    torch.cuda.synchronize()
    assert float(t0[0]) == 7.0


def test_noalloc_rejects_more_rays_than_its_array():
    from paper_1310_1854_gb300 import VoronoiGrid, _lib
    lib = _lib.load()
    vg = VoronoiGrid(gen.cubic_lattice(2), gen.CUBE_BOX)
    O = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    tau = torch.zeros(1, dtype=torch.float32, device="cuda")
    n = _lib.NOALLOC_MAX_RAYS + 1
    # rejected before anything is enqueued, so the short buffers are never read
    rc = lib.vgrid_trace_noalloc(vg._h, _p(O), _p(O), n, _lib.FP32_RECHECK, _p(tau), None, None)
    assert rc == _lib.ERR_ARG
    assert b"VGRID_NOALLOC_MAX_RAYS" in lib.vgrid_last_error()
