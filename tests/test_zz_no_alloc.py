"""vgrid_trace_noalloc: tau per ray with no device allocation.

This entry point is for callers that cannot call cudaMalloc (their device
memory is owned by another allocator under a fixed budget, or they run
latency-bound loops that must not take the implicit synchronisation of
cudaMalloc/cudaFree). Its work buffers live in a fixed device array inside
the library. Called through the C-ABI, it must give what vgrid_trace gives
in tau mode, on two calls in a row (the second one sees the array as the
first left it), in both arithmetic forms.
"""
import ctypes

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu

TAU32_REL = 1e-5
TAU64_REL = 1e-12


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_trace_on_two_calls():
    from paper_1310_1854_gb300 import VoronoiGrid, _lib
    lib = _lib.load()
    g, rays = gen.config1(6000)
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).cuda(), 1.0)
    O = torch.from_numpy(rays.origin).cuda()
    D = torch.from_numpy(rays.dir).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for prec, name, dt, rel in ((_lib.FP32_RECHECK, "fp32", torch.float32, TAU32_REL),
                                (_lib.FP64, "fp64", torch.float64, TAU64_REL)):
        # two calls in a row: all rays, then a shifted subset, so the second
        # call starts from the array the first one left behind
        for lo, hi in ((0, 6000), (1234, 5000)):
            o, d = O[lo:hi].contiguous(), D[lo:hi].contiguous()
            want = vg.trace(o, d, precision=name).tau
            got = torch.full((hi - lo,), float("nan"), dtype=dt, device="cuda")
            st = torch.full((hi - lo,), -1, dtype=torch.int32, device="cuda")
            rc = lib.vgrid_trace_noalloc(vg._h, _p(o), _p(d), hi - lo, prec, _p(got), _p(st), stream)
            assert rc == 0, lib.vgrid_last_error()
            torch.cuda.synchronize()
            w = want.double().cpu().numpy()
            x = got.double().cpu().numpy()
            assert np.all(np.isfinite(x))
            assert np.all(np.abs(x - w) <= rel * np.abs(w)), np.max(np.abs(x - w) / np.maximum(np.abs(w), 1e-300))
            assert np.all(st.cpu().numpy() == 0)


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
