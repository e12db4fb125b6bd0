"""Straight-path traversal of 3D Voronoi grids on one GB300 GPU.

Python face of libvgrid (include/vgrid.h): argument marshalling only, every
step of the path runs in the library's CUDA kernels. PyTorch supplies device
memory and streams.

The method is that of Camps, Baes & Saftly (2013), Sect. 2: rays are
followed cell by cell through the Voronoi tessellation of a set of sites in
a cuboidal domain; the exit from the current cell is the nearest bisector
plane (Eq. 1-4) or domain wall (Eq. 5) ahead; the optical depth is
tau = sum kappa rho_cell l.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib
from ._lib import VGridError, check, load

__all__ = ["VoronoiGrid", "Batch", "TraceResult", "optical_depth", "probe_l2", "VGridError", "load"]

_PREC = {"fp64": _lib.FP64, "fp32": _lib.FP32_RECHECK, "fp32_exact": _lib.FP32_EXACT}


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else None


def _rays(t, name, device):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA float64 tensor of shape (N, 3)")
    if t.dim() != 2 or t.shape[1] != 3:
        raise ValueError(f"{name} must have shape (N, 3)")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, the grid on {device}")
    return t.contiguous()


@dataclasses.dataclass
class TraceResult:
    tau: torch.Tensor | None
    seg_off: torch.Tensor | None = None
    seg_cell: torch.Tensor | None = None
    seg_len: torch.Tensor | None = None
    status: torch.Tensor | None = None
    stats: dict | None = None

    def segments(self, i):
        a, b = int(self.seg_off[i]), int(self.seg_off[i + 1])
        return self.seg_cell[a:b], self.seg_len[a:b]


class VoronoiGrid:
    """A Voronoi grid on the current CUDA device.

    sites: (M, 3) array of float32-representable positions inside ``box``
    (xmin, ymin, zmin, xmax, ymax, zmax). The neighbour lists, cell volumes,
    bounding boxes and block lists are built on the host by the library.
    ``sphere=(cx, cy, cz, R)`` makes the domain that ball (inside ``box``,
    every site inside it): paths end on the sphere, points outside it are
    outside the domain.
    """

    def __init__(self, sites, box, *, round_sites=False, reorder=True, blocks_per_site=8.0,
                 max_steps=100_000, threads=0, device=None, host_only=False, gpu_build=False, zero_run_max=4,
                 sphere=None):
        lib = load()
        S = np.ascontiguousarray(np.asarray(sites, dtype=np.float64).reshape(-1, 3))
        B = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(6))
        opts = _lib.Opts()
        lib.vgrid_default_opts(ctypes.byref(opts))
        opts.threads = int(threads)
        opts.round_sites = int(bool(round_sites))
        opts.reorder = int(bool(reorder))
        opts.blocks_per_site = float(blocks_per_site)
        opts.max_steps = int(max_steps)
        opts.host_only = int(bool(host_only))
        opts.gpu_build = int(bool(gpu_build))
        opts.zero_run_max = int(zero_run_max)
        if sphere is not None:
            opts.domain = _lib.DOMAIN_SPHERE
            for c, v in enumerate(np.asarray(sphere, np.float64).reshape(4)):
                opts.sphere[c] = float(v)
        h = ctypes.c_void_p()
        args = (S.ctypes.data_as(ctypes.c_void_p), S.shape[0], B.ctypes.data_as(ctypes.c_void_p),
                ctypes.byref(opts), ctypes.byref(h))
        if host_only:
            self.device = None
            check(lib.vgrid_create(*args))
        else:
            self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
            with torch.cuda.device(self.device):
                torch.cuda.init()
                check(lib.vgrid_create(*args))
        self._h = h
        self.M = S.shape[0]
        self.box = B.copy()
        self.sphere = None if sphere is None else np.asarray(sphere, np.float64).reshape(4).copy()
        self.kappa = 1.0
        self._seg_per_ray = None  # segments per ray of the last segment-list call

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().vgrid_destroy(h)
            except Exception:
                pass
            self._h = None

    # ------------------------------------------------------------------ info
    def info(self) -> dict:
        i = _lib.Info()
        check(load().vgrid_info(self._h, ctypes.byref(i)))
        return {"M": i.M, "nnz": i.nnz, "block_entries": i.block_entries, "block_dim": list(i.block_dim),
                "box": list(i.box), "build_seconds": i.build_seconds, "device_bytes": i.device_bytes,
                "host_fallback_cells": i.host_fallback_cells, "phase_seconds": list(i.phase_seconds),
                "rel_bytes": i.rel_bytes}

    def neighbors(self):
        """CSR (off int64[M+1], idx int32) in the caller's ids, walls -1..-6."""
        nnz = self.info()["nnz"]
        off = np.zeros(self.M + 1, np.int64)
        idx = np.zeros(max(nnz, 1), np.int32)
        check(load().vgrid_get_neighbors(self._h, off.ctypes.data_as(ctypes.c_void_p),
                                         idx.ctypes.data_as(ctypes.c_void_p)))
        return off, idx[:nnz]

    def cells(self):
        """(volume float64[M], bbox float64[M, 6])."""
        vol = np.zeros(self.M, np.float64)
        bb = np.zeros((self.M, 6), np.float64)
        check(load().vgrid_get_cells(self._h, vol.ctypes.data_as(ctypes.c_void_p), bb.ctypes.data_as(ctypes.c_void_p)))
        return vol, bb

    # -------------------------------------------------------------- launch
    def set_launch(self, lanes_per_ray=1, block=128, blocks_per_sm=0, fp64_lanes_per_ray=1, order=0):
        """Launch shape of the traversal kernels; order: 1 = longest estimated
        path first, -1 = the caller's order, 0 = automatic (see vgrid.h)."""
        l = _lib.Launch(int(lanes_per_ray), int(block), int(blocks_per_sm), int(fp64_lanes_per_ray), int(order))
        check(load().vgrid_set_launch(self._h, ctypes.byref(l)))

    def get_launch(self):
        l = _lib.Launch()
        check(load().vgrid_get_launch(self._h, ctypes.byref(l)))
        return {"lanes_per_ray": l.lanes_per_ray, "block": l.block, "blocks_per_sm": l.blocks_per_sm,
                "fp64_lanes_per_ray": l.fp64_lanes_per_ray, "order": l.order}

    def enable_timing(self, enable=True):
        check(load().vgrid_enable_timing(self._h, int(bool(enable))))

    def read_timing(self):
        """(locate_ms, trace_ms, traversal launches) since the last read."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        check(load().vgrid_read_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return a.value, b.value, n.value

    # ------------------------------------------------------------- density
    def set_density(self, rho: torch.Tensor, kappa: float = 1.0, stream=None):
        if rho.dtype != torch.float32 or not rho.is_cuda or rho.numel() != self.M:
            raise TypeError("rho must be a CUDA float32 tensor with one value per site")
        rho = rho.contiguous()
        check(load().vgrid_set_density(self._h, _ptr(rho), float(kappa), _stream(stream)))
        self.kappa = float(kappa)

    # ------------------------------------------------------------- compute
    def locate(self, points: torch.Tensor, precision="fp32", stream=None) -> torch.Tensor:
        P = _rays(points, "points", self.device)
        out = torch.empty(P.shape[0], dtype=torch.int32, device=self.device)
        check(load().vgrid_locate(self._h, _ptr(P), P.shape[0], _PREC[precision], _ptr(out), _stream(stream)))
        return out

    def trace(self, origin, direction, precision="fp32", segments=False, status=False, stats=False,
              seg_capacity=None, stream=None, out_tau=None, enter=False) -> TraceResult:
        lib = load()
        O = _rays(origin, "origin", self.device)
        D = _rays(direction, "direction", self.device)
        N = O.shape[0]
        prec = _PREC[precision]
        flag = _lib.ENTER if enter else 0
        tdt = torch.float64 if prec == _lib.FP64 else torch.float32
        tau = out_tau if out_tau is not None else torch.empty(N, dtype=tdt, device=self.device)
        st = torch.empty(N, dtype=torch.int32, device=self.device) if status else None
        cs = _lib.Stats() if (stats or segments) else None
        sref = ctypes.byref(cs) if cs is not None else None
        if not segments:
            check(lib.vgrid_trace(self._h, _ptr(O), _ptr(D), N, prec, _lib.TAU | flag, _ptr(tau), None, None, None, 0,
                                  _ptr(st), sref, _stream(stream)))
            return TraceResult(tau, status=st, stats=cs.as_dict() if cs is not None else None)
        seg_off = torch.empty(N + 1, dtype=torch.int64, device=self.device)
        if seg_capacity is not None:
            cap = int(seg_capacity)
        elif self._seg_per_ray is not None:
            # a guess from the last call (one traversal when it is enough;
            # otherwise the call reports the total and runs again); large
            # calls count first rather than size buffers on a guess
            cap = int(N * self._seg_per_ray * 1.25) + 1024
            if cap > (1 << 27):
                cap = 0
        else:
            cap = 0  # the first call counts, then traces again with the total
        cells = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
        lens = torch.empty(max(cap, 1), dtype=tdt, device=self.device)
        rc = lib.vgrid_trace(self._h, _ptr(O), _ptr(D), N, prec, _lib.SEGMENTS | flag, _ptr(tau), _ptr(seg_off),
                             _ptr(cells), _ptr(lens), cap, _ptr(st), sref, _stream(stream))
        if rc == _lib.ERR_CAPACITY and seg_capacity is None:
            total = int(seg_off[N].item())
            cells = torch.empty(max(total, 1), dtype=torch.int32, device=self.device)
            lens = torch.empty(max(total, 1), dtype=tdt, device=self.device)
            rc = lib.vgrid_trace(self._h, _ptr(O), _ptr(D), N, prec, _lib.SEGMENTS | flag, _ptr(tau), _ptr(seg_off),
                                 _ptr(cells), _ptr(lens), total, _ptr(st), sref, _stream(stream))
        check(rc)
        total = int(seg_off[N].item())
        if N > 0:
            self._seg_per_ray = total / N
        return TraceResult(tau, seg_off, cells[:total], lens[:total], st, cs.as_dict())

    def trace_host(self, origin, direction, precision="fp32", out_tau=None, status=False, stats=False, chunk=0,
                   stream=None, wait=True) -> TraceResult:
        """tau of rays held in host memory (CPU float64 tensors of shape
        (N, 3); pinned for the copies to overlap the traversal), results in
        host memory: vgrid_trace_host. With wait=False (and no stats) the call
        only queues the work: the results are valid once the stream has been
        synchronised, and consecutive calls overlap their copies with the
        previous traversal."""
        for t, name in ((origin, "origin"), (direction, "direction")):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.is_cuda:
                raise TypeError(f"{name} must be a CPU float64 tensor of shape (N, 3)")
            if t.dim() != 2 or t.shape[1] != 3:
                raise ValueError(f"{name} must have shape (N, 3)")
        O, D = origin.contiguous(), direction.contiguous()
        N = O.shape[0]
        if D.shape[0] != N:
            raise ValueError("origin and direction differ in length")
        prec = _PREC[precision]
        tdt = torch.float64 if prec == _lib.FP64 else torch.float32
        tau = out_tau if out_tau is not None else torch.empty(N, dtype=tdt, pin_memory=O.is_pinned())
        if tau.is_cuda or tau.dtype != tdt or tau.numel() != N or not tau.is_contiguous():
            raise ValueError(f"out_tau must be a contiguous CPU {tdt} tensor of N elements")
        st = torch.empty(N, dtype=torch.int32, pin_memory=O.is_pinned()) if status else None
        cs = _lib.Stats() if stats else None
        check(load().vgrid_trace_host(self._h, _ptr(O), _ptr(D), N, prec, _ptr(tau), _ptr(st), int(chunk),
                                      ctypes.byref(cs) if cs is not None else None, _stream(stream)))
        if wait and N > 0:
            (stream if stream is not None else torch.cuda.current_stream()).synchronize()
        return TraceResult(tau, status=st, stats=cs.as_dict() if cs is not None else None)

    def interact(self, origin, direction, tau_int: torch.Tensor, weight: torch.Tensor | None = None,
                 absorbed: bool | torch.Tensor = False, stream=None):
        """Where each ray's running tau reaches tau_int: (cell int32, s float32,
        absorbed float32[M] or None); cell -1 means the ray left the domain."""
        O = _rays(origin, "origin", self.device)
        D = _rays(direction, "direction", self.device)
        N = O.shape[0]
        ti = tau_int.detach().to(torch.float32).contiguous()
        w = weight.detach().to(torch.float32).contiguous() if weight is not None else None
        cell = torch.empty(N, dtype=torch.int32, device=self.device)
        s = torch.empty(N, dtype=torch.float32, device=self.device)
        if isinstance(absorbed, torch.Tensor):
            ab = absorbed
        else:
            ab = torch.zeros(self.M, dtype=torch.float32, device=self.device) if absorbed else None
        check(load().vgrid_interact(self._h, _ptr(O), _ptr(D), N, _ptr(ti), _ptr(w), _ptr(cell), _ptr(s), _ptr(ab),
                                    _stream(stream)))
        return cell, s, ab

    def segments_grad(self, res: TraceResult, dL_dtau: torch.Tensor, out: torch.Tensor | None = None, stream=None,
                      kappa: float | None = None):
        """dL/drho (float32[M]) from the float32 segment lists of a trace
        (``trace(..., segments=True)``) without tracing again; accumulates
        into ``out``. ``kappa``: the opacity the lists' tau was computed
        with (default: the grid's current one)."""
        if res.seg_off is None or res.seg_len.dtype != torch.float32:
            raise TypeError("needs the float32 segment lists of trace(..., precision='fp32', segments=True)")
        N = res.seg_off.shape[0] - 1
        g = dL_dtau.detach().to(torch.float32).contiguous()
        if g.numel() != N:
            raise ValueError("dL_dtau needs one value per ray of the trace")
        if out is None:
            out = torch.zeros(self.M, dtype=torch.float32, device=self.device)
        k = self.kappa if kappa is None else float(kappa)
        check(load().vgrid_segments_grad(self._h, _ptr(res.seg_off), _ptr(res.seg_cell), _ptr(res.seg_len), N, _ptr(g),
                                         k, _ptr(out), _stream(stream)))
        return out

    def trace_grad(self, origin, direction, dL_dtau: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """dL/drho (float32[M]) for dL/dtau per ray; accumulates into ``out``."""
        O = _rays(origin, "origin", self.device)
        D = _rays(direction, "direction", self.device)
        g = dL_dtau.detach().to(torch.float32).contiguous()
        if out is None:
            out = torch.zeros(self.M, dtype=torch.float32, device=self.device)
        check(load().vgrid_trace_grad(self._h, _ptr(O), _ptr(D), O.shape[0], _ptr(g), _ptr(out), _stream(stream)))
        return out


class Batch:
    """Many (grid, rays) sets traced in one persistent launch, float32 form.

    ``sets`` is a list of (VoronoiGrid, origin, direction); outputs are
    allocated here. With ``graph=True`` the launch sequence is captured into a
    CUDA graph on the first run and replayed afterwards.
    """

    def __init__(self, sets, lanes_per_ray=1, block=128, blocks_per_sm=0, order=0):
        self._keep = []
        self.sets = list(sets)
        arr = (_lib.Rayset * len(sets))()
        self.tau = []
        self.status = []
        for i, (grid, o, d) in enumerate(sets):
            O = _rays(o, "origin", grid.device)
            D = _rays(d, "direction", grid.device)
            t = torch.empty(O.shape[0], dtype=torch.float32, device=grid.device)
            s = torch.empty(O.shape[0], dtype=torch.int32, device=grid.device)
            self._keep += [grid, O, D, t, s]
            self.tau.append(t)
            self.status.append(s)
            arr[i] = _lib.Rayset(grid._h.value, O.data_ptr() if O.numel() else None,
                                 D.data_ptr() if D.numel() else None, O.shape[0],
                                 t.data_ptr() if t.numel() else None, s.data_ptr() if s.numel() else None)
        l = _lib.Launch(int(lanes_per_ray), int(block), int(blocks_per_sm), 0, int(order))
        h = ctypes.c_void_p()
        check(load().vgrid_batch_create(arr, len(sets), ctypes.byref(l), ctypes.byref(h)))
        self._h = h

    def set_launch(self, lanes_per_ray=1, block=128, blocks_per_sm=0, order=0):
        """Launch shape of the batch's traversal; order 1 takes the work items
        of all sets longest estimated path first, otherwise set after set.
        A captured graph is dropped (the next graph run captures again)."""
        l = _lib.Launch(int(lanes_per_ray), int(block), int(blocks_per_sm), 0, int(order))
        check(load().vgrid_batch_set_launch(self._h, ctypes.byref(l)))

    def get_launch(self):
        l = _lib.Launch()
        check(load().vgrid_batch_get_launch(self._h, ctypes.byref(l)))
        return {"lanes_per_ray": l.lanes_per_ray, "block": l.block, "blocks_per_sm": l.blocks_per_sm,
                "order": l.order}

    @property
    def rays(self) -> int:
        return sum(int(t.numel()) for t in self.tau)

    def run(self, graph=False, stats=False, stream=None):
        cs = _lib.Stats() if stats else None
        check(load().vgrid_batch_run(self._h, int(bool(graph)), ctypes.byref(cs) if cs is not None else None,
                                     _stream(stream)))
        return cs.as_dict() if cs is not None else None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                load().vgrid_batch_destroy(h)
            except Exception:
                pass
            self._h = None


def probe_l2(nbytes: int, mode: str = "stream", stream=None) -> float:
    """Read-bandwidth ceiling (GB/s) measured on the current device with a
    buffer of ``nbytes`` (held in L2 when smaller than it): ``"stream"``,
    256-bit loads over the whole buffer, or ``"chase"``, a dependent chain of
    288-byte blocks at random positions per thread (vgrid_probe_l2)."""
    out = ctypes.c_double()
    check(load().vgrid_probe_l2(int(nbytes), {"stream": 0, "chase": 1}[mode], ctypes.byref(out), _stream(stream)))
    return out.value


class _OpticalDepth(torch.autograd.Function):
    """tau(rho) for fixed rays. Backward is the adjoint from the segment lists
    kept by forward (keep_segments), else the library's adjoint traversal.
    The adjoint uses the kappa of this forward call, whatever the grid holds
    by the time backward runs (the paths do not depend on rho or kappa).
    With precision "fp32_exact" the lengths of both passes come from the
    float32 form with exact lengths (backward traces again with it when the
    lists were not kept)."""

    @staticmethod
    def forward(ctx, rho, grid, origin, direction, kappa, keep_segments, precision):
        grid.set_density(rho.detach().to(torch.float32).contiguous(), kappa)
        res = grid.trace(origin, direction, precision=precision, segments=keep_segments)
        ctx.grid = grid
        ctx.kappa = float(kappa)
        ctx.precision = precision
        ctx.res = res if keep_segments else None
        ctx.save_for_backward(origin, direction)
        return res.tau

    @staticmethod
    def backward(ctx, g):
        grid, kappa = ctx.grid, ctx.kappa
        g = g.contiguous()
        if ctx.res is not None:
            d = grid.segments_grad(ctx.res, g, kappa=kappa)
        else:
            origin, direction = ctx.saved_tensors
            if ctx.precision != "fp32":
                d = grid.segments_grad(grid.trace(origin, direction, precision=ctx.precision, segments=True), g,
                                       kappa=kappa)
            elif grid.kappa == kappa:
                d = grid.trace_grad(origin, direction, g)
            elif grid.kappa != 0.0:
                # the adjoint traversal multiplies by the grid's kappa
                d = grid.trace_grad(origin, direction, g * (kappa / grid.kappa))
            else:
                d = grid.segments_grad(grid.trace(origin, direction, precision="fp32", segments=True), g,
                                       kappa=kappa)
        return d, None, None, None, None, None, None


def optical_depth(grid: VoronoiGrid, rho: torch.Tensor, origin: torch.Tensor, direction: torch.Tensor,
                  kappa: float = 1.0, keep_segments: bool = True, precision: str = "fp32") -> torch.Tensor:
    """Differentiable tau per ray with respect to the per-cell densities rho.

    With keep_segments (default) forward keeps the segment lists (8 bytes per
    segment on the device until backward) and backward reads them instead of
    tracing the rays again; without, backward traces again. precision:
    "fp32" (the float32 form) or "fp32_exact" (the same cells, every length
    from the exact site difference)."""
    if precision not in ("fp32", "fp32_exact"):
        raise ValueError("optical_depth takes precision 'fp32' or 'fp32_exact'")
    return _OpticalDepth.apply(rho, grid, origin, direction, kappa, bool(keep_segments), precision)
