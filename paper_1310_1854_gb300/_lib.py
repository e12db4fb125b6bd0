"""ctypes declarations of the libvgrid C-ABI (include/vgrid.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_float = ctypes.c_float
c_void_p = ctypes.c_void_p

OK = 0
ERR_ARG = -1
ERR_DUP_SITE = -2
ERR_OUTSIDE = -3
ERR_CAPACITY = -4
ERR_STEP_LIMIT = -5
ERR_CUDA = -6
ERR_NOMEM = -7
ERR_BUILD = -8
ERROR_NAMES = {ERR_ARG: "ARG", ERR_DUP_SITE: "DUP_SITE", ERR_OUTSIDE: "OUTSIDE", ERR_CAPACITY: "CAPACITY",
               ERR_STEP_LIMIT: "STEP_LIMIT", ERR_CUDA: "CUDA", ERR_NOMEM: "NOMEM", ERR_BUILD: "BUILD"}

FP64 = 0
FP32_RECHECK = 1
FP32_EXACT = 2
TAU = 0
SEGMENTS = 1
ENTER = 0x100
DOMAIN_BOX, DOMAIN_SPHERE = 0, 1

RAY_OK, RAY_OUTSIDE, RAY_STEP_LIMIT, RAY_BAD_DIR = 0, 1, 2, 3


class Opts(ctypes.Structure):
    _fields_ = [("threads", c_int32), ("round_sites", c_int32), ("reorder", c_int32),
                ("blocks_per_site", c_double), ("max_steps", c_int64), ("host_only", c_int32),
                ("gpu_build", c_int32), ("zero_run_max", c_int32), ("domain", c_int32),
                ("sphere", c_double * 4)]


class Stats(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in ("rays", "crossings", "decisions", "rechecks", "fallbacks", "zero_steps",
                                       "step_limit", "outside")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("M", c_int64), ("nnz", c_int64), ("block_entries", c_int64), ("block_dim", c_int32 * 3),
                ("box", c_double * 6), ("build_seconds", c_double), ("device_bytes", c_int64),
                ("host_fallback_cells", c_int64), ("phase_seconds", c_double * 6), ("rel_bytes", c_int64)]


class Launch(ctypes.Structure):
    _fields_ = [("lanes_per_ray", c_int32), ("block", c_int32), ("blocks_per_sm", c_int32),
                ("fp64_lanes_per_ray", c_int32), ("order", c_int32)]


class Rayset(ctypes.Structure):
    _fields_ = [("grid", c_void_p), ("origin", c_void_p), ("dir", c_void_p), ("n", c_int64), ("tau", c_void_p),
                ("status", c_void_p)]


class VGridError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vgrid error {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("vgrid_last_error", ctypes.c_char_p, []),
    ("vgrid_default_opts", None, [ctypes.POINTER(Opts)]),
    ("vgrid_create", c_int32, [c_void_p, c_int64, c_void_p, ctypes.POINTER(Opts), ctypes.POINTER(c_void_p)]),
    ("vgrid_destroy", c_int32, [c_void_p]),
    ("vgrid_info", c_int32, [c_void_p, ctypes.POINTER(Info)]),
    ("vgrid_get_neighbors", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("vgrid_get_cells", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("vgrid_set_density", c_int32, [c_void_p, c_void_p, c_float, c_void_p]),
    ("vgrid_locate", c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    ("vgrid_trace", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_int64, c_void_p, ctypes.POINTER(Stats), c_void_p]),
    ("vgrid_kernel_launches", c_int64, []),
    ("vgrid_trace_host", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int64,
                                   c_void_p, c_void_p]),
    ("vgrid_trace_grad", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    ("vgrid_segments_grad", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_float, c_void_p,
                                      c_void_p]),
    ("vgrid_set_launch", c_int32, [c_void_p, ctypes.POINTER(Launch)]),
    ("vgrid_get_launch", c_int32, [c_void_p, ctypes.POINTER(Launch)]),
    ("vgrid_batch_create", c_int32, [ctypes.POINTER(Rayset), c_int32, ctypes.POINTER(Launch),
                                     ctypes.POINTER(c_void_p)]),
    ("vgrid_batch_run", c_int32, [c_void_p, c_int32, ctypes.POINTER(Stats), c_void_p]),
    ("vgrid_batch_destroy", c_int32, [c_void_p]),
    ("vgrid_batch_set_launch", c_int32, [c_void_p, ctypes.POINTER(Launch)]),
    ("vgrid_batch_get_launch", c_int32, [c_void_p, ctypes.POINTER(Launch)]),
    ("vgrid_enable_timing", c_int32, [c_void_p, c_int32]),
    ("vgrid_read_timing", c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                    ctypes.POINTER(c_int64)]),
    ("vgrid_interact", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p]),
    ("vgrid_probe_l2", c_int32, [c_int64, c_int32, ctypes.POINTER(c_double), c_void_p]),
    ("vgrid_trace_noalloc", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_void_p]),
]

NOALLOC_MAX_RAYS = 1 << 18


def load():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise RuntimeError(f"libvgrid is not built ({LIB} missing); run __graft_entry__.build() or "
                               "python -m paper_1310_1854_gb300.build")
        lib = ctypes.CDLL(LIB)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(rc: int):
    if rc != OK:
        raise VGridError(rc, load().vgrid_last_error().decode(errors="replace"))
