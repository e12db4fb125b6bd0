"""CPU oracle for Voronoi-grid straight-path traversal.

TEST INFRASTRUCTURE. Plain FP64 code written from the paper (Camps, Baes &
Saftly 2013, Sect. 2). Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the GPU library never does.

The arithmetic lives in ``voronoi_oracle.c`` (compiled with contraction off so
results do not depend on the host's FMA support); this module only marshals
numpy arrays and adds the plain numpy parts:

* ``cells``    Voronoi cells by bisector clipping (Sect. 2.1, 2.3): neighbour
               lists with walls as -1..-6, volumes, bounding boxes.
* ``locate``   C(r) by brute-force nearest site (Sect. 2.3).
* ``trace``    the straight-path loop of Sect. 2.2 (Eq. 1-5).
* a spherical domain (``sphere=(cx, cy, cz, R)``, a ball inside the box;
  Sect. 2.2 notes the method carries over to other domain geometries):
  cells keep the box's neighbour lists, a point is inside when its squared
  distance to the centre is at most R^2, and the exit from the domain is the
  sphere's, from the current point at every step (wall id -7).
* ``tau_grad`` gradient of a loss of tau with respect to cell densities:
               tau_r = sum_c kappa rho_c l_rc is linear in rho, so
               d tau_r / d rho_c = kappa l_rc (the segment bookkeeping of
               Sect. 2.2).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voronoi_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

WALL_IDS = (-1, -2, -3, -4, -5, -6)   # x=xmin, x=xmax, y=ymin, y=ymax, z=zmin, z=zmax
TIE_REL = 1e-9                        # near-tie threshold on the decision margin
ZERO_RUN_MAX = 4                      # zero-length steps in a row before the epsilon nudge (R6)
STATUS = {0: "ok", 1: "outside", 2: "step_limit", 3: "capacity"}


def build(force: bool = False) -> str:
    """Compile the oracle's C source with gcc (no contraction, -O2, pthreads).
    ORACLE_LIB names an already built library instead (the tests' planted
    mistakes: a copy of the source with one change, built the same way)."""
    if os.environ.get("ORACLE_LIB"):
        return os.environ["ORACLE_LIB"]
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = compile_command(_SRC, tmp)
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def compile_command(src: str, out: str) -> list:
    return ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
            "-o", out, src, "-lm"]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_cells.argtypes = [P, i64, P, P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_cells.restype = ctypes.c_int
        lib.oracle_locate.argtypes = [P, i64, P, P, P, i64, P, ctypes.c_int]
        lib.oracle_locate.restype = None
        lib.oracle_trace.argtypes = [P, i64, P, P, P, P, P, ctypes.c_double, P, P, i64, i64, P, P, P, P, P, P,
                                     P, P, P, i64, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.oracle_trace.restype = None
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _threads(n):
    if n is not None:
        return int(n)
    return int(os.environ.get("ORACLE_THREADS", "0"))


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _sphere(sphere):
    if sphere is None:
        return None
    sph = _f64c(sphere).reshape(4)
    assert sph[3] > 0, "sphere radius must be positive"
    return sph


def default_eps(box) -> float:
    box = np.asarray(box, dtype=np.float64)
    return 1e-12 * float(np.linalg.norm(box[3:] - box[:3]))


@dataclasses.dataclass
class Cells:
    ids: np.ndarray       # (n,) site indices
    nbr: list             # list of int32 arrays (ascending ids, walls negative)
    area: list            # matching face areas
    vol: np.ndarray       # (n,) volumes
    bbox: np.ndarray      # (n, 6) xmin, ymin, zmin, xmax, ymax, zmax


def cells(sites, box, ids=None, brute=False, maxdeg=256, eps=None, area_tol=None, threads=None) -> Cells:
    """Voronoi cells of ``ids`` (default: all sites) clipped by the box."""
    lib = _load()
    S = _f64c(sites)
    box = _f64c(box)
    M = S.shape[0]
    ids = np.arange(M, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    n = ids.size
    eps = default_eps(box) if eps is None else float(eps)
    diag = float(np.linalg.norm(box[3:] - box[:3]))
    area_tol = (1e-20 * diag * diag) if area_tol is None else float(area_tol)
    nbr = np.zeros((n, maxdeg), np.int32)
    deg = np.zeros(n, np.int32)
    area = np.zeros((n, maxdeg), np.float64)
    vol = np.zeros(n, np.float64)
    bbox = np.zeros((n, 6), np.float64)
    err = np.zeros(n, np.int32)
    rc = lib.oracle_cells(_p(S), M, _p(box), _p(ids), n, int(bool(brute)), maxdeg, eps, area_tol, _p(nbr),
                          _p(deg), _p(area), _p(vol), _p(bbox), _p(err), _threads(threads))
    if rc != 0:
        bad = np.nonzero(err)[0]
        raise RuntimeError(f"oracle_cells failed for {bad.size} cells (first {ids[bad[:5]]}, codes {err[bad[:5]]})")
    return Cells(ids, [nbr[i, :deg[i]].copy() for i in range(n)], [area[i, :deg[i]].copy() for i in range(n)],
                 vol, bbox)


def csr(c: Cells, M: int):
    """CSR (off int64[M+1], idx int32) from cells computed for all M sites."""
    assert c.ids.size == M and np.array_equal(c.ids, np.arange(M))
    deg = np.array([a.size for a in c.nbr], np.int64)
    off = np.zeros(M + 1, np.int64)
    np.cumsum(deg, out=off[1:])
    idx = np.concatenate(c.nbr).astype(np.int32) if M else np.zeros(0, np.int32)
    return off, idx


def locate(sites, box, pts, threads=None, sphere=None) -> np.ndarray:
    """Nearest site per point (lowest index on exact ties); -1 outside the
    box (or outside the ball ``sphere``)."""
    lib = _load()
    S = _f64c(sites)
    box = _f64c(box)
    sph = _sphere(sphere)
    P = _f64c(pts).reshape(-1, 3)
    out = np.empty(P.shape[0], np.int64)
    lib.oracle_locate(_p(S), S.shape[0], _p(box), _p(sph), _p(P), P.shape[0], _p(out), _threads(threads))
    return out


@dataclasses.dataclass
class Trace:
    nseg: np.ndarray
    seg_cell: np.ndarray      # (N, cap) int32
    seg_len: np.ndarray       # (N, cap) float64
    tau: np.ndarray
    length: np.ndarray
    min_margin: np.ndarray
    near_tie: np.ndarray
    nfallback: np.ndarray
    status: np.ndarray

    def segments(self, i):
        n = int(self.nseg[i])
        return self.seg_cell[i, :n], self.seg_len[i, :n]


def trace(sites, box, rho, origin, direction, off=None, idx=None, kappa=1.0, cap=1024, max_steps=1_000_000,
          tie_rel=TIE_REL, zero_run_max=ZERO_RUN_MAX, threads=None, sphere=None) -> Trace:
    """Trace rays with the paper's loop. With off/idx None every site and all
    walls are candidates (the plain definition of the exit). More than
    ``zero_run_max`` zero-length steps in a row nudge the point by
    epsilon = 1e-12 |Dmax - Dmin| and locate it again (Sect. 2.2). With
    ``sphere`` the domain is that ball and its exit ends the path."""
    lib = _load()
    S = _f64c(sites)
    box = _f64c(box)
    sph = _sphere(sphere)
    rho = _f64c(rho)
    O = _f64c(origin).reshape(-1, 3)
    D = _f64c(direction).reshape(-1, 3)
    N = O.shape[0]
    if off is not None:
        off = np.ascontiguousarray(off, np.int64)
        idx = np.ascontiguousarray(idx, np.int32)
    cap = int(cap)
    seg_cell = np.zeros((N, max(cap, 1)), np.int32)
    seg_len = np.zeros((N, max(cap, 1)), np.float64)
    out = {k: np.zeros(N, t) for k, t in [("nseg", np.int32), ("tau", np.float64), ("length", np.float64),
                                         ("min_margin", np.float64), ("near_tie", np.int32),
                                         ("nfallback", np.int32), ("status", np.int32)]}
    lib.oracle_trace(_p(S), S.shape[0], _p(box), _p(sph), _p(off), _p(idx), _p(rho), float(kappa), _p(O), _p(D), N,
                     cap,
                     _p(seg_cell), _p(seg_len), _p(out["nseg"]), _p(out["tau"]), _p(out["length"]),
                     _p(out["min_margin"]), _p(out["near_tie"]), _p(out["nfallback"]), _p(out["status"]),
                     int(max_steps), int(zero_run_max), float(tie_rel), _threads(threads))
    return Trace(out["nseg"], seg_cell, seg_len, out["tau"], out["length"], out["min_margin"], out["near_tie"],
                 out["nfallback"], out["status"])


def tau_grad(tr: Trace, M: int, dL_dtau, kappa=1.0) -> np.ndarray:
    """dL/drho_c = sum_r dL/dtau_r * kappa * l_rc, summed in FP64."""
    dL = np.asarray(dL_dtau, np.float64)
    N = tr.nseg.size
    cap = tr.seg_cell.shape[1]
    mask = np.arange(cap)[None, :] < tr.nseg[:, None]
    cells_ = tr.seg_cell[mask]
    w = (dL[:, None] * kappa * tr.seg_len)[mask]
    assert cells_.size == int(tr.nseg.sum()), "segment capacity exceeded"
    return np.bincount(cells_, weights=w, minlength=M)[:M] if N else np.zeros(M)


def enter_points(box, origin, direction, sphere=None):
    """For rays that start outside the closed box, the first point of the ray
    r0 + s k (s >= 0) inside it: the largest of the per-axis entry parameters
    of the slabs, if it does not exceed the smallest exit parameter. Rays
    inside are returned unchanged; rays that miss keep their origin.

    With ``sphere`` (a ball inside the box): a ray outside the ball that
    meets it ahead starts epsilon = 1e-12 |Dmax - Dmin| past its entry point,
    the smaller root of |r0 + s k - c|^2 = R^2 (written as q / (sqrt(b^2 - q)
    - b), b = k.(r0 - c) < 0, q = |r0 - c|^2 - R^2 > 0, so that no digits
    cancel), where it is inside the ball unless it only grazes it."""
    box = np.asarray(box, np.float64)
    O = np.array(origin, np.float64).reshape(-1, 3)
    D = np.asarray(direction, np.float64).reshape(-1, 3)
    out = O.copy()
    if sphere is not None:
        sph = _sphere(sphere)
        eps = default_eps(box)
        for i in range(O.shape[0]):
            r, k = O[i], D[i]
            o = r - sph[:3]
            q = ((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]) - sph[3] * sph[3]
            if q <= 0.0:
                continue
            b = (k[0] * o[0] + k[1] * o[1]) + k[2] * o[2]
            disc = b * b - q
            if not (b < 0.0 and disc >= 0.0):
                continue
            t = q / (np.sqrt(disc) - b) + eps
            out[i] = r + t * k
        return out
    for i in range(O.shape[0]):
        r, k = O[i], D[i]
        if np.all((r >= box[:3]) & (r <= box[3:])):
            continue
        t_in, t_out, miss = -np.inf, np.inf, False
        for c in range(3):
            if k[c] != 0.0:
                t1 = (box[c] - r[c]) / k[c]
                t2 = (box[3 + c] - r[c]) / k[c]
                t_in = max(t_in, min(t1, t2))
                t_out = min(t_out, max(t1, t2))
            elif r[c] < box[c] or r[c] > box[3 + c]:
                miss = True
        if not miss and t_in <= t_out and t_out >= 0.0:
            t = max(t_in, 0.0)
            out[i] = np.minimum(np.maximum(r + t * k, box[:3]), box[3:])
    return out


def interact(tr: Trace, rho, tau_int, weight=None, kappa=1.0):
    """Interaction point of each traced ray: the cell where the running
    tau = sum kappa rho l first reaches tau_int, the distance to it, and the
    part w (exp(-tau_in) - exp(-tau_out)) of the package each cell removes
    (tau capped at tau_int). Plain loop over the oracle's segments, FP64.
    Returns (cell [-1: leaves first], s, absorbed per cell, ambiguous) where
    ambiguous marks rays whose tau_int lies within 1e-4 relative of a cell
    boundary's running tau (the cell is then decided by rounding)."""
    rho = np.asarray(rho, np.float64)
    ti = np.asarray(tau_int, np.float64)
    w = np.ones_like(ti) if weight is None else np.asarray(weight, np.float64)
    N = tr.nseg.size
    cell = np.full(N, -1, np.int64)
    s = np.zeros(N)
    amb = np.zeros(N, bool)
    absorbed = np.zeros(rho.size)
    for i in range(N):
        cells, lens = tr.segments(i)
        tau = 0.0
        dist = 0.0
        for c, l in zip(cells, lens):
            k = kappa * rho[c]
            d = k * l
            if abs(tau + d - ti[i]) <= 1e-4 * ti[i] or abs(tau - ti[i]) <= 1e-4 * ti[i]:
                amb[i] = True
            if tau + d >= ti[i]:
                part = ti[i] - tau
                absorbed[c] += w[i] * (np.exp(-tau) - np.exp(-ti[i]))
                cell[i] = c
                s[i] = dist + (part / k if k > 0 else 0.0)
                break
            absorbed[c] += w[i] * (np.exp(-tau) - np.exp(-(tau + d)))
            tau += d
            dist += l
        else:
            s[i] = dist
    return cell, s, absorbed, amb


def exp_loss(tau, target):
    """Loss sum_r (exp(-tau_r) - target_r)^2 and dL/dtau_r."""
    e = np.exp(-np.asarray(tau, np.float64))
    t = np.asarray(target, np.float64)
    return float(np.sum((e - t) ** 2)), -2.0 * (e - t) * e
