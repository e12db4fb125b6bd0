"""Seeded small grids and rays for the GPU fuzz test, chosen to reach the
degenerate corners of the method: lattices (edges and vertices where four
or eight cells meet), coplanar sites (prism cells, rays along faces),
near-duplicate pairs (very thin cells), sites on the walls, boxes of large
aspect ratio away from the origin, and rays starting on sites, on walls and
along the axes. No arithmetic of the method lives here: only inputs.
"""
from __future__ import annotations

import numpy as np

import gen

KINDS = ("uniform", "lattice", "jitter", "coplanar", "pairs", "walls")


def _box(rng):
    lo = rng.uniform(-5.0, 5.0, 3)
    ext = rng.uniform(0.5, 1.0, 3) * np.array([1.0, 1.0, 1.0]) * 2.0 ** rng.integers(-2, 4, 3)
    lo = np.float32(lo).astype(np.float64)
    hi = np.float32(lo + ext).astype(np.float64)
    return np.concatenate([lo, hi])


def _sites(kind, rng, box):
    lo, hi = box[:3], box[3:]
    ext = hi - lo
    if kind == "uniform":
        S = lo + rng.random((int(rng.integers(2, 300)), 3)) * ext
    elif kind in ("lattice", "jitter"):
        n = int(rng.integers(2, 7))
        g = (np.arange(n) + 0.5) / n
        S = lo + np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * ext
        if kind == "jitter":
            S = S + rng.normal(0.0, float(rng.choice([1e-7, 1e-5, 1e-3])), S.shape) * ext
    elif kind == "coplanar":
        m = int(rng.integers(3, 120))
        S = lo + rng.random((m, 3)) * ext
        axis = int(rng.integers(0, 3))
        S[: m - min(3, m // 4), axis] = lo[axis] + 0.5 * ext[axis]   # most sites on one plane
    elif kind == "pairs":
        m = int(rng.integers(2, 150))
        S = lo + rng.random((m, 3)) * ext
        k = max(1, m // 5)
        d = rng.normal(size=(k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        S = np.concatenate([S, S[:k] + 1e-6 * np.linalg.norm(ext) * d])
    else:  # walls: some sites on the faces and corners of the box
        m = int(rng.integers(4, 150))
        S = lo + rng.random((m, 3)) * ext
        for i in range(m // 3):
            c = int(rng.integers(0, 3))
            S[i, c] = lo[c] if rng.random() < 0.5 else hi[c]
        S[0] = lo
        S[1] = hi
    S = np.clip(np.float32(S).astype(np.float64), lo, hi)
    # float32 rounding may push a coordinate past the box: keep it inside
    S = np.where(S < lo, lo, np.where(S > hi, hi, S))
    return np.unique(S, axis=0)


def _rays(S, box, rng, n):
    lo, hi = box[:3], box[3:]
    ext = hi - lo
    O = lo + rng.random((n, 3)) * ext
    kind = rng.integers(0, 10, n)
    at_site = kind == 0
    O[at_site] = S[rng.integers(0, len(S), at_site.sum())]
    on_wall = kind == 1
    c = rng.integers(0, 3, n)
    side = rng.random(n) < 0.5
    O[on_wall, c[on_wall]] = np.where(side[on_wall], lo[c[on_wall]], hi[c[on_wall]])
    D = rng.normal(size=(n, 3))
    axis = kind >= 8   # exactly along an axis
    D[axis] = 0.0
    D[axis, c[axis]] = np.where(side[axis], 1.0, -1.0)
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    return gen.Rays(O, D)


def case(i: int):
    """Fuzz case i: (kind, Grid, Rays)."""
    rng = gen.rng_for(gen.SEED_BASE + 9000 + i)
    kind = KINDS[i % len(KINDS)]
    box = _box(rng)
    S = _sites(kind, rng, box)
    rho = rng.uniform(0.1, 10.0, len(S)).astype(np.float32)
    # kappa travels through the C ABI as a float32: draw a float32 value
    kappa = float(np.float32(rng.uniform(0.5, 2.0)))
    return kind, gen.Grid(S, box, rho, kappa=kappa), _rays(S, box, rng, 300)
