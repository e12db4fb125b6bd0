"""Grid-quality measure of Table 1: the standard deviation of the difference
between the model's density rho_t and the gridded density rho_g at random
points spread uniformly over the domain (Sect. 3.3). rho_g at a point is the
density of the cell containing it, found with C(r) on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch


def sample_points(box, n: int, seed: int, sphere=None) -> np.ndarray:
    """n uniform points of the domain: the box, or the ball sphere = (cx, cy,
    cz, R) (rejection from its bounding cube; a point is in the ball when
    ((dx dx + dy dy) + dz dz) <= R R, the domain's own test)."""
    box = np.asarray(box, np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    if sphere is None:
        return box[:3] + (box[3:] - box[:3]) * rng.random((n, 3))
    c = np.asarray(sphere, np.float64).reshape(4)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        q = c[:3] + c[3] * (2.0 * rng.random((2 * (n - out.shape[0]) + 16, 3)) - 1.0)
        d = q - c[:3]
        out = np.concatenate([out, q[(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= c[3] * c[3]]])
    return out[:n]


def grid_quality(grid, rho_cell, rho_true, n_points: int = 1_000_000, seed: int = 1310_1854,
                 precision: str = "fp32", chunk: int = 4_000_000) -> dict:
    """std(rho_t - rho_g) over n_points uniform points of the grid's domain
    (its box, or its ball for a spherical domain).

    rho_cell: per-cell density (caller order, length M); rho_true: callable
    mapping an (n, 3) float64 array of points to their model density.
    """
    rho_cell = np.asarray(rho_cell, np.float64)
    pts = sample_points(grid.box, n_points, seed, getattr(grid, "sphere", None))
    diffs = np.empty(n_points)
    for a in range(0, n_points, chunk):
        p = pts[a:a + chunk]
        cell = grid.locate(torch.from_numpy(np.ascontiguousarray(p)).to(grid.device), precision=precision)
        cell = cell.cpu().numpy()
        if np.any(cell < 0):
            raise RuntimeError("a sample point fell outside the grid's domain")
        diffs[a:a + chunk] = np.asarray(rho_true(p), np.float64) - rho_cell[cell]
    return {"std": float(diffs.std()), "mean": float(diffs.mean()), "points": n_points}
