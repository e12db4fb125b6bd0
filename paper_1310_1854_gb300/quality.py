"""Grid-quality measure of Table 1: the standard deviation of the difference
between the model's density rho_t and the gridded density rho_g at random
points spread uniformly over the domain (Sect. 3.3). rho_g at a point is the
density of the cell containing it, found with C(r) on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch


def sample_points(box, n: int, seed: int) -> np.ndarray:
    box = np.asarray(box, np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    return box[:3] + (box[3:] - box[:3]) * rng.random((n, 3))


def grid_quality(grid, rho_cell, rho_true, n_points: int = 1_000_000, seed: int = 1310_1854,
                 precision: str = "fp32", chunk: int = 4_000_000) -> dict:
    """std(rho_t - rho_g) over n_points uniform points of the grid's box.

    rho_cell: per-cell density (caller order, length M); rho_true: callable
    mapping an (n, 3) float64 array of points to their model density.
    """
    rho_cell = np.asarray(rho_cell, np.float64)
    pts = sample_points(grid.box, n_points, seed)
    diffs = np.empty(n_points)
    for a in range(0, n_points, chunk):
        p = pts[a:a + chunk]
        cell = grid.locate(torch.from_numpy(np.ascontiguousarray(p)).to(grid.device), precision=precision)
        cell = cell.cpu().numpy()
        if np.any(cell < 0):
            raise RuntimeError("a sample point fell outside the grid's box")
        diffs[a:a + chunk] = np.asarray(rho_true(p), np.float64) - rho_cell[cell]
    return {"std": float(diffs.std()), "mean": float(diffs.mean()), "points": n_points}
