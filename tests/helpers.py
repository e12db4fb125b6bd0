"""Independent reference computations used to pin the oracle.

Nothing here shares code with the oracle or with the GPU library: these are
textbook routines (ray-box slab distance, 3-D DDA voxel walk, brute-force
nearest site in numpy) used as checks.
"""
import numpy as np


def slab_length(box, origin, direction):
    """Distance from each origin to the boundary of the box along its
    direction: the smallest of the per-axis slab exits (ray-box test)."""
    box = np.asarray(box, np.float64)
    O = np.asarray(origin, np.float64).reshape(-1, 3)
    D = np.asarray(direction, np.float64).reshape(-1, 3)
    out = np.full(O.shape[0], np.inf)
    for a in range(3):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(D[:, a] > 0, (box[3 + a] - O[:, a]) / D[:, a],
                         np.where(D[:, a] < 0, (box[a] - O[:, a]) / D[:, a], np.inf))
        out = np.minimum(out, t)
    return out


def nearest_site(sites, pts, chunk=4096):
    """Index of the nearest site for each point (numpy brute force)."""
    S = np.asarray(sites, np.float64)
    P = np.asarray(pts, np.float64).reshape(-1, 3)
    out = np.empty(P.shape[0], np.int64)
    s2 = (S * S).sum(1)
    for i in range(0, P.shape[0], chunk):
        q = P[i:i + chunk]
        d2 = ((q[:, None, :] - S[None, :, :]) ** 2).sum(-1)
        out[i:i + chunk] = d2.argmin(1)
    return out


def dda_voxels(box, n, origin, direction):
    """Amanatides-Woo walk through an n^3 voxel grid filling box.

    Returns a list of (voxel (i, j, k), length) along the ray until it leaves
    the box. The voxel containing the origin is found by flooring.
    """
    box = np.asarray(box, np.float64)
    lo, hi = box[:3], box[3:]
    h = (hi - lo) / n
    o = np.asarray(origin, np.float64)
    d = np.asarray(direction, np.float64)
    v = np.minimum(np.floor((o - lo) / h).astype(int), n - 1)
    t_next = np.empty(3)
    t_delta = np.empty(3)
    step = np.zeros(3, int)
    for a in range(3):
        if d[a] > 0:
            step[a] = 1
            t_next[a] = (lo[a] + (v[a] + 1) * h[a] - o[a]) / d[a]
            t_delta[a] = h[a] / d[a]
        elif d[a] < 0:
            step[a] = -1
            t_next[a] = (lo[a] + v[a] * h[a] - o[a]) / d[a]
            t_delta[a] = -h[a] / d[a]
        else:
            t_next[a] = np.inf
            t_delta[a] = np.inf
    t = 0.0
    out = []
    while True:
        a = int(np.argmin(t_next))
        out.append((tuple(v.tolist()), t_next[a] - t))
        t = t_next[a]
        v[a] += step[a]
        if v[a] < 0 or v[a] >= n:
            return out
        t_next[a] += t_delta[a]
