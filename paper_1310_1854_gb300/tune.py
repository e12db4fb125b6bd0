"""Launch-shape autotuner for the traversal kernels (single grids and batches).

The shape that traces fastest depends on the GPU, the arithmetic form and
the workload (sites per grid, rays, mean path length): lanes per ray
(1, 2, 4, 8), threads per block, and persistent blocks per SM. The tuner
times each candidate shape with CUDA events on a seeded sample of the
caller's rays, keeps the fastest, and caches it per (GPU, form, size class)
in a JSON file so later runs skip the search.

Timing uses the library's own event record around the traversal launch
(vgrid_enable_timing / vgrid_read_timing), so only kernel time counts.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Iterable

DEFAULT_SPACE = tuple((l, b, 0) for l in (1, 2, 4) for b in (128, 256))
_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("VGRID_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "vgrid", "tune.json")


def shape_key(gpu: str, precision: str, sites: int, rays: int) -> str:
    """Size class: powers of two of the site and ray counts."""
    ls = int(round(math.log2(max(sites, 1))))
    lr = int(round(math.log2(max(rays, 1))))
    return f"{gpu}|{precision}|M2^{ls}|N2^{lr}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    with _lock:
        d = load_cache(path)
        d[key] = entry
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def search(space: Iterable[tuple[int, int, int]], time_fn: Callable[[tuple[int, int, int]], float],
           repeats: int = 3) -> tuple[tuple[int, int, int], dict]:
    """Best shape of `space` by the smallest median of `repeats` timings."""
    results = {}
    for shape in space:
        ts = sorted(time_fn(shape) for _ in range(repeats))
        results[shape] = ts[len(ts) // 2]
    best = min(results, key=results.get)
    return best, {f"{l},{b},{s}": t for (l, b, s), t in results.items()}


def autotune(grid, origin, direction, precision: str = "fp32", sample: int = 200_000, space=DEFAULT_SPACE,
             use_cache: bool = True, path: str | None = None) -> dict:
    """Pick and apply the fastest launch shape for tracing these rays
    through `grid`; returns {"lanes_per_ray", "block", "blocks_per_sm",
    "ms", "cached", "key"}."""
    import torch

    name = torch.cuda.get_device_name(grid.device).replace("|", "/")
    key = shape_key(name, precision, grid.M, origin.shape[0])
    if use_cache:
        hit = load_cache(path).get(key)
        if hit:
            cur = grid.get_launch()
            if precision == "fp64":
                grid.set_launch(cur["lanes_per_ray"], hit["block"], hit["blocks_per_sm"], hit["lanes_per_ray"],
                                cur["order"])
            else:
                grid.set_launch(hit["lanes_per_ray"], hit["block"], hit["blocks_per_sm"], cur["fp64_lanes_per_ray"],
                                cur["order"])
            return dict(hit, cached=True, key=key)
    n = min(sample, origin.shape[0])
    g = torch.Generator(device="cpu").manual_seed(1310_1854)
    sel = torch.randperm(origin.shape[0], generator=g)[:n].sort().values.to(origin.device)
    o = origin.index_select(0, sel).contiguous()
    d = direction.index_select(0, sel).contiguous()
    tau = torch.empty(n, dtype=torch.float64 if precision == "fp64" else torch.float32, device=origin.device)
    prev = grid.get_launch()
    fp64_lanes = prev["fp64_lanes_per_ray"]

    def time_fn(shape):
        if precision == "fp64":
            grid.set_launch(prev["lanes_per_ray"], shape[1], shape[2], shape[0], prev["order"])
        else:
            grid.set_launch(shape[0], shape[1], shape[2], fp64_lanes, prev["order"])
        grid.trace(o, d, precision=precision, out_tau=tau)  # warm
        grid.enable_timing(True)
        grid.read_timing()
        grid.trace(o, d, precision=precision, out_tau=tau)
        _, ms, launches = grid.read_timing()
        grid.enable_timing(False)
        return ms / max(launches, 1)

    try:
        best, table = search(space, time_fn)
    except Exception:
        grid.set_launch(prev["lanes_per_ray"], prev["block"], prev["blocks_per_sm"], fp64_lanes, prev["order"])
        raise
    time_fn(best)
    entry = {"lanes_per_ray": best[0], "block": best[1], "blocks_per_sm": best[2], "ms": table[f"{best[0]},{best[1]},{best[2]}"],
             "sample_rays": n, "table": table}
    if use_cache:
        store(key, entry, path)
    return dict(entry, cached=False, key=key)


# lanes per ray, threads per block, blocks per SM, ray order (-1: set after
# set in the caller's order, 1: all work items longest estimated path first)
BATCH_SPACE = tuple((l, b, 0, o) for l in (1, 2, 4) for b in (64, 128, 256) for o in (-1, 1))


def batch_key(gpu: str, G: int, sites: int, rays: int) -> str:
    ls = int(round(math.log2(max(sites, 1))))
    lr = int(round(math.log2(max(rays, 1))))
    return f"{gpu}|batch|G{G}|M2^{ls}|N2^{lr}"


def autotune_batch(batch, sample_rays: int = 4_000_000, space=BATCH_SPACE, use_cache: bool = True,
                   path: str | None = None, repeats: int = 3) -> dict:
    """Pick and apply the fastest launch shape (lanes per ray, block, blocks
    per SM, ray order) for a Batch: each candidate is timed with CUDA events
    over whole batch runs (start records and the persistent traversal) of a
    seeded sample of every set's rays (all rays when the batch has at most
    ``sample_rays``), the median of ``repeats`` runs; the best is cached per
    (GPU, size class) and applied to ``batch``. Results do not depend on the
    shape. Returns {"lanes_per_ray", "block", "blocks_per_sm", "order", "ms",
    "cached", "key", "sample_rays", "table"}."""
    import torch

    from . import Batch

    dev = batch.tau[0].device if batch.tau else torch.device("cuda")
    name = torch.cuda.get_device_name(dev).replace("|", "/")
    grids = {id(g): g for g, _, _ in batch.sets}
    key = batch_key(name, len(batch.sets), sum(g.M for g in grids.values()), batch.rays)
    if use_cache:
        hit = load_cache(path).get(key)
        if hit:
            batch.set_launch(hit["lanes_per_ray"], hit["block"], hit["blocks_per_sm"], hit["order"])
            return dict(hit, cached=True, key=key)
    total = batch.rays
    if total > sample_rays:
        frac = sample_rays / total
        gen_ = torch.Generator(device="cpu").manual_seed(1310_1854)
        sub = []
        for g, o, d in batch.sets:
            n = o.shape[0]
            k = max(1, int(round(n * frac))) if n else 0
            sel = torch.randperm(n, generator=gen_)[:k].sort().values.to(o.device)
            sub.append((g, o.index_select(0, sel).contiguous(), d.index_select(0, sel).contiguous()))
        probe = Batch(sub)
        n_sample = probe.rays
    else:
        probe = batch
        n_sample = total
    prev = batch.get_launch()
    stream = torch.cuda.current_stream(dev)

    def time_fn(shape):
        probe.set_launch(*shape)
        probe.run(stream=stream)  # warm
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        probe.run(stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    results = {}
    try:
        for shape in space:
            ts = sorted(time_fn(shape) for _ in range(repeats))
            results[shape] = ts[len(ts) // 2]
    except Exception:
        batch.set_launch(prev["lanes_per_ray"], prev["block"], prev["blocks_per_sm"], prev["order"])
        raise
    best = min(results, key=results.get)
    batch.set_launch(*best)
    entry = {"lanes_per_ray": best[0], "block": best[1], "blocks_per_sm": best[2], "order": best[3],
             "ms": results[best], "sample_rays": n_sample,
             "table": {",".join(str(v) for v in k): t for k, t in results.items()}}
    if use_cache:
        store(key, entry, path)
    return dict(entry, cached=False, key=key)
