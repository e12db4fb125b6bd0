"""The N > 1 path on CPU: two gloo ranks shard the rays, trace their shard
with the oracle (standing in for one GPU each), and combine counts, the
max-over-ranks time and the density gradient the way bench.py and
paper_1310_1854_gb300.shard do on GPUs. No GPU is touched."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import gen
import oracle
from paper_1310_1854_gb300.shard import allreduce_sum_, max_over_ranks, shard_range, sum_over_ranks


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 1001):
        for w in (1, 2, 3, 8):
            parts = [shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, rays = gen.config1(400)
        c = oracle.cells(g.sites, g.box, threads=1)
        off, idx = oracle.csr(c, len(g.sites))
        a, b = shard_range(len(rays.origin), rank, world)
        tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin[a:b], rays.dir[a:b], off=off,
                          idx=idx, threads=1)
        segs = sum_over_ranks(float(tr.nseg.sum()))
        tmax = max_over_ranks(float(rank + 1))
        _, dL = oracle.exp_loss(tr.tau, np.exp(-0.5 * tr.tau))
        grad = torch.from_numpy(oracle.tau_grad(tr, len(g.sites), dL))
        allreduce_sum_(grad)
        out[rank] = (segs, tmax, grad.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    g, rays = gen.config1(400)
    c = oracle.cells(g.sites, g.box)
    off, idx = oracle.csr(c, len(g.sites))
    tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin, rays.dir, off=off, idx=idx)
    _, dL = oracle.exp_loss(tr.tau, np.exp(-0.5 * tr.tau))
    full = oracle.tau_grad(tr, len(g.sites), dL)
    for r in range(world):
        segs, tmax, grad = out[r]
        assert segs == tr.nseg.sum()
        assert tmax == world
        np.testing.assert_allclose(grad, full, rtol=1e-12, atol=1e-15)


def _bench(*args, env=None):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    e = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        e.pop(k, None)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                          env=e, timeout=600)


def test_bench_gpus_flag_starts_the_ranks():
    """`bench.py --gpus 2` outside torchrun starts two ranks itself (under
    torch.distributed.run, rendezvous on 127.0.0.1); --dry-run runs their
    bookkeeping with gloo on the CPU: rank 0 alone prints one line that
    reports both ranks and sums their own rays."""
    import json
    p = _bench("--gpus", "2", "--dry-run", "--rays", "3000")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["gpus_requested"] == 2 and d["rays_all"] == 6000
    import bench
    want = sum(float(np.abs(gen.disk_rays(3000, bench.rank_rays_seed(r)).origin).sum()) for r in range(2))
    assert d["origin_abs_sum"] == pytest.approx(want, rel=1e-12)


def test_bench_refuses_a_world_size_that_differs_from_gpus():
    p = _bench("--gpus", "2", "--dry-run", env={"WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"})
    assert p.returncode != 0 and "WORLD_SIZE=1" in p.stderr


def test_assign_sets_balances_the_batch():
    from paper_1310_1854_gb300.shard import assign_sets, estimated_crossings
    plan = gen.config4_plan()
    w = [estimated_crossings(n, m) for _, m, n in plan]
    for world in (1, 2, 3, 4, 8):
        a = assign_sets(w, world)
        assert len(a) == len(w) and set(a) <= set(range(world))
        load = np.bincount(a, weights=w, minlength=world)
        # greedy largest-first: within 4/3 of the optimum, and no worse than
        # the mean plus the largest single set
        lower = max(sum(w) / world, max(w))
        assert load.max() <= 4.0 / 3.0 * lower + 1e-9
        assert load.max() <= sum(w) / world + max(w) + 1e-9
        assert a == assign_sets(w, world)  # the same on every rank
    assert assign_sets([], 4) == []
    with pytest.raises(ValueError):
        assign_sets([1.0], 0)
    with pytest.raises(ValueError):
        assign_sets([-1.0], 2)


def _batch_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1310_1854_gb300.shard import assign_sets, estimated_crossings, sum_over_ranks
        sets = gen.config4(G=6, scale=0.01)
        a = assign_sets([estimated_crossings(len(r.origin), len(g.sites)) for g, r in sets], world)
        segs = 0.0
        for k, (g, r) in enumerate(sets):
            if a[k] != rank:
                continue
            c = oracle.cells(g.sites, g.box, threads=1)
            off, idx = oracle.csr(c, len(g.sites))
            tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), r.origin, r.dir, off=off, idx=idx, threads=1)
            segs += float(tr.nseg.sum())
        out[rank] = (sum_over_ranks(segs), a)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_a_batch_by_grid():
    """A batch split by whole grids over two gloo ranks (oracle standing in
    for the GPUs): both ranks compute the same assignment, and the summed
    crossings equal those of one process tracing every grid."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_batch_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    total = 0
    for g, r in gen.config4(G=6, scale=0.01):
        c = oracle.cells(g.sites, g.box)
        off, idx = oracle.csr(c, len(g.sites))
        total += int(oracle.trace(g.sites, g.box, g.rho.astype(np.float64), r.origin, r.dir, off=off, idx=idx).nseg.sum())
    assert out[0][1] == out[1][1] and set(out[0][1]) == {0, 1}
    assert out[0][0] == out[1][0] == total
