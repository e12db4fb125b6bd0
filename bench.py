"""Benchmark: Voronoi path segments per second on one GB300.

Workload (N = 1): a 10^5-site exponential-disk grid (sites drawn from
rho ~ exp(-R - |z|/0.1) in [-4,4]^2 x [-0.5,0.5], cell density = that rho)
and 10^6 rays per GPU from the same distribution with isotropic directions.
One step = start-cell location plus the traversal of every ray to the domain
boundary, computing tau per ray, float32 plane tests with float64 rechecks.
The float64 form runs on the same rays for comparison.

The line also carries: the roofline of the traversal kernel against read
ceilings of L2 measured in this process (the grid's cell blocks stay in L2),
the CPU oracle timed on the host with the accuracy of both forms against it,
and summaries of the other workloads (10^6 clumpy sites with 10^7 rays, 64
uneven grids in one autotuned batch launch, the adjoint on the 10^6-site
disk).

With torchrun (N > 1) every rank traces its own 10^6 rays through a copy of
the grid (weak scaling, no collective on the data path); the time is the
maximum over ranks. `--gpus N` without torchrun starts N ranks under
torch.distributed.run itself. `--dry-run` runs the rank bookkeeping of that
path on the CPU with the gloo backend (no GPU, no timing).

--impl reference times the CPU oracle (plain float64 C, the paper's loop over
neighbour lists) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import socket
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Voronoi path segments/sec on 1 GB300 (FP32+recheck vs FP64) at ≤1e-5 rel tau err"
UNIT = "segments/s"
WORKLOAD = "exp-disk 1e5 sites, 1e6 rays/GPU, tau per ray, fp32 plane tests + fp64 recheck"
L2_BYTES = 129 * 2 ** 20
TAU32_REL = 1e-5


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the traversal kernel: trace.cuh, the
    descriptors in internal.h and fsplit.h, and the kernel's argument struct
    in kernels.h (a committed ncu summary carries it, so a figure taken from
    an older kernel is not used)."""
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1310_1854_gb300", "csrc")
    for f in ("trace.cuh", "internal.h", "fsplit.h"):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    k = open(os.path.join(src, "kernels.h")).read()
    i = k.index("struct TraceArgs")
    h.update(k[i:k.index("};", i)].encode())
    return h.hexdigest()[:16]


def profiled(name, key):
    """A per-launch figure from a committed ncu summary, if it was taken from
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt)
    t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", txt)
    if m and t and m.group(1) == kernel_source_hash():
        return float(t.group(1))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        load = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_launches():
    """Kernels the library has launched in this process (its own counter)."""
    from paper_1310_1854_gb300 import _lib
    return int(_lib.load().vgrid_kernel_launches())


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts) and parts[local_rank].strip().isdigit():
            return int(parts[local_rank])
    return local_rank


def rank_rays_seed(rank):
    """Seed of one rank's rays: every rank traces its own 10^6 rays."""
    import gen
    return gen.SEED_BASE + 2 + 1000 + 7919 * rank


# ---------------------------------------------------------------------------
# several ranks: start them under torch.distributed.run when not started so
# ---------------------------------------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def relaunch(n, argv):
    """Run this script as n ranks under torch.distributed.run (one node,
    rendezvous on 127.0.0.1) with the same arguments; rank 0 prints the line.
    Returns the launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def run_dry(args):
    """The multi-rank path without a GPU: gloo process group, each rank's own
    rays, a barrier, and the reductions that form the line (max of the times,
    sums of rays and crossings) -- the bookkeeping of the GPU leg with the
    traversal left out."""
    import torch
    import torch.distributed as tdist

    import gen
    ws, rank, _ = dist_info()
    if ws > 1:
        tdist.init_process_group("gloo")
    rays = gen.disk_rays(args.rays, rank_rays_seed(rank))
    if ws > 1:
        tdist.barrier()
    t0 = time.perf_counter()
    checksum = float(np.abs(rays.origin).sum())
    dt = time.perf_counter() - t0

    def red(x, op):
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        tdist.all_reduce(t, op=op)
        return float(t.item())

    seconds_max = red(dt, tdist.ReduceOp.MAX if ws > 1 else None)
    rays_all = red(float(len(rays.origin)), tdist.ReduceOp.SUM if ws > 1 else None)
    checks = red(checksum, tdist.ReduceOp.SUM if ws > 1 else None)
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": ws, "gpus_requested": args.gpus, "rays_per_rank": args.rays,
                          "rays_all": rays_all, "seconds_max": seconds_max, "origin_abs_sum": checks,
                          "scaling": "weak"}), flush=True)
    if ws > 1:
        tdist.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU oracle leg (rank 0, N = 1; and the --impl reference arm)
# ---------------------------------------------------------------------------

def oracle_setup(g):
    import oracle
    oracle.build()
    t = time.time()
    c = oracle.cells(g.sites, g.box, maxdeg=96)
    off, idx = oracle.csr(c, len(g.sites))
    return off, idx, time.time() - t


def oracle_sample(g, rays, off, idx, n, seed):
    import oracle
    sel = np.sort(np.random.default_rng(seed).choice(len(rays.origin), n, replace=False))
    t = time.time()
    tr = oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin[sel], rays.dir[sel], off=off, idx=idx,
                      cap=1)
    dt = time.time() - t
    return tr, sel, dt


def oracle_threads():
    n = int(os.environ.get("ORACLE_THREADS", "0"))
    return n if n > 0 else (os.cpu_count() or 1)


def _rel_stats(x):
    if x.size == 0:
        return None
    return {"max": float(x.max()), "p99": float(np.quantile(x, 0.99)), "mean": float(x.mean())}


def cpu_baseline(g, rays, tau32, tau64, target_s=10.0, tau32x=None):
    """The oracle timed on a bounded seeded sample of the workload's rays
    (about target_s of CPU time, all rays if they fit), and the tau of the
    GPU forms on those rays against the oracle's."""
    off, idx, setup_s = oracle_setup(g)
    n = 2000
    tr, sel, dt = oracle_sample(g, rays, off, idx, n, 1)
    if dt < target_s:
        n = int(min(len(rays.origin), max(n, n * target_s / max(dt, 1e-3))))
        tr, sel, dt = oracle_sample(g, rays, off, idx, n, 2)
    segs = int(tr.nseg.sum())
    base = {"value": segs / dt, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "sample": f"{n} of the {len(rays.origin)} rays (seeded), neighbour-list traversal with "
                      f"brute-force C(r0), float64; cell construction ({setup_s:.1f} s) not timed",
            "seconds": dt, "segments": segs}
    # status 3 (capacity) only says that the timing run kept one segment per
    # ray; its tau is complete
    ok = (tr.near_tie == 0) & np.isin(tr.status, (0, 3)) & (tr.tau > 0)
    t32 = tau32[sel].astype(np.float64)
    t64 = tau64[sel]
    rel32 = np.abs(t32 - tr.tau) / np.maximum(tr.tau, 1e-300)
    rel64 = np.abs(t64 - tr.tau) / np.maximum(tr.tau, 1e-300)
    pos = tr.tau > 0
    acc = {"reference": "CPU oracle, float64, neighbour lists from its own bisector clipping",
           "rays_compared": int(n), "near_tie_fraction": float(1.0 - ok.mean()),
           "fp32_tau_rel_err": _rel_stats(rel32[ok]), "fp64_tau_rel_err": _rel_stats(rel64[ok]),
           "fp32_tau_rel_err_incl_near_ties": _rel_stats(rel32[pos]),
           "fp32_rays_over_1e-5": int((rel32[ok] > TAU32_REL).sum()),
           "oracle_fallbacks": int(tr.nfallback.sum())}
    if tau32x is not None:
        relx = np.abs(tau32x[sel].astype(np.float64) - tr.tau) / np.maximum(tr.tau, 1e-300)
        acc["fp32_exact_tau_rel_err"] = _rel_stats(relx[ok])
    return base, acc


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import gen
    g, rays = gen.config2()
    off, idx, setup_s = oracle_setup(g)
    n = 20000
    for _ in range(args.warmup):
        oracle_sample(g, rays, off, idx, 2000, 0)
    segs_total, secs = 0, 0.0
    for k in range(args.steps):
        tr, _, dt = oracle_sample(g, rays, off, idx, n, 100 + k)
        segs_total += int(tr.nseg.sum())
        secs += dt
    v = segs_total / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sites": len(g.sites), "rays": len(rays.origin)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                             "sample": f"{n} seeded rays per step of the {len(rays.origin)}; neighbour lists built "
                                       f"by the oracle before timing ({setup_s:.1f} s)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# roofline
# ---------------------------------------------------------------------------

def l2_ceilings(nbytes):
    """Read ceilings of L2 for a buffer the size of the grid's cell blocks:
    256-bit streaming reads and the dependent chase over 288-byte blocks."""
    from paper_1310_1854_gb300 import probe_l2
    nbytes = int(max(nbytes, 1 << 20))
    return {"stream_gbs": probe_l2(nbytes, "stream"), "chase_gbs": probe_l2(nbytes, "chase"), "bytes": nbytes}


def roofline(crossings, bytes_per_crossing, kernel_ms, rel_bytes, ceil, traffic=None, kernel="trace_kernel"):
    """Roofline entry of a traversal launch: algorithmic bytes per launch over
    its CUDA-event time, against the level that serves its cell blocks (L2
    when they fit in half of it, else HBM), with the other ceilings beside."""
    hbm, hbm_kind = measured_peaks()
    achieved = crossings * bytes_per_crossing / (kernel_ms / 1e3) / 1e9
    r = {"achieved": achieved, "unit": "GB/s", "traffic": traffic, "kernel": kernel,
         "algorithmic_bytes_per_crossing": bytes_per_crossing, "crossings_per_launch": crossings,
         "kernel_ms_per_launch": kernel_ms, "cell_block_bytes": rel_bytes,
         "hbm_peak": hbm, "frac_of_hbm": achieved / hbm,
         "hbm_peak_source": f"{hbm_kind} hbm_gbs (MEASURED_PEAKS.json)"}
    if ceil is not None:
        r.update({"l2_stream_peak": ceil["stream_gbs"], "frac_of_l2_stream": achieved / ceil["stream_gbs"],
                  "l2_chase_ceiling": ceil["chase_gbs"], "frac_of_l2_chase": achieved / ceil["chase_gbs"],
                  "l2_source": f"measured in this process (vgrid_probe_l2) on a {ceil['bytes'] / 1e6:.0f} MB "
                               "buffer held in L2: 256-bit streaming reads (stream) and a dependent chase over "
                               "288-byte blocks at random positions (chase)"})
    if rel_bytes <= 0.5 * L2_BYTES and ceil is not None:
        r.update({"bound": "l2", "peak": ceil["stream_gbs"], "frac": achieved / ceil["stream_gbs"]})
    else:
        r.update({"bound": "hbm", "peak": hbm, "frac": achieved / hbm})
    return r


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lanes", type=int, default=int(os.environ.get("VGRID_LANES", "0")))
    ap.add_argument("--block", type=int, default=int(os.environ.get("VGRID_BLOCK", "0")))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="leave out the summaries of the other workloads")
    ap.add_argument("--dry-run", action="store_true", help="multi-rank bookkeeping on the CPU (gloo), no GPU")
    ap.add_argument("--rays", type=int, default=1_000_000)
    ap.add_argument("--workload", default="disk1e5", choices=["disk1e5", "clumpy1e6", "batched64", "grad1e6", "segments1e5", "next"],
                    help="disk1e5 is the benchmark line; the others measure the remaining workloads")
    args = ap.parse_args()
    if args.gpus < 1:
        ap.error("--gpus must be at least 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # one process per GPU: start them, each reads its rank from the env
        sys.exit(relaunch(args.gpus, sys.argv[1:]))
    ws, rank, _ = dist_info()
    if ws != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={ws}")
    if args.dry_run:
        return run_dry(args)
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)
    if args.workload != "disk1e5":
        if ws > 1:
            sys.exit("bench.py: --workload other than disk1e5 runs on one GPU")
        return run_extra(args)

    import torch
    import torch.distributed as tdist

    import gen
    from paper_1310_1854_gb300 import VoronoiGrid

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    g, _ = gen.config2(n_rays=1)
    rays = gen.disk_rays(args.rays, rank_rays_seed(rank))
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    if args.lanes or args.block:
        cur = vg.get_launch()
        vg.set_launch(args.lanes or cur["lanes_per_ray"], args.block or cur["block"])
    launch = vg.get_launch()
    info = vg.info()
    O = torch.from_numpy(rays.origin).to(dev)
    D = torch.from_numpy(rays.dir).to(dev)
    N = O.shape[0]
    tau = torch.empty(N, dtype=torch.float32, device=dev)
    tau64 = torch.empty(N, dtype=torch.float64, device=dev)

    st32 = vg.trace(O, D, precision="fp32", stats=True).stats
    st64 = vg.trace(O, D, precision="fp64", stats=True).stats
    crossings = st32["crossings"]
    assert st64["crossings"] == crossings or abs(st64["crossings"] - crossings) <= 1e-6 * crossings

    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    ceil = l2_ceilings(info["rel_bytes"])

    def timed(precision, out, steps, warm):
        for _ in range(warm):
            vg.trace(O, D, precision=precision, out_tau=out)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        vg.enable_timing(True)
        vg.read_timing()
        if ws > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        n0 = kernel_launches()
        for k in range(steps):
            flush.zero_()                      # L2 flushed between steps
            ev[k][0].record()
            vg.trace(O, D, precision=precision, out_tau=out)
            ev[k][1].record()
        torch.cuda.synchronize()
        if ws > 1:
            tdist.barrier()
        step_ms = sum(a.elapsed_time(b) for a, b in ev)
        loc_ms, tr_ms, launches = vg.read_timing()
        vg.enable_timing(False)
        timed.kernels = kernel_launches() - n0
        return step_ms, loc_ms, tr_ms, launches

    sampler = ClockSampler(gpu_index(local))
    sampler.start()
    step_ms, loc_ms, tr_ms, launches = timed("fp32", tau, args.steps, args.warmup)
    clocks = sampler.stop()
    gpu_launches = timed.kernels
    k64 = max(3, args.steps // 4)
    step64_ms, _, tr64_ms, launches64 = timed("fp64", tau64, k64, 2)
    # the float32 form with exact lengths (same decisions, float-pair lengths)
    tau32x = torch.empty(N, dtype=torch.float32, device=dev)
    kx = max(3, args.steps // 2)
    stepx_ms, _, trx_ms, launchesx = timed("fp32_exact", tau32x, kx, 2)

    # accuracy of the float32 form against the float64 form on these rays
    t32 = tau.double()
    rel = ((t32 - tau64).abs() / tau64.clamp_min(1e-300))[tau64 > 0]
    tau_err = {"max": float(rel.max()), "p99": float(torch.quantile(rel[:1_000_000].float(), 0.99)),
               "mean": float(rel.mean())}

    # end to end through the public call for host-resident rays
    # (vgrid_trace_host): pinned host origins and directions in, tau out to
    # pinned host memory, every step; consecutive calls overlap the next
    # step's copy in with this step's traversal. L2 is flushed between the
    # calls as between the device-resident steps (the flush is queued on the
    # traversal's stream; the copies in run on the library's copy stream).
    Oh = torch.from_numpy(rays.origin).pin_memory()
    Dh = torch.from_numpy(rays.dir).pin_memory()
    Th = torch.empty(N, dtype=torch.float32).pin_memory()
    for _ in range(2):
        vg.trace_host(Oh, Dh, precision="fp32", out_tau=Th, wait=False)
    if ws > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        flush.zero_()
        vg.trace_host(Oh, Dh, precision="fp32", out_tau=Th, wait=False)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    assert np.array_equal(Th.numpy(), tau.cpu().numpy()), "host-pipelined tau differs from the device call"

    def reduce_max(x):
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        return float(t.item())

    def reduce_sum(x):
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.SUM)
        return float(t.item())

    step_ms_max = reduce_max(step_ms)
    step64_max = reduce_max(step64_ms)
    stepx_max = reduce_max(stepx_ms)
    e2e_max = reduce_max(e2e_ms)
    seg_all = reduce_sum(float(crossings))
    rays_all = reduce_sum(float(N))
    value = seg_all * args.steps / (step_ms_max / 1e3)
    value64 = seg_all * k64 / (step64_max / 1e3)

    # roofline of the traversal kernel: algorithmic bytes per crossing
    deg = info["nnz"] / info["M"]
    bytes_per_crossing = 28.0 + 20.0 * deg
    trace_launch_ms = tr_ms / max(launches, 1)
    traffic = profiled("trace_kernel_disk1e5.md", "dram bytes per full launch")
    roof = roofline(crossings, bytes_per_crossing, trace_launch_ms, info["rel_bytes"], ceil, traffic,
                    "trace_kernel<1,false,TAU,false>")
    roof["locate_ms_per_step"] = loc_ms / max(launches, 1)

    if rank != 0:
        if ws > 1:
            tdist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": info["M"], "rays_per_gpu": N, "mean_degree": round(deg, 3),
                   "l2": "flushed between timed steps (2x L2 buffer written), also between the e2e calls",
                   "launch": launch, "parallelism": f"rays sharded over {ws} GPU(s)"},
        "rays_per_s": rays_all * args.steps / (step_ms_max / 1e3),
        "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": step64_max / k64,
                      "trace_ms_per_launch": tr64_ms / max(launches64, 1)},
        "fp32_over_fp64": value / value64,
        "fp32_exact_form": {"value": seg_all * kx / (stepx_max / 1e3), "unit": UNIT, "ms_per_step": stepx_max / kx,
                            "trace_ms_per_launch": trx_ms / max(launchesx, 1),
                            "lengths": "float32 decisions, each crossing's length from the exact site difference "
                                       "in float-pair arithmetic"},
        "tau_rel_err_vs_fp64": tau_err,
        "stats_per_step": st32,
        "recheck_rate": st32["rechecks"] / max(st32["decisions"], 1),
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "e2e": {"value": seg_all * args.steps / (e2e_max / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(O.numel() * 8 + D.numel() * 8), "d2h_bytes_per_step": int(N * 4)},
        "clocks": clocks,
    }
    if ws == 1 and not args.no_cpu_baseline:
        base, acc = cpu_baseline(g, rays, tau.cpu().numpy(), tau64.cpu().numpy(), tau32x=tau32x.cpu().numpy())
        acc.update({"gpu_recheck_rate": st32["rechecks"] / max(st32["decisions"], 1),
                    "gpu_fallbacks_fp32": st32["fallbacks"], "gpu_fallbacks_fp64": st64["fallbacks"]})
        line["cpu_baseline"] = base
        line["accuracy"] = acc
    if ws == 1 and not args.no_other_configs:
        del O, D, tau, tau64, tau32x, Oh, Dh, Th
        del vg
        torch.cuda.empty_cache()
        other = {}
        for name, fn in (("clumpy1e6", measure_clumpy1e6), ("batched64", measure_batched64),
                         ("grad1e6", measure_grad1e6)):
            r = fn(steps=5, warmup=3, flush=flush, sampler=ClockSampler(gpu_index(local)))
            other[name] = {k: r[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "clocks",
                                             "gpu_launches", "roofline") if k in r}
            for k in ("launch", "tuned", "via_segment_lists", "fd_check"):
                if k in r:
                    other[name][k] = r[k]
            torch.cuda.empty_cache()
        line["other_configs"] = other
    print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()


# ---------------------------------------------------------------------------
# other workloads (one GPU): 10^6 clumpy sites, 64 uneven grids in one
# launch, the adjoint on the 10^6-site disk, and segment lists on the
# 10^5-site disk
# ---------------------------------------------------------------------------

def _events_ms(fn, steps, flush):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        fn()
        ev[k][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def _base_line():
    return {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic"}


def measure_clumpy1e6(steps, warmup, flush, sampler):
    """10^6 clumpy sites (2,000 Gaussian clumps), 10^7 uniform rays, tau."""
    import torch

    import gen
    from paper_1310_1854_gb300 import VoronoiGrid
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    g, rays = gen.config3()
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    build_s = time.time() - t0
    info = vg.info()
    O = torch.from_numpy(rays.origin).to(dev)
    D = torch.from_numpy(rays.dir).to(dev)
    N = O.shape[0]
    tau = torch.empty(N, dtype=torch.float32, device=dev)
    st = vg.trace(O, D, precision="fp32", stats=True).stats
    fn = lambda: vg.trace(O, D, precision="fp32", out_tau=tau)
    for _ in range(warmup):
        fn()
    vg.enable_timing(True)
    vg.read_timing()
    sampler.start()
    n0 = kernel_launches()
    ms = _events_ms(fn, steps, flush)
    n_kernels = kernel_launches() - n0
    clocks = sampler.stop()
    loc_ms, tr_ms, launches = vg.read_timing()
    vg.enable_timing(False)
    deg = info["nnz"] / info["M"]
    kern = tr_ms / max(launches, 1)
    line = dict(_base_line(), value=st["crossings"] * steps / (ms / 1e3), ms_per_step=ms / steps, steps=steps,
                warmup=warmup,
                config={"workload": "clumpy 1e6 sites (2,000 clumps), 1e7 uniform rays, tau per ray",
                        "sites": info["M"], "rays": N, "mean_degree": round(deg, 3), "host_build_s": round(build_s, 2),
                        "device_bytes": info["device_bytes"], "l2": "flushed between timed steps"},
                stats_per_step=st, rays_per_s=N * steps / (ms / 1e3), gpu_launches=n_kernels, clocks=clocks,
                launch=vg.get_launch(),
                roofline=roofline(st["crossings"], 28.0 + 20.0 * deg, kern, info["rel_bytes"], None,
                                  profiled("trace_kernel_clumpy1e6.md", "dram bytes per full launch")),
                e2e=None)
    line["roofline"]["locate_ms_per_step"] = loc_ms / max(launches, 1)
    return line


def measure_grad1e6(steps, warmup, flush, sampler):
    """10^6-site disk, 512^2 detector + 10^6 interior rays: tau, the loss
    sum (exp(-tau) - target)^2 and its gradient with respect to all cell
    densities; by a second (adjoint) traversal, and from the segment lists
    kept by the forward traversal."""
    import torch

    import gen
    from paper_1310_1854_gb300 import VoronoiGrid
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    g, det, inner, rho_t = gen.config5()
    rays = gen.concat_rays(det, inner)
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    build_s = time.time() - t0
    info = vg.info()
    O = torch.from_numpy(rays.origin).to(dev)
    D = torch.from_numpy(rays.dir).to(dev)
    N = O.shape[0]
    tau = torch.empty(N, dtype=torch.float32, device=dev)
    st = vg.trace(O, D, precision="fp32", stats=True).stats
    vg.set_density(torch.from_numpy(rho_t).to(dev))
    target = torch.exp(-vg.trace(O, D, precision="fp32").tau)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    grad = torch.zeros(g.sites.shape[0], dtype=torch.float32, device=dev)

    def fn():
        t = vg.trace(O, D, precision="fp32", out_tau=tau).tau
        e = torch.exp(-t)
        dL = -2.0 * (e - target) * e
        grad.zero_()
        vg.trace_grad(O, D, dL, out=grad)

    for _ in range(warmup):
        fn()
    vg.enable_timing(True)
    vg.read_timing()
    sampler.start()
    n0 = kernel_launches()
    ms = _events_ms(fn, steps, flush)
    n_kernels = kernel_launches() - n0
    clocks = sampler.stop()
    loc_ms, tr_ms, launches = vg.read_timing()
    vg.enable_timing(False)
    segs = st["crossings"] * 2
    kern = tr_ms / max(launches, 1)
    cap = st["crossings"]

    def fn_seg():
        r = vg.trace(O, D, precision="fp32", segments=True, seg_capacity=cap)
        e = torch.exp(-r.tau)
        dL = -2.0 * (e - target) * e
        grad.zero_()
        vg.segments_grad(r, dL, out=grad)

    g_two = grad.clone()
    fn_seg()
    torch.cuda.synchronize()
    rel = float(((grad - g_two).abs().max() / g_two.abs().max()).item())
    for _ in range(warmup):
        fn_seg()
    ms_seg = _events_ms(fn_seg, steps, flush)
    deg = info["nnz"] / info["M"]
    return dict(_base_line(), value=segs * steps / (ms / 1e3), ms_per_step=ms / steps, steps=steps, warmup=warmup,
                config={"workload": "exp-disk 1e6 sites, 512^2 detector + 1e6 interior rays, tau and adjoint "
                                    "d loss / d rho (two traversals per step)",
                        "sites": info["M"], "rays": N, "mean_degree": round(deg, 3), "traversals_per_step": 2,
                        "host_build_s": round(build_s, 2), "device_bytes": info["device_bytes"],
                        "l2": "flushed between timed steps"},
                stats_per_traversal=st, rays_per_s=N * 2 * steps / (ms / 1e3), gpu_launches=n_kernels,
                clocks=clocks, launch=vg.get_launch(),
                via_segment_lists={"value": segs * steps / (ms_seg / 1e3), "ms_per_step": ms_seg / steps,
                                   "max_rel_diff_vs_two_traversals": rel},
                roofline=roofline(st["crossings"], 28.0 + 20.0 * deg, kern, info["rel_bytes"], None),
                e2e=None)


def measure_batched64(steps, warmup, flush, sampler):
    """64 grids (sites log-uniform in 2e3..2e5, rays log-uniform in
    1e4..1e6) in one persistent launch replayed from a CUDA graph, with the
    launch shape chosen by the autotuner."""
    import torch

    import gen
    from paper_1310_1854_gb300 import Batch, VoronoiGrid, tune
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    sets = gen.config4()
    grids = []
    total_sites = 0
    for g, r in sets:
        vg = VoronoiGrid(g.sites, g.box)
        vg.set_density(torch.from_numpy(g.rho).to(dev))
        grids.append((vg, torch.from_numpy(r.origin).to(dev), torch.from_numpy(r.dir).to(dev)))
        total_sites += g.sites.shape[0]
    build_s = time.time() - t0
    b = Batch(grids)
    t0 = time.time()
    tuned = tune.autotune_batch(b)
    tune_s = time.time() - t0
    st = b.run(stats=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(warmup):
            b.run(graph=True, stream=s)
        s.synchronize()
        sampler.start()
        n0 = kernel_launches()
        ms = _events_ms(lambda: b.run(graph=True, stream=s), steps, flush)
        n_kernels = kernel_launches() - n0
        clocks = sampler.stop()
    infos = [vg.info() for vg, _, _ in grids]
    rel = sum(i["rel_bytes"] for i in infos)
    # roofline of the step: the graph holds the start-cell pass, the order
    # and the traversal, so the whole step's time stands in for the
    # traversal's (a lower bound on its rate); each grid is traced while its
    # blocks are held in L2, so the ceilings are measured on a buffer the
    # size of the largest grid's blocks
    deg = sum(i["nnz"] for i in infos) / max(sum(i["M"] for i in infos), 1)
    big = max(i["rel_bytes"] for i in infos)
    roof = roofline(st["crossings"], 28.0 + 20.0 * deg, ms / steps, big, l2_ceilings(big), None,
                    "trace_kernel<1,false,TAU,true> (the whole step's time)")
    roof["note"] = ("the batch's grids are traced one after another, each held in L2; the graph gives no "
                    "per-kernel time, so the step's time (start cells, order, traversal) is used")
    roof["cell_block_bytes_all_grids"] = rel
    return dict(_base_line(), value=st["crossings"] * steps / (ms / 1e3), ms_per_step=ms / steps, steps=steps,
                warmup=warmup,
                config={"workload": "64 grids, sites log-uniform 2e3..2e5, rays log-uniform 1e4..1e6, one "
                                    "persistent launch replayed from a CUDA graph, autotuned launch shape",
                        "grids": len(sets), "sites": total_sites, "rays": st["rays"],
                        "host_build_s": round(build_s, 2), "l2": "flushed between timed steps"},
                stats_per_step=st, rays_per_s=st["rays"] * steps / (ms / 1e3), gpu_launches=n_kernels,
                clocks=clocks, launch=b.get_launch(),
                tuned={k: tuned[k] for k in ("lanes_per_ray", "block", "blocks_per_sm", "order", "cached",
                                             "sample_rays", "key")} | {"tune_s": round(tune_s, 2)},
                roofline=roof, e2e=None)


def measure_segments1e5(steps, warmup, flush, sampler, n_rays=1_000_000):
    """The disk workload with segment lists (CSR cell + length) and tau."""
    import torch

    import gen
    from paper_1310_1854_gb300 import VoronoiGrid
    dev = torch.device("cuda", torch.cuda.current_device())
    g, _ = gen.config2(n_rays=1)
    rays = gen.disk_rays(n_rays, gen.SEED_BASE + 2 + 1000)
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    info = vg.info()
    O = torch.from_numpy(rays.origin).to(dev)
    D = torch.from_numpy(rays.dir).to(dev)
    N = O.shape[0]
    ceil = l2_ceilings(info["rel_bytes"])
    res = {}
    for prec in ("fp32", "fp64"):
        r = vg.trace(O, D, precision=prec, segments=True, stats=True)
        cap = int(r.seg_off[N].item())
        fn = lambda: vg.trace(O, D, precision=prec, segments=True, seg_capacity=cap)
        for _ in range(warmup):
            fn()
        k = steps if prec == "fp32" else max(3, steps // 4)
        vg.enable_timing(True)
        vg.read_timing()
        sampler.start()
        n0 = kernel_launches()
        ms = _events_ms(fn, k, flush)
        n_kernels = kernel_launches() - n0
        clocks = sampler.stop()
        _, tr_ms, launches = vg.read_timing()
        vg.enable_timing(False)
        res[prec] = (cap * k / (ms / 1e3), ms / k, n_kernels, clocks, r.stats, tr_ms / max(launches, 1))
    v32, ms32, nk, clocks, st, kern = res["fp32"]
    deg = info["nnz"] / info["M"]
    # the traversal's algorithmic bytes per crossing plus the 8-byte slot
    # it stores per segment
    bpc = 28.0 + 20.0 * deg + 8.0
    return dict(_base_line(), value=v32, ms_per_step=ms32, steps=steps, warmup=warmup,
                config={"workload": "exp-disk 1e5 sites, 1e6 rays, segment list (cell, length) of every ray in "
                                    "CSR form plus tau", "sites": info["M"], "rays": N,
                        "segments": st["crossings"], "l2": "flushed between timed steps"},
                fp64={"value": res["fp64"][0], "ms_per_step": res["fp64"][1],
                      "traversal_ms_per_launch": res["fp64"][5]},
                stats_per_step=st, gpu_launches=nk, clocks=clocks,
                roofline=roofline(st["crossings"], bpc, kern, info["rel_bytes"], ceil), e2e=None)


def run_extra(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(gpu_index(0))
    if args.workload == "next":
        base = dict(_base_line(), steps=args.steps, warmup=args.warmup)
        return run_next(args, base, flush, sampler)
    fn = {"segments1e5": measure_segments1e5, "clumpy1e6": measure_clumpy1e6, "grad1e6": measure_grad1e6,
          "batched64": measure_batched64}[args.workload]
    print(json.dumps(fn(args.steps, args.warmup, flush, sampler)), flush=True)


def run_next(args, base, flush, sampler):
    """One line per row built after the hot path: Monte Carlo interaction
    sampling along the path, rays entering from outside the box, a spherical
    domain, C(r) at uniform points for the grid-quality measure (Table 1),
    and the cell construction on the GPU."""
    import torch

    import gen
    from paper_1310_1854_gb300 import VoronoiGrid
    from paper_1310_1854_gb300.quality import grid_quality, sample_points
    dev = torch.device("cuda", 0)
    g, _ = gen.config2(n_rays=1)
    vg = VoronoiGrid(g.sites, g.box)
    vg.set_density(torch.from_numpy(g.rho).to(dev))
    N = args.rays
    rays = gen.disk_rays(N, gen.SEED_BASE + 2 + 1000)
    O = torch.from_numpy(rays.origin).to(dev)
    D = torch.from_numpy(rays.dir).to(dev)
    rng = gen.rng_for(gen.SEED_BASE + 77)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        sampler.start()
        n0 = kernel_launches()
        ms = _events_ms(fn, steps, flush)
        return ms / steps, kernel_launches() - n0, sampler.stop()

    # f1: tau_int = -ln(xi) per package; the package stops in the cell where
    # the running tau reaches it, and the absorbed weight is booked per cell
    tau_int = torch.from_numpy(-np.log(rng.random(N))).to(dev, torch.float32)
    absorbed = torch.zeros(g.sites.shape[0], dtype=torch.float32, device=dev)
    cell, _, _ = vg.interact(O, D, tau_int, absorbed=absorbed)
    interacted = int((cell >= 0).sum().item())
    ms, nk, clocks = timed(lambda: vg.interact(O, D, tau_int, absorbed=absorbed), args.steps)
    line = dict(base, metric="Monte Carlo photon packages/sec (interaction point sampled along the path)",
                unit="packages/s", value=N / (ms / 1e3), ms_per_step=ms, gpu_launches=nk, clocks=clocks,
                config={"workload": "exp-disk 1e5 sites, 1e6 packages from the disk sampler, tau_int = -ln xi, "
                                    "absorbed weight booked per cell", "sites": g.sites.shape[0], "packages": N,
                        "interacting": interacted, "l2": "flushed between timed steps"},
                roofline=None, e2e=None)
    print(json.dumps(line), flush=True)

    # f2: rays from a sphere around the box aimed at uniform points inside it
    c = 0.5 * (g.box[:3] + g.box[3:])
    R = 0.6 * float(np.linalg.norm(g.box[3:] - g.box[:3]))
    u = rng.standard_normal((N, 3))
    org = c + R * u / np.linalg.norm(u, axis=1, keepdims=True)
    tgt = sample_points(g.box, N, gen.SEED_BASE + 78)
    dirs = tgt - org
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Oe = torch.from_numpy(org).to(dev)
    De = torch.from_numpy(dirs).to(dev)
    st = vg.trace(Oe, De, precision="fp32", stats=True, enter=True).stats
    tau = torch.empty(N, dtype=torch.float32, device=dev)
    ms, nk, clocks = timed(lambda: vg.trace(Oe, De, precision="fp32", out_tau=tau, enter=True), args.steps)
    line = dict(base, value=st["crossings"] / (ms / 1e3), ms_per_step=ms, gpu_launches=nk, clocks=clocks,
                config={"workload": "exp-disk 1e5 sites, 1e6 rays from a sphere around the box aimed at uniform "
                                    "points inside it (entry point by the slab test, then the same traversal)",
                        "sites": g.sites.shape[0], "rays": N, "l2": "flushed between timed steps"},
                stats_per_step=st, roofline=None, e2e=None)
    print(json.dumps(line), flush=True)

    # f2, another domain geometry: a ball (the unit ball inscribed in
    # [-1,1]^3), 1e5 sites and 1e6 rays inside it
    gb = gen.make_ball_grid(100_000, gen.SEED_BASE + 80)
    vb = VoronoiGrid(gb.sites, gb.box, sphere=gen.UNIT_BALL)
    vb.set_density(torch.from_numpy(gb.rho).to(dev))
    rb = gen.ball_rays(N, gen.SEED_BASE + 81)
    Ob = torch.from_numpy(rb.origin).to(dev)
    Db = torch.from_numpy(rb.dir).to(dev)
    st = vb.trace(Ob, Db, precision="fp32", stats=True).stats
    ms, nk, clocks = timed(lambda: vb.trace(Ob, Db, precision="fp32", out_tau=tau), args.steps)
    line = dict(base, value=st["crossings"] / (ms / 1e3), ms_per_step=ms, gpu_launches=nk, clocks=clocks,
                config={"workload": "spherical domain: 1e5 sites uniform in the unit ball, rho = exp(-3|r|), "
                                    "1e6 rays from uniform points of the ball, paths ending on the sphere",
                        "sites": gb.sites.shape[0], "rays": N, "l2": "flushed between timed steps"},
                stats_per_step=st, roofline=None, e2e=None)
    print(json.dumps(line), flush=True)

    # f3: C(r) at 1e7 uniform points of the 1e6-site disk (Table 1's measure)
    g5, _, _, _ = gen.config5(npix=1, n_interior=1)
    v5 = VoronoiGrid(g5.sites, g5.box)
    P = torch.from_numpy(sample_points(g5.box, 10_000_000, gen.SEED_BASE + 79)).to(dev)
    ms, nk, clocks = timed(lambda: v5.locate(P), args.steps)
    q = grid_quality(v5, g5.rho, gen.disk_density, n_points=10_000_000)
    line = dict(base, metric="C(r) point locations/sec (grid-quality sampling, Table 1)", unit="points/s",
                value=P.shape[0] / (ms / 1e3), ms_per_step=ms, gpu_launches=nk, clocks=clocks,
                config={"workload": "exp-disk 1e6 sites, 1e7 uniform points of the box, float32 distances with "
                                    "float64 recheck", "sites": g5.sites.shape[0], "points": P.shape[0],
                        "l2": "flushed between timed steps"},
                quality={"std_rho_t_minus_rho_g": q["std"], "mean": q["mean"], "points": q["points"]},
                roofline=None, e2e=None)
    print(json.dumps(line), flush=True)

    # f4: the cells of the 1e6-site clumpy grid built on the GPU (the whole
    # vgrid_create, host phases included, wall clock); the host builder once
    # beside it
    del v5, P
    g3, _ = gen.config3(n_rays=1)
    reps = max(1, min(args.steps, 3))
    VoronoiGrid(g3.sites, g3.box, gpu_build=True)  # warm-up
    sampler.start()
    n0 = kernel_launches()
    t0 = time.perf_counter()
    for _ in range(reps):
        vg3 = VoronoiGrid(g3.sites, g3.box, gpu_build=True)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / reps
    nk = (kernel_launches() - n0) // reps
    clocks = sampler.stop()
    info = vg3.info()
    t0 = time.perf_counter()
    VoronoiGrid(g3.sites, g3.box)
    host_sec = time.perf_counter() - t0
    M3 = g3.sites.shape[0]
    line = dict(base, metric="Voronoi cells built/sec (GPU cell construction, whole vgrid_create)", unit="cells/s",
                value=M3 / sec, ms_per_step=sec * 1e3, steps=reps, higher_is_better=True, gpu_launches=nk,
                clocks=clocks, dtype="f64",
                config={"workload": "clumpy 1e6 sites (2,000 clumps): neighbour lists, volumes and bounding boxes "
                                    "cut on the GPU, then the device layout", "sites": M3,
                        "phase_seconds": [round(x, 4) for x in info["phase_seconds"]],
                        "cell_kernel_cells_per_s": M3 / max(info["phase_seconds"][2], 1e-9),
                        "host_fallback_cells": info["host_fallback_cells"],
                        "host_builder_seconds": round(host_sec, 3), "timing": "wall clock, host and device"},
                roofline=None, e2e=None)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
