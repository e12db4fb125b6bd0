"""Accuracy of the GPU traversal against the CPU oracle on the full-size
workloads (the paper's precision question for this build: how far the
float32 form with float64 rechecks, and the float64 form, are from a plain
float64 evaluation of Eq. 1-5 along the path of Sect. 2.2).

For every workload the GPU traces all of its rays in the launch shape the
benchmark uses: tau in both forms, and the segment lists of the float32 form
(and of the float64 form where they fit comfortably). A seeded sample of at
least 10^4 rays is traced by the oracle over its own neighbour lists (pinned
equal to the exit over all sites). On the sample's rays that are not near
ties (any decision margin <= 1e-9, a winning plane through the point, or an
ambiguous start) the cell sequences must be identical and tau within 1e-5
(float32) / 1e-12 (float64) relative; float64 lengths within 1e-12 relative.
The report gives the max, p99 and mean relative tau error, the near-tie
fraction of the sample, and the recheck rate and fallback count of all rays.

Test infrastructure: it calls the oracle. `python -m tests.accuracy [name ...]`
on a GPU machine prints one JSON line per workload.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402

TAU32_REL = 1e-5
TAU64_REL = 1e-12
LEN64_REL = 1e-12
SAMPLE = 10_000


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_lists(g):
    c = oracle.cells(g.sites, g.box, maxdeg=128)
    return oracle.csr(c, len(g.sites))


def oracle_sample(g, rays, sel, off, idx, cap=4096):
    return oracle.trace(g.sites, g.box, g.rho.astype(np.float64), rays.origin[sel], rays.dir[sel], off=off, idx=idx,
                        kappa=float(g.kappa), cap=cap)


def gather_segments(res, sel):
    """The segment lists of rays `sel` from a GPU TraceResult, gathered on
    the device: (cells, lengths, per-ray offsets) as numpy arrays."""
    import torch
    so = res.seg_off
    s = torch.as_tensor(np.asarray(sel), dtype=torch.int64, device=so.device)
    a, b = so[s], so[s + 1]
    cnt = b - a
    first = torch.cumsum(cnt, 0) - cnt
    tot = int(cnt.sum().item())
    ray = torch.repeat_interleave(torch.arange(s.numel(), device=so.device), cnt)
    pos = torch.arange(tot, device=so.device) - first[ray] + a[ray]
    off = np.zeros(s.numel() + 1, np.int64)
    off[1:] = np.cumsum(cnt.cpu().numpy())
    return res.seg_cell[pos].cpu().numpy(), res.seg_len[pos].cpu().numpy().astype(np.float64), off


def _stats(x):
    if x.size == 0:
        return None
    return {"max": float(x.max()), "p99": float(np.quantile(x, 0.99)), "mean": float(x.mean())}


def compare(ref, ok, tau32=None, tau64=None, seg32=None, seg64=None, diag=1.0):
    """Sample rays against the oracle. ok: rays that are not near ties. seg*:
    (cells, lengths, offsets) of the sample's rays. Returns the statistics
    and the lists of rays that break each bound."""
    out = {"sample": int(ok.size), "near_tie_fraction": float(1.0 - ok.mean()),
           "oracle_fallbacks": int(ref.nfallback.sum()), "oracle_status_ok": bool(np.all(ref.status == 0))}
    bad = {}
    pos = ok & (ref.tau > 0)
    if tau32 is not None:
        rel = np.abs(tau32.astype(np.float64) - ref.tau) / np.maximum(ref.tau, 1e-300)
        out["fp32_tau_rel_err"] = _stats(rel[pos])
        out["fp32_tau_rel_err_incl_near_ties"] = _stats(rel[ref.tau > 0])
        bad["fp32_tau"] = np.nonzero(pos & (rel > TAU32_REL))[0].tolist()
    if tau64 is not None:
        rel = np.abs(tau64 - ref.tau) / np.maximum(ref.tau, 1e-300)
        out["fp64_tau_rel_err"] = _stats(rel[pos])
        bad["fp64_tau"] = np.nonzero(pos & (rel > TAU64_REL))[0].tolist()
    for name, seg in (("fp32", seg32), ("fp64", seg64)):
        if seg is None:
            continue
        cells, lens, so = seg
        mism, lbad = [], []
        for i in np.nonzero(ok)[0]:
            rc, rl = ref.segments(i)
            gc = cells[so[i]:so[i + 1]]
            if not np.array_equal(gc, rc):
                mism.append(int(i))
            elif name == "fp64":
                gl = lens[so[i]:so[i + 1]]
                tol = np.where(rl < 1e-6 * diag, 1e-12 * diag, LEN64_REL * rl)
                if not np.all(np.abs(gl - rl) <= tol):
                    lbad.append(int(i))
        out[f"{name}_sequences_compared"] = int(ok.sum())
        out[f"{name}_sequence_mismatches"] = len(mism)
        bad[f"{name}_sequence"] = mism
        if name == "fp64":
            bad["fp64_length"] = lbad
    return out, bad


def _gpu_stats(st):
    return {"gpu_rays": st["rays"], "gpu_crossings": st["crossings"],
            "gpu_recheck_rate": st["rechecks"] / max(st["decisions"], 1), "gpu_rechecks": st["rechecks"],
            "gpu_fallbacks": st["fallbacks"], "gpu_zero_steps": st["zero_steps"]}


def _grid(g, **kw):
    import torch
    from paper_1310_1854_gb300 import VoronoiGrid
    vg = VoronoiGrid(g.sites, g.box, **kw)
    vg.set_density(torch.from_numpy(g.rho).cuda(), float(g.kappa))
    return vg


def _single(name, g, rays, sample_sel, fp64_segments=True, seed=0):
    """One grid: all rays on the GPU, the sample against the oracle."""
    vg = _grid(g)
    O, D = _dev(rays.origin), _dev(rays.dir)
    t32 = vg.trace(O, D, precision="fp32", stats=True)
    t64 = vg.trace(O, D, precision="fp64", stats=True)
    s32 = vg.trace(O, D, precision="fp32", segments=True)
    seg32 = gather_segments(s32, sample_sel)
    del s32
    seg64 = None
    if fp64_segments:
        s64 = vg.trace(O, D, precision="fp64", segments=True)
        seg64 = gather_segments(s64, sample_sel)
        del s64
    tau32 = t32.tau.cpu().numpy()[sample_sel]
    tau64 = t64.tau.cpu().numpy()[sample_sel]
    t0 = time.time()
    off, idx = oracle_lists(g)
    ref = oracle_sample(g, rays, sample_sel, off, idx)
    t_or = time.time() - t0
    ok = ref.near_tie == 0
    diag = float(np.linalg.norm(g.box[3:] - g.box[:3]))
    stats, bad = compare(ref, ok, tau32, tau64, seg32, seg64, diag)
    stats.update(_gpu_stats(t32.stats))
    stats.update({"workload": name, "rays": len(rays.origin), "sites": len(g.sites), "launch": vg.get_launch(),
                  "gpu_fallbacks_fp64": t64.stats["fallbacks"], "oracle_seconds": round(t_or, 1)})
    return stats, bad, (vg, O, D, t32, ref, sample_sel)


def disk1e5(n_sample=SAMPLE):
    """10^5-site disk, 10^6 rays (the benchmark workload)."""
    g, rays = gen.config2()
    sel = np.sort(gen.rng_for(501).choice(len(rays.origin), n_sample, replace=False))
    stats, bad, _ = _single("disk1e5: 1e5-site exp-disk, 1e6 rays", g, rays, sel)
    return stats, bad


def clumpy1e6(n_sample=SAMPLE):
    """10^6 clumpy sites, 10^7 rays: tau of both forms and the float32
    segment lists from the full ordered launch."""
    g, rays = gen.config3()
    sel = np.sort(gen.rng_for(502).choice(len(rays.origin), n_sample, replace=False))
    stats, bad, _ = _single("clumpy1e6: 1e6 clumpy sites, 1e7 rays", g, rays, sel, fp64_segments=False)
    return stats, bad


def grad1e6(n_sample=SAMPLE, n_detector=2000, keep=False):
    """10^6-site disk, 512^2 detector rays and 10^6 interior rays; the sample
    holds n_detector detector rays."""
    g, det, inner, rho_t = gen.config5()
    rays = gen.concat_rays(det, inner)
    nd = len(det.origin)
    rng = gen.rng_for(503)
    sel = np.sort(np.concatenate([rng.choice(nd, n_detector, replace=False),
                                  nd + rng.choice(len(inner.origin), n_sample - n_detector, replace=False)]))
    stats, bad, ctx = _single("grad1e6: 1e6-site exp-disk, 512^2 detector + 1e6 interior rays", g, rays, sel)
    stats["detector_rays_in_sample"] = int((sel < nd).sum())
    stats["detector_rays_compared"] = int(((sel < nd) & (ctx[4].near_tie == 0)).sum())
    return (stats, bad, ctx, g, rays, rho_t) if keep else (stats, bad)


def batched64(n_sample=SAMPLE, tuned=True):
    """64 grids in one batch launch (autotuned shape): tau of every set from
    the batch; segment lists from single-grid launches of every full set;
    the sample spread over the grids in proportion to their rays (at least
    20 per grid)."""
    import torch
    from paper_1310_1854_gb300 import Batch, tune
    sets = gen.config4()
    grids = []
    for g, r in sets:
        grids.append((_grid(g), _dev(r.origin), _dev(r.dir)))
    b = Batch(grids)
    tuned_shape = tune.autotune_batch(b, use_cache=False) if tuned else None
    st = b.run(stats=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(graph=True, stream=s)
    s.synchronize()
    total = sum(len(r.origin) for _, r in sets)
    rng = gen.rng_for(504)
    agg = {"sample": 0, "near_tie": 0, "oracle_fallbacks": 0, "fp32_seq": 0, "fp32_mism": 0}
    rels, rels_all, bad_all = [], [], {"fp32_tau": [], "fp32_sequence": [], "batch_vs_single": []}
    t_or = 0.0
    for k, ((g, r), (vg, O, D)) in enumerate(zip(sets, grids)):
        n = len(r.origin)
        m = min(n, max(20, int(round(n_sample * n / total))))
        sel = np.sort(rng.choice(n, m, replace=False))
        single = vg.trace(O, D, precision="fp32").tau.cpu().numpy()
        if not np.array_equal(single, b.tau[k].cpu().numpy()):
            bad_all["batch_vs_single"].append(k)
        seg = gather_segments(vg.trace(O, D, precision="fp32", segments=True), sel)
        t0 = time.time()
        off, idx = oracle_lists(g)
        ref = oracle_sample(g, r, sel, off, idx)
        t_or += time.time() - t0
        ok = ref.near_tie == 0
        stats, bad = compare(ref, ok, b.tau[k].cpu().numpy()[sel], None, seg, None)
        pos = ok & (ref.tau > 0)
        t = b.tau[k].cpu().numpy()[sel].astype(np.float64)
        rels.append((np.abs(t - ref.tau) / np.maximum(ref.tau, 1e-300))[pos])
        rels_all.append((np.abs(t - ref.tau) / np.maximum(ref.tau, 1e-300))[ref.tau > 0])
        agg["sample"] += m
        agg["near_tie"] += int((~ok).sum())
        agg["oracle_fallbacks"] += int(ref.nfallback.sum())
        agg["fp32_seq"] += stats["fp32_sequences_compared"]
        agg["fp32_mism"] += stats["fp32_sequence_mismatches"]
        bad_all["fp32_tau"] += [(k, i) for i in bad["fp32_tau"]]
        bad_all["fp32_sequence"] += [(k, i) for i in bad["fp32_sequence"]]
    out = {"workload": "batched64: 64 grids, sites 2e3..2e5, rays 1e4..1e6, one persistent launch (CUDA graph)",
           "rays": total, "sites": sum(len(g.sites) for g, _ in sets), "sample": agg["sample"],
           "near_tie_fraction": agg["near_tie"] / agg["sample"], "oracle_fallbacks": agg["oracle_fallbacks"],
           "fp32_tau_rel_err": _stats(np.concatenate(rels)),
           "fp32_tau_rel_err_incl_near_ties": _stats(np.concatenate(rels_all)),
           "fp32_sequences_compared": agg["fp32_seq"], "fp32_sequence_mismatches": agg["fp32_mism"],
           "batch_launch": b.get_launch(), "oracle_seconds": round(t_or, 1)}
    if tuned_shape is not None:
        out["tuned"] = {k: tuned_shape[k] for k in ("lanes_per_ray", "block", "blocks_per_sm", "order")}
    out.update(_gpu_stats(st))
    return out, bad_all


WORKLOADS = {"disk1e5": disk1e5, "clumpy1e6": clumpy1e6, "batched64": batched64, "grad1e6": grad1e6}


def main(names):
    for name in names or list(WORKLOADS):
        t0 = time.time()
        stats, bad = WORKLOADS[name]()
        stats["violations"] = {k: len(v) for k, v in bad.items()}
        stats["seconds"] = round(time.time() - t0, 1)
        print(json.dumps(stats), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
