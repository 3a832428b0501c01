"""Benchmark: min-cut solve throughput (Mnodes/s) on the 512x512x384 seismic-scale volume.

One step = one whole solve of the volume through the C ABI: graph construction
(pog_build), push-relabel with global relabels to a maximum preflow, cut extraction and
surface heights (pog_maxflow + pog_surface). `value` times steps whose input already
sits in HBM; `e2e` times the same solve from a pinned host buffer, with the H2D copy of
the costs and the D2H read of the heights and flow inside the timed region.

--impl reference times the CPU oracle (explicit-edge Dinic) on a bounded crop of the same
workload. Several GPUs: one independent replica per rank (the single-volume solve does
not shard), max-over-ranks timing, value = all ranks' nodes / that time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "min-cut solve Mnodes/s at 512x512x384 (plain vs batched); % of HBM roofline"
UNIT = "Mnodes/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(name):
    from paper_2601_17026_gb300 import synth

    if name == "seismic":
        return synth.seismic_volume()
    if name == "medium":
        return synth.medium_volume()
    if name == "small":
        return synth.small_volume()
    if name == "seismic-crop":
        return synth.seismic_crop()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of this rank's values over all ranks of the initialised
    process group (the values themselves without one, or at one rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(ranks, nodes, steps, ms):
    """Whole-job Mnodes/s of independent replicas: every rank's nodes over the slowest
    rank's time."""
    return ranks * nodes * steps / (ms / 1e3) / 1e6


def algorithmic_bytes(N, alpha, tiles_per_sweep, scans_per_sweep):
    """Per-launch algorithmic bytes of each kernel family.

    S = residual state per node: label, excess, sink residual (4 B each) plus the arc
    words (down flow, 4 hard flows, and 2 soft pair values when alpha > 0).
    tiled sweep: each visited tile of 1024 nodes is loaded whole (S per node) and its
                 owner-written words (label, sink residual: 8 B per node) are stored; the
                 first sweep after each global relabel also scans 4 B of excess per node
                 (`scans_per_sweep` = such sweeps / all sweeps).
    global relabel: every node's sink residual is read and its label written (8 B), its
                 arc words read once (4 B each), and the termination count reads
                 excess and label (8 B).
    cut: excess read, mark written, arc words read once.
    build: costs read (4 B per node), state written (S per node).
    """
    arc_words = 1 + 4 + (2 if alpha > 0 else 0)
    S = 4 * (3 + arc_words)
    return {
        "sweep": 4 * N * scans_per_sweep + tiles_per_sweep * 1024 * (S + 8),
        "bfs": (16 + 4 * arc_words) * N,
        "cut": (8 + 4 * arc_words) * N,
        "build": (4 + S) * N,
    }, S


# DRAM bytes per unit of work of the two dominant kernels, from ncu captures of the
# 256x256x384 crop of the benchmark volume (dram__bytes_read.sum + dram__bytes_write.sum
# of one launch divided by the launch's units: tile visits for the tiled sweep, nodes
# for the global relabel), with the SHA-256 prefix of the kernel source they were taken
# on. A kernel whose source changed since reports no traffic.
MEASURED_TRAFFIC = {
    # 64 launches after the first global relabel (warm L2, --cache-control none): 18.44 GB over
    # 290,567 tile visits
    "k_tile_push_relabel": {"bytes_per_unit": 63479, "unit": "tile visit", "source_sha": "80e2f306e500ec0b"},
    # the global relabel after those 64 sweeps: 4.57 GB over 25,165,824 nodes
    "k_global_relabel": {"bytes_per_unit": 181.4, "unit": "node", "source_sha": "ee6bef5d91380cd9"},
    # convex solve, 128x128x128 (delta 9, f(t) = 4 t^2): the 64 push launches between the first two
    # global relabels, 6.92 GB over 5,532,113 listed nodes
    "k_cv_push_relabel": {"bytes_per_unit": 1250.9, "unit": "listed node", "source_sha": "3e3c2d8a8aeb826c"},
}


def _source_sha(kernel):
    import hashlib

    src = {"k_tile_push_relabel": "pog_tile.cu", "k_global_relabel": "pog_bfs.cu",
           "k_cv_push_relabel": "pog_convex.cu"}.get(kernel)
    if src is None:
        return None
    h = hashlib.sha256()
    for name in (src, "pog_internal.cuh"):  # the kernel's file and the arc enumeration it uses
        with open(os.path.join(ROOT, "paper_2601_17026_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, units):
    """DRAM bytes of one launch processing `units` units, scaled from the ncu capture, or
    None when there is no capture of the current kernel source."""
    entry = MEASURED_TRAFFIC.get(kernel)
    if not entry or entry["source_sha"] != _source_sha(kernel) or not units:
        return None
    return entry["bytes_per_unit"] * units


def run_ours(args):
    import torch

    import __graft_entry__
    from paper_2601_17026_gb300 import pog

    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist

        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    __graft_entry__.build()
    from paper_2601_17026_gb300 import autotune

    vol = _workload(args.workload)
    X, Y, Z = vol.cost.shape
    N = vol.n
    host = torch.from_numpy(vol.cost).pin_memory()
    dev = host.cuda()
    stream = torch.cuda.current_stream()
    params = autotune.tuned_params(X, Y, Z, vol.delta, vol.alpha)
    if args.sweeps_per_relabel is not None:
        params["sweeps_per_relabel"] = args.sweeps_per_relabel
    opts = pog.make_options(flags=pog.POG_FLAG_TIMING, **params)
    plain_opts = pog.make_options(**params)

    def step(src_dev):
        with pog.pog_build(src_dev, vol.delta, vol.alpha, opts) as g:
            flow = pog.pog_maxflow(g)
            h = pog.pog_surface(g)
            st = pog.pog_stats(g)
        return flow, h, st

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flow0, h0, _ = step(dev)
    h0 = h0.cpu()

    # --- device-resident timed region
    barrier()
    stats = []
    with ClockSampler(torch.cuda.current_device()) as clocks:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            flow, h, st = step(dev)
            stats.append(st)
        t1.record(stream)
        barrier()
    ms = t0.elapsed_time(t1)
    assert flow == flow0 and torch.equal(h.cpu(), h0), "solves of the same volume disagree"

    # --- end to end from pinned host memory, through the public API
    hbuf = torch.empty((X, Y), dtype=torch.int32).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        d = host.to("cuda", non_blocking=True)
        with pog.pog_build(d, vol.delta, vol.alpha, plain_opts) as g:
            pog.pog_maxflow(g)  # flow value: 8 bytes read back
            hbuf.copy_(pog.pog_surface(g), non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    ms, e2e_ms = max_over_ranks([ms, e2e_ms], device="cuda")
    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    per_step = ms / args.steps
    value = job_throughput(ws, N, args.steps, ms)
    e2e_value = job_throughput(ws, N, args.steps, e2e_ms)
    # roofline of the two dominant kernel families, timed live with events on the solve stream
    tiles_per_sweep = sum(s["tiles_visited"] for s in stats) / max(sum(s["sweeps"] for s in stats), 1)
    scans_per_sweep = sum(s["rounds"] - 1 for s in stats) / max(sum(s["sweeps"] for s in stats), 1)
    bytes_per, S = algorithmic_bytes(N, vol.alpha, tiles_per_sweep, scans_per_sweep)
    fam = {"sweep": ("sweep_ms", "sweeps"), "bfs": ("bfs_ms", "rounds"), "cut": ("cut_ms", None),
           "build": ("build_ms", None)}
    tot = {k: sum(s[v[0]] for s in stats) for k, v in fam.items()}
    launches = {k: (sum(s[v[1]] for s in stats) if v[1] else len(stats)) for k, v in fam.items()}
    peak, peak_src = _peaks()
    kernel_name = {"sweep": "k_tile_push_relabel", "bfs": "k_global_relabel", "cut": "k_cut_reach",
                   "build": "k_build"}
    units = {"sweep": tiles_per_sweep, "bfs": N}

    def roofline(k):
        avg_ms = tot[k] / max(launches[k], 1)
        achieved = bytes_per[k] / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
        traffic = measured_traffic(kernel_name[k], units.get(k, 0))
        return {"bound": "hbm", "kernel": kernel_name[k], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None if traffic is None else int(traffic),
                "traffic_ratio": None if traffic is None else round(traffic / bytes_per[k], 2),
                "peak_source": peak_src, "bytes_per_launch": int(bytes_per[k]),
                "launches_per_step": launches[k] / len(stats), "avg_launch_ms": round(avg_ms, 5)}

    dom = max(("sweep", "bfs"), key=tot.get)
    st0 = stats[-1]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{X}x{Y}x{Z} layered-horizon volume, delta={vol.delta}, alpha={vol.alpha}",
                   "nodes": N, "state_bytes": int(st0["state_bytes"]), "params": params,
                   "l2": "inputs larger than L2 (cost 4N B, state ~%d B/node)" % S,
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * X * Y + 8},
        "roofline": roofline(dom),
        "rooflines": {kernel_name[k]: roofline(k) for k in ("sweep", "bfs")},
        "kernel_ms_per_step": {k: round(v / len(stats), 3) for k, v in tot.items()},
        "solver": {k: st0[k] for k in ("rounds", "sweeps", "bfs_passes", "cut_passes", "gaps", "active_initial",
                                        "tiles_visited")},
        "solver_spread": {"rounds": [int(s["rounds"]) for s in stats],
                          "ms_sweep": [round(s["sweep_ms"], 1) for s in stats],
                          "ms_relabel": [round(s["bfs_ms"], 1) for s in stats]},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clocks.summary(),
        "flow": flow,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, vol)
    if args.extras:
        line["batched"] = _leg(batched_leg, args)
        line["differentiable"] = _leg(differentiable_leg, args)
        line["narrow_band"] = _leg(narrow_band_leg, args)
        line["convex"] = _leg(convex_leg, args)
        if not args.no_cpu_baseline:
            line["cpu_baseline_batched"] = _leg(cpu_baseline_batched, args)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _leg(fn, args):
    """One extra leg of the line; a failure is reported in the leg's entry (the headline
    numbers above it stand on their own)."""
    try:
        return fn(args)
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def _timed_median(fn, warmup, steps):
    """Median wall time (s) of `steps` calls after `warmup` calls, device synchronised
    around each, and the last call's result."""
    import torch

    for _ in range(warmup):
        fn()
    times, out = [], None
    for _ in range(steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    return statistics.median(times), times, out


def batched_leg(args, warmup=1, steps=3):
    """The 64 uneven volumes through pog_solve_batch (inputs resident), aggregate Mnodes/s
    (median of `steps` solves); flows and surfaces checked against the oracle's stored
    values (tests/golden/batch.json)."""
    import hashlib

    import torch

    from paper_2601_17026_gb300 import autotune, pog, synth

    vols = synth.batch_volumes()
    costs = [torch.from_numpy(v.cost).cuda() for v in vols]
    deltas = [v.delta for v in vols]
    alphas = [v.alpha for v in vols]
    params = autotune.batch_params("uneven-64")
    opts = pog.make_options(**params)
    dt, times, (flows, heights) = _timed_median(lambda: pog.pog_solve_batch(costs, deltas, alphas, opts), warmup,
                                                steps)
    n = sum(v.n for v in vols)
    out = {"value": round(n / dt / 1e6, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 2),
           "ms_all_steps": [round(t * 1e3, 1) for t in times], "volumes": len(vols), "nodes": n,
           "driver": "one solve of the disjoint union of the volumes; finished volumes leave at each global relabel",
           "params": params}
    gold = os.path.join(ROOT, "tests", "golden", "batch.json")
    if os.path.exists(gold):
        with open(gold) as f:
            ref = json.load(f)["volumes"]
        ok = 0
        for r, fl, h in zip(ref, flows, heights):
            hh = hashlib.sha256(h.cpu().numpy().astype(np.int32).tobytes()).hexdigest()
            ok += int(r["flow"] == fl and r["heights_sha256"] == hh)
        out["oracle_parity"] = f"{ok}/{len(ref)} volumes bit-exact"
    return out


def differentiable_leg(args, warmup=1, steps=3):
    """16 float volumes of 128^3: quantise + energy solve + loss-augmented solve (warm,
    from the energy solve's state) + structured-hinge loss + one-hot backward, aggregate
    Mnodes/s of the volumes processed (median of `steps`); every energy, loss and surface
    checked against the oracle's stored values (tests/golden/diff.json)."""
    import hashlib

    import torch

    from paper_2601_17026_gb300 import autograd as pag
    from paper_2601_17026_gb300 import synth

    fc = torch.from_numpy(synth.diff_volumes_f32()).cuda()
    B, X, Y, Z = fc.shape
    ht = torch.from_numpy(synth.diff_target(B, X)).cuda()

    def step():
        x = fc.clone().requires_grad_(True)
        e, loss, h, hh = pag.solve_with_hinge(x, ht, synth.DIFF_DELTA, synth.DIFF_ALPHA, synth.DIFF_MARGIN)
        (e.sum() + loss.sum()).backward()
        return e, loss, h, hh, x.grad

    dt, times, (e, loss, h, hh, grad) = _timed_median(step, warmup, steps)
    out = {"value": round(B * X * Y * Z / dt / 1e6, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 2),
           "ms_all_steps": [round(t * 1e3, 1) for t in times],
           "step": "forward (energy solve + warm loss-augmented solve + hinge) + backward", "volumes": B}
    gold = os.path.join(ROOT, "tests", "golden", "diff.json")
    if os.path.exists(gold):
        with open(gold) as f:
            ref = json.load(f)["volumes"]
        sha = lambda t: hashlib.sha256(t.cpu().numpy().astype(np.int32).tobytes()).hexdigest()  # noqa: E731
        ok = sum(int(e[b].item() * 1024 == r["energy"] and loss[b].item() * 1024 == r["hinge_q"]
                     and sha(h[b]) == r["heights_sha256"] and sha(hh[b]) == r["aug_heights_sha256"])
                 for b, r in enumerate(ref))
        zs = torch.arange(Z, device="cuda", dtype=torch.int32)
        want = (h[..., None] == zs).float() + (ht[..., None] == zs).float() - (hh[..., None] == zs).float()
        out["oracle_parity"] = (f"{ok}/{len(ref)} volumes bit-exact (energy, hinge, both surfaces); gradient "
                                f"{'exact' if torch.equal(grad, want) else 'DIFFERS'}")
    return out


def narrow_band_leg(args, warmup=1, steps=3):
    """The narrow band of the 512x512x384 volume around 64 landmarks on its central
    horizon (stick 16, band factor 2: 65 rows, 17.0M band nodes): band construction +
    solve + image heights, Mnodes/s of band nodes (median of `steps`). The band volume, its
    center surface, the band solve's flow and surface and the image heights are checked bit
    for bit against the oracle's stored results (tests/golden/band.json)."""
    import hashlib

    import torch

    from paper_2601_17026_gb300 import autotune, pog, synth

    spec = synth.spec_seismic()
    cost_np = synth.horizon_cost(spec)
    lm_np = synth.horizon_landmarks(spec, 8)
    cost = torch.from_numpy(cost_np).cuda()
    lm = torch.from_numpy(lm_np).cuda()
    stick, factor, outside = synth.BAND_STICK, synth.BAND_FACTOR, synth.BAND_OUTSIDE
    half = stick * factor
    X, Y = cost.shape[:2]
    Zb = 2 * half + 1
    opts = pog.make_options(**autotune.tuned_params(X, Y, Zb, 3, 50))

    def step():
        b, c = pog.pog_narrow_band(cost, lm, stick, factor, outside)
        with pog.pog_build(b, 3, 50, opts) as g:
            flow = pog.pog_maxflow(g)
            hb = pog.pog_surface(g)
            himg = pog.pog_band_heights(hb, c, half)
        return b, c, flow, hb, himg

    dt, times, (b, c, flow, hb, himg) = _timed_median(step, warmup, steps)
    n = X * Y * Zb
    out = {"value": round(n / dt / 1e6, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 2),
           "ms_all_steps": [round(t * 1e3, 1) for t in times], "band_nodes": n, "rows": Zb, "landmarks": len(lm_np),
           "step": "band construction + solve (build, max-flow, surface) + image heights"}
    gold = os.path.join(ROOT, "tests", "golden", "band.json")
    if os.path.exists(gold):
        with open(gold) as fh:
            ref = json.load(fh)
        sha = lambda t: hashlib.sha256(t.cpu().numpy().astype(np.int32).tobytes()).hexdigest()  # noqa: E731
        band_ok = sha(b) == ref["band_sha256"] and sha(c) == ref["center_sha256"]
        solve_ok = (flow == ref["flow"] and sha(hb) == ref["heights_sha256"]
                    and sha(himg) == ref["image_heights_sha256"])
        out["oracle_parity"] = (f"band volume {'bit-exact' if band_ok else 'DIFFERS'} vs the oracle's construction; "
                                f"band solve {'bit-exact' if solve_ok else 'DIFFERS'} vs the oracle's stored flow "
                                f"and surfaces")
    return out


def convex_sweep_model(f):
    """(layers d >= 1 with k_d > 0, out-arcs of an interior node, algorithmic bytes per listed
    node of one push/relabel step) of the convex solve with profile f(1..delta): the node's
    excess and label, each out-arc word and its far-end label, three atomic words."""
    f = np.asarray(f, dtype=np.int64)
    nl = int(np.count_nonzero(np.diff(np.concatenate([[0], f]), 2))) if f.size > 1 else 0
    arcs = 3 + 4 * (2 + int(f.size > 0 and f[0] > 0) + 2 * nl)
    return nl, arcs, 20 + 8 * arcs


def _energy_pairwise(cost, h, fv):
    """sum_col c(col, h) + sum over 4-neighbour pairs fv[|h_p - h_q|] (numpy, int64)."""
    h = h.astype(np.int64)
    e = int(np.take_along_axis(cost, h[:, :, None], axis=2).astype(np.int64).sum())
    return e + int(fv[np.abs(np.diff(h, axis=0))].sum() + fv[np.abs(np.diff(h, axis=1))].sum())


def convex_leg(args, warmup=1, steps=3):
    """Convex pairwise costs (the general proper-order graph: an edge interval of 10 vertices
    per adjacent column, delta 9, f(t) = 4 t^2) on the 256x256x128 layered-horizon volume
    through pog_solve_convex, Mnodes/s (median of `steps`). Checks: the two mid-size volumes
    of tests/golden/convex.json bit for bit against the oracle's stored results, and the
    full-size surface's energy, from its definition, equal to the energy the solve reports
    (flow - K)."""
    import hashlib

    import torch

    from paper_2601_17026_gb300 import pog, synth

    X, Y, Z = synth.CONVEX_SHAPE
    cost_np = synth.convex_cost(X, Y, Z)
    f = synth.convex_profile()
    delta = synth.CONVEX_DELTA
    cost = torch.from_numpy(cost_np).cuda()
    opts = pog.make_options(flags=pog.POG_FLAG_TIMING)
    dt, times, (flow, energy, h, st) = _timed_median(lambda: pog.pog_solve_convex(cost, delta, f, options=opts),
                                                     warmup, steps)
    n = X * Y * Z
    nl, arcs, per_node = convex_sweep_model(f)
    sweeps = max(int(st["sweeps"]), 1)
    scan = 8 * (n - X * Y)  # k_cv_collect: excess and label of every node above the bottom layer
    sweep_bytes = st["tiles_visited"] * per_node + sweeps * scan
    peak, peak_src = _peaks()
    achieved = sweep_bytes / (st["sweep_ms"] / 1e3) / 1e9 if st["sweep_ms"] > 0 else 0.0
    push_traffic = measured_traffic("k_cv_push_relabel", st["tiles_visited"] / sweeps)
    traffic = None if push_traffic is None else int(push_traffic + scan)
    fv = np.concatenate([[0], f])
    hn = h.cpu().numpy()
    e_def = _energy_pairwise(cost_np, hn, fv)
    out = {"value": round(n / dt / 1e6, 3), "unit": UNIT, "ms_per_step": round(dt * 1e3, 2),
           "ms_all_steps": [round(t * 1e3, 1) for t in times], "nodes": n, "delta": delta,
           "f": "4 t^2", "layers": nl + 1, "arcs_per_node": arcs,
           "solver": {k: st[k] for k in ("rounds", "sweeps", "bfs_passes", "cut_passes", "launches")},
           "listed_nodes": st["tiles_visited"],
           "kernel_ms": {"sweep": round(st["sweep_ms"], 1), "relabel": round(st["bfs_ms"], 1),
                         "cut": round(st["cut_ms"], 1), "build": round(st["build_ms"], 1)},
           "roofline": {"bound": "hbm", "kernel": "k_cv_collect + k_cv_push_relabel (one sweep)",
                        "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": traffic,
                        "traffic_ratio": None if traffic is None else round(traffic / (sweep_bytes / sweeps), 2),
                        "bytes_per_launch": int(sweep_bytes / sweeps), "avg_launch_ms": round(st["sweep_ms"] / sweeps, 4),
                        "peak_source": peak_src, "bytes_per_listed_node": per_node},
           "energy_identity": "holds" if e_def == energy else f"DIFFERS ({e_def} vs {energy})"}
    gold = os.path.join(ROOT, "tests", "golden", "convex.json")
    if os.path.exists(gold):
        with open(gold) as fh:
            ref = json.load(fh)["volumes"]
        ok = 0
        for r in ref:
            c = torch.from_numpy(synth.convex_cost(*r["shape"])).cuda()
            fl, en, hh, _ = pog.pog_solve_convex(c, r["delta"], np.array(r["f"], dtype=np.int64))
            sha = hashlib.sha256(hh.cpu().numpy().astype(np.int32).tobytes()).hexdigest()
            ok += int(fl == r["flow"] and en == r["energy"] and sha == r["heights_sha256"])
        out["oracle_parity"] = f"{ok}/{len(ref)} stored oracle volumes bit-exact"
    return out


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def _crop(vol, X, Y):
    from paper_2601_17026_gb300.synth import Volume

    return Volume(np.ascontiguousarray(vol.cost[:X, :Y, :]), vol.delta, vol.alpha)


def cpu_baseline(args, vol, sample_xy=32):
    """The oracle (explicit-edge Dinic, one core) on a bounded crop of the workload."""
    import oracle

    crop = _crop(vol, sample_xy, sample_xy)
    t = time.perf_counter()
    oracle.solve(crop.cost, crop.delta, crop.alpha)
    dt = time.perf_counter() - t
    nproc, model = host_cpu()
    return {"value": round(crop.n / dt / 1e6, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cores": nproc, "cpu_model": model,
            "sample": f"{sample_xy}x{sample_xy}x{vol.cost.shape[2]} crop (x,y < {sample_xy}) of the workload, "
                      f"{crop.n} nodes, {dt:.1f} s single-threaded explicit-edge Dinic"}


def cpu_baseline_batched(args, count=16, sample_xy=32):
    """The oracle on a thread pool of min(volumes, cores) threads over a bounded sample of
    the uneven batch: the x,y < 32 crops of its first `count` volumes."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    from paper_2601_17026_gb300 import synth

    vols = [_crop(v, sample_xy, sample_xy) for v in synth.batch_volumes(limit=count)]
    nproc, model = host_cpu()
    workers = max(1, min(len(vols), nproc))
    oracle.build()
    t = time.perf_counter()
    with ThreadPoolExecutor(workers) as ex:  # the oracle releases the GIL inside C
        list(ex.map(lambda v: oracle.solve(v.cost, v.delta, v.alpha), vols))
    dt = time.perf_counter() - t
    n = sum(v.n for v in vols)
    return {"value": round(n / dt / 1e6, 5), "unit": UNIT, "cores": workers, "kind": "oracle",
            "host_cores": nproc, "cpu_model": model,
            "sample": f"x,y < {sample_xy} crops of the first {len(vols)} volumes of the 64-volume batch "
                      f"({n} nodes), {dt:.1f} s on {workers} threads"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle

    vol = _workload(args.workload)
    crop = _crop(vol, 32, 32)
    oracle.build()
    for _ in range(args.warmup):
        oracle.solve(crop.cost[:8, :8], crop.delta, crop.alpha)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(crop.cost, crop.delta, crop.alpha)
    dt = time.perf_counter() - t
    value = crop.n * args.steps / dt / 1e6
    X, Y, Z = vol.cost.shape
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{X}x{Y}x{Z} layered-horizon volume, delta={vol.delta}, alpha={vol.alpha}",
                   "sample": "32x32 crop per step"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host_cores": host_cpu()[0], "cpu_model": host_cpu()[1],
                         "sample": f"32x32x{Z} crop of the workload ({crop.n} nodes) per step"},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="seismic", choices=["seismic", "seismic-crop", "medium", "small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps-per-relabel", type=int, default=None,
                    help="fix the sweeps per global relabel (0 = adaptive); default: the tuned value")
    ap.add_argument("--extras", dest="extras", action="store_true", default=True,
                    help="also time the batched and differentiable workloads (default)")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
