#!/usr/bin/env python3
"""STKDE benchmark: voxel-point updates/s and ms per grid on GB300.

One step = one stkde_compute of the whole hot path (re-centre, binning sort,
bin bounds + gather, tile kernel writing every voxel) on a synthetic clustered
event set already resident in HBM.  Default workload: n = 2,000,000 events,
1024 x 1024 x 512 grid, hs = 25, ht = 20 voxels (the large configuration), in
the tensor bf16x3 form.  The L2 is flushed (256 MiB write) before every timed
step; the 2.1 GB output is also larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank computes its own instance (seed offset = rank): the
instances are independent, so scaling is weak and no collective touches the
data; the only collectives are the barrier and the max-over-ranks of the time.
``--impl reference`` times the FP64 CPU oracle (the paper has no GPU code) on a
bounded sample of tiles of the same workload.  ``--bandwidth adaptive`` gives
every event its own bandwidths (log-uniform in [h/spread, h*spread] around the
workload's pair) and times stkde_compute_adaptive instead; ``--bandwidth abramson``
takes them from stkde_abramson_bandwidths (a pilot density by Abramson's law).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1705_09366_gb300 import synth  # noqa: E402

METRIC = "STKDE voxel-updates/s & ms/grid vs plain GPU at stated err; serve p50/p99"
UNIT = "voxel-point updates/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
# error gates (max |gpu - oracle| / grid max after the tie slack); the one-product
# tf32 form is reported without a gate
ERR_GATE = {"bf16x3": 2e-5, "fp16x3": 1e-5, "tf32x3": 1e-5, "tf32x1": None, "fp32": 1e-5,
            "scatter": 1e-5}
PRODUCTS = {"bf16x3": 3, "fp16x3": 3, "tf32x3": 3, "tf32x1": 1, "fp32": 1, "scatter": 1}
DTYPE = {"bf16x3": "bf16", "fp16x3": "f16", "tf32x3": "tf32", "tf32x1": "tf32", "fp32": "f32",
         "scatter": "f32"}
TENSOR_FORMS = ("bf16x3", "fp16x3", "tf32x3", "tf32x1")
# nominal dense tensor rates relative to bf16 (2.25 PFLOP/s): tf32 1.1 PFLOP/s
NOMINAL_RATIO = {"bf16x3": 1.0, "fp16x3": 1.0, "tf32x3": 1.1 / 2.25, "tf32x1": 1.1 / 2.25}
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(synth.WORKLOADS), default="large")
    ap.add_argument("--form", default="bf16x3", choices=list(ERR_GATE))
    ap.add_argument("--compare", default="fp16x3,tf32x3,tf32x1,fp32,scatter",
                    help="other forms timed beside the main one ('' for none)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--bandwidth", choices=["fixed", "adaptive", "abramson"], default="fixed",
                    help="adaptive: per-event bandwidths log-uniform in [h/spread, h*spread]; "
                         "abramson: from a pilot density by Abramson's law, factors clamped "
                         "to [1/spread, spread]")
    ap.add_argument("--spread", type=float, default=2.0)
    ap.add_argument("--batch-count", type=int, default=64,
                    help="instances of the batched workload timed beside the main line (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving run reported beside the main line (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-load-requests", type=int, default=4000,
                    help="requests of a second serving run at --serve-load-rate (0: skip)")
    ap.add_argument("--serve-load-rate", type=float, default=800.0)
    ap.add_argument("--medium", type=int, default=1,
                    help="also time the medium workload in the main form (0: skip)")
    return ap.parse_args()


def workload_bandwidths(args, w, seed, ctx=None, pts=None):
    """(name, hs, ht): the workload's fixed pair, or per-event arrays (host).  The
    Abramson bandwidths come from the library (ctx, device events) or, without a
    context, from the FP64 oracle."""
    if args.bandwidth == "fixed":
        return w.name, w.hs, w.ht
    if args.bandwidth == "abramson":
        lo, hi = 1.0 / args.spread, args.spread
        if ctx is not None:
            hs, ht = ctx.abramson_bandwidths(pts, (w.gx, w.gy, w.gt), w.hs, w.ht, alpha=0.5,
                                             lam_min=lo, lam_max=hi)
            ctx.synchronize()
            hs, ht = hs.cpu().numpy(), ht.cpu().numpy()
        else:
            import oracle
            p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht)
            hs, ht, _ = oracle.abramson(w.points, p, alpha=0.5, lam_min=lo, lam_max=hi)
        return f"{w.name}-abramson-x{args.spread:g}", hs, ht
    hs, ht = synth.adaptive_bandwidths(w.n, w.hs, w.ht, spread=args.spread, seed=seed)
    return f"{w.name}-adaptive-x{args.spread:g}", hs, ht


def bandwidth_label(args):
    if args.bandwidth == "adaptive":
        return f"per event, log-uniform in [h/{args.spread:g}, h*{args.spread:g}]"
    if args.bandwidth == "abramson":
        return (f"per event, Abramson's law (alpha 1/2) on the fixed-pair pilot, factors in "
                f"[1/{args.spread:g}, {args.spread:g}]")
    return "fixed"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# ----------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------ CPU oracle ---

def tile_boxes(w, seed=0):
    """All 16 x 8 x gt tile boxes of the grid in a seeded random order."""
    nx, ny = (w.gx + 15) // 16, (w.gy + 7) // 8
    rng = np.random.default_rng(seed)
    order = rng.permutation(nx * ny)
    return [(int(c // ny) * 16, min(w.gx, int(c // ny) * 16 + 16), int(c % ny) * 8,
             min(w.gy, int(c % ny) * 8 + 8), 0, w.gt) for c in order]


def oracle_sample(w, seconds, seed=0, calib=None, bw=None, nthreads=0):
    """Times the FP64 oracle (Algorithm 2 on random tiles, all host cores) for
    about `seconds`, growing the sample in batches; returns (pairs, elapsed,
    boxes, results, seconds per box).  bw: per-event (hs, ht) arrays or None."""
    import oracle
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht, x0=w.x0, y0=w.y0, t0=w.t0, sres=w.sres,
                      tres=w.tres, nthreads=nthreads)
    boxes = tile_boxes(w, seed)
    done, pairs, elapsed, res = 0, 0, 0.0, []
    per_box = calib
    while done < len(boxes) and elapsed < seconds:
        if per_box is None:
            k = 16
        else:
            k = int(max(1, round((seconds - elapsed) / max(per_box, 1e-6))))
        sel = boxes[done:done + k]
        t = time.perf_counter()
        if bw is None:
            r, c = oracle.pb_boxes(w.points, p, sel, with_slack=True, pair_counts=True)
        else:
            r, c = oracle.pb_adaptive_boxes(w.points, bw[0], bw[1], p, sel, with_slack=True,
                                            pair_counts=True)
        dt = time.perf_counter() - t
        res.extend(r)
        pairs += int(c.sum())
        elapsed += dt
        done += len(sel)
        per_box = elapsed / done
    return pairs, elapsed, boxes[:done], res, per_box


# ------------------------------------------------------------- reference ---

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = synth.WORKLOADS[args.workload]()
    name, hs, ht = workload_bandwidths(args, w, 0)
    bw = None if args.bandwidth == "fixed" else (hs, ht)
    total_budget = 150.0
    per_step = max(1.0, total_budget / max(1, args.steps + args.warmup))
    _, _, _, _, per_box = oracle_sample(w, 0.5, bw=bw)
    vals = []
    ntiles = []
    for i in range(args.warmup + args.steps):
        pairs, dt, sel, _, _ = oracle_sample(w, per_step, seed=i, calib=per_box, bw=bw)
        if i >= args.warmup:
            vals.append((pairs, dt))
            ntiles.append(len(sel))
    pairs = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    value = pairs / secs
    cores = oracle.max_threads()
    tiles = int(round(statistics.mean(ntiles)))
    sample = (f"FP64 oracle (Algorithm 2) on {tiles} random 16x8x{w.gt} tiles per step of the "
              f"{name} workload, {cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "n": w.n, "grid": [w.gx, w.gy, w.gt], "hs": w.hs,
                   "ht": w.ht, "bandwidth": args.bandwidth, "sample": "tiles"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours ---

def code_only(src: str) -> str:
    """The source without // comments and blank lines: the key under which DRAM
    counters are recorded, so that edits to the prose do not void them."""
    lines = []
    for ln in src.splitlines():
        code = ln.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return "\n".join(lines)


def recorded_traffic(args):
    """DRAM bytes (read + write) of one tile-kernel launch from the committed ncu
    summary, if it was taken on this workload and form with the current kernel
    code (the source hashed without comments); else None."""
    if args.workload != "large" or args.form != "bf16x3" or args.bandwidth != "fixed":
        return None
    import hashlib
    prof = os.path.join(ROOT, "profiles", "tile_tc_large_dram.md")
    src = os.path.join(ROOT, "paper_1705_09366_gb300", "csrc", "tile_tc.cu")
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    with open(src) as f:
        sha = hashlib.sha256(code_only(f.read()).encode()).hexdigest()
    rec = {}
    with open(prof) as f:
        for ln in f:
            k, _, v = ln.strip().partition(":")
            if k in ("tile_tc_sha256_prefix", "traffic_bytes_per_launch"):
                rec[k] = v.strip()
    if not rec.get("tile_tc_sha256_prefix") or not sha.startswith(rec["tile_tc_sha256_prefix"]):
        return None
    try:
        return int(rec["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_ours(args):
    import torch
    import paper_1705_09366_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1705_09366_gb300 import replicas

    peaks, peaks_src = load_peaks()
    w = synth.WORKLOADS[args.workload](seed_offset=replicas.instance_offset(rank))
    adaptive = args.bandwidth != "fixed"
    dims = (w.gx, w.gy, w.gt)
    stream = torch.cuda.current_stream(dev)
    pts = torch.from_numpy(w.points).to(dev)
    with pkg.Context(device=local, stream=stream, form=args.form) as bctx:
        wname, hs_h, ht_h = workload_bandwidths(args, w, rank, bctx, pts)
    hs_d = torch.from_numpy(hs_h).to(dev) if adaptive else w.hs
    ht_d = torch.from_numpy(ht_h).to(dev) if adaptive else w.ht
    out = torch.empty(dims, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def compute(c, p, o, hs=hs_d, ht=ht_d):
        if adaptive:
            return c.compute_adaptive(p, dims, hs, ht, out=o)
        return c.compute(p, dims, hs, ht, out=o)

    ctx = pkg.Context(device=local, stream=stream, form=args.form, profile=False)
    if adaptive:
        updates = ctx.count_updates_adaptive(pts, dims, hs_d, ht_d)
    else:
        updates = ctx.count_updates(pts, dims, w.hs, w.ht)

    # ---- timed steps: device-resident inputs, L2 flushed before each step
    for _ in range(args.warmup):
        compute(ctx, pts, out)
    ctx.synchronize()
    launches_per_step = ctx.last_launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    barrier()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        compute(ctx, pts, out)
        ends[i].record(stream)
    barrier()
    clk = clocks.stop() if rank == 0 else None
    ctx.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # independent replicas: units of all ranks over the slowest rank's time
    value, total_s, _ = replicas.job_throughput(dist, float(updates) * args.steps,
                                                sum(step_ms) / 1000.0, dev)
    ms_per_step = 1000.0 * total_s / args.steps

    # ---- dominant kernel: library events around each phase (same stream)
    pctx = pkg.Context(device=local, stream=stream, form=args.form, profile=True)
    phases = []
    for i in range(args.steps):
        flush.fill_(float(i))
        compute(pctx, pts, out)
        phases.append(pctx.phase_times())
    pctx.synchronize()
    pctx.close()
    ph = np.array(phases)
    phase_ms = {name: float(ph[:, k].mean()) for k, name in
                enumerate(["recentre", "sort", "bounds_gather", "tile"][:ph.shape[1]])}
    tile_ms = phase_ms.get("tile", float("nan"))

    grid_bytes = 4 * w.gx * w.gy * w.gt
    prods = PRODUCTS[args.form]
    flops = 2.0 * prods * updates
    if args.form in TENSOR_FORMS:
        peak = peaks["bf16_tflops"] * NOMINAL_RATIO[args.form]
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "achieved": flops / (tile_ms * 1e-3) / 1e12, "peak": peak}
        roof["frac"] = roof["achieved"] / peak
        own = "bf16" if NOMINAL_RATIO[args.form] == 1.0 else \
            f"tf32 (= bf16 x {NOMINAL_RATIO[args.form]:.3f}, the nominal dense-rate ratio)"
        roof["note"] = (f"algorithmic FLOPs = 2 x {prods} products x {updates} voxel-point "
                        f"updates; peak = {peaks_src} dense {own} (burst)")
        # the same kernel against the FP32 CUDA-core roofline (one FMA per update)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_fma = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
        roof["frac_of_fp32_fma_roofline"] = (updates / fp32_fma) / (tile_ms * 1e-3)
    else:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = 2.0 * 128 * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s",
                "achieved": flops / (tile_ms * 1e-3) / 1e12, "peak": peak}
        roof["frac"] = roof["achieved"] / peak
        roof["note"] = f"peak = {sms} SMs x 128 FP32 lanes x 2 x max SM clock"
    hbm = grid_bytes / (tile_ms * 1e-3) / 1e9
    roof["hbm_write_gbs"] = hbm
    roof["hbm_frac_of_" + peaks_src] = hbm / peaks["hbm_gbs"]
    roof["traffic"] = recorded_traffic(args)
    roof["kernel_ms"] = tile_ms
    roof["roofline_ms"] = 1e3 * max(grid_bytes / (peaks["hbm_gbs"] * 1e9),
                                    (flops / (peak * 1e12)))

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if args.e2e_steps > 0:
        hpts = torch.from_numpy(w.points).pin_memory()
        hout = torch.empty(dims, dtype=torch.float32, pin_memory=True)
        hhs = torch.from_numpy(hs_h).pin_memory() if adaptive else w.hs
        hht = torch.from_numpy(ht_h).pin_memory() if adaptive else w.ht
        h2d = int(w.points.nbytes) + (int(hs_h.nbytes + ht_h.nbytes) if adaptive else 0)
        compute(ctx, hpts, hout, hhs, hht)
        ctx.synchronize()
        barrier()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            compute(ctx, hpts, hout, hhs, hht)
            ctx.synchronize()
        barrier()
        e2e_v, e2e_s, _ = replicas.job_throughput(dist, float(updates) * args.e2e_steps,
                                                  time.perf_counter() - t, dev)
        e2e = {"value": e2e_v, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": grid_bytes,
               "ms_per_step": 1e3 * e2e_s / args.e2e_steps}
        del hout, hpts

    # ---- other forms on the same input (rank 0, N = 1)
    def form_entry(f, ms, tms):
        e = {"ms_per_grid": ms, "updates_per_s": updates / (ms * 1e-3), "tile_kernel_ms": tms}
        if f in TENSOR_FORMS and tms == tms:
            fpk = peaks["bf16_tflops"] * NOMINAL_RATIO[f]
            e["tensor_tflops"] = 2.0 * PRODUCTS[f] * updates / (tms * 1e-3) / 1e12
            e["frac_of_own_peak"] = e["tensor_tflops"] / fpk
        return e

    forms = {args.form: form_entry(args.form, ms_per_step, tile_ms)}
    forms[args.form]["updates_per_s"] = value / max(world, 1)
    if rank == 0 and world == 1 and args.compare:
        for f in [x for x in args.compare.split(",")
                  if x and x != args.form and not (adaptive and x in ("scatter", "tf32x3", "tf32x1"))]:
            fo = torch.empty(dims, dtype=torch.float32, device=dev)
            with pkg.Context(device=local, stream=stream, form=f) as fc:
                reps = 1 if f == "scatter" else 3
                compute(fc, pts, fo)
                fc.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                tot = 0.0
                for i in range(reps):
                    flush.fill_(float(i))
                    s0.record(stream)
                    compute(fc, pts, fo)
                    s1.record(stream)
                    fc.synchronize()
                    tot += s0.elapsed_time(s1)
            with pkg.Context(device=local, stream=stream, form=f, profile=True) as pc:
                flush.fill_(0.5)
                compute(pc, pts, fo)
                pt = pc.phase_times()
                pc.synchronize()
            forms[f] = form_entry(f, tot / reps, pt[3] if len(pt) > 3 else float("nan"))
            forms[f]["_out"] = fo

    # ---- the medium workload in the main form (rank 0, N = 1)
    medium = None
    if rank == 0 and world == 1 and args.medium and not adaptive:
        medium = run_medium(pkg, torch, dev, stream, args.form, peaks, peaks_src, flush)

    # ---- CPU oracle baseline + error against it on the sampled tiles (rank 0, N = 1)
    cpu = None
    errs = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        if medium is not None:
            medium_error(medium)
        import oracle
        pairs, dt, boxes, res, _ = oracle_sample(w, args.cpu_seconds, seed=rank,
                                                 bw=(hs_h, ht_h) if adaptive else None)
        cores = oracle.max_threads()
        cpu = {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle (Algorithm 2) on {len(boxes)} random 16x8x{w.gt} tiles "
                         f"of the {wname} workload ({pairs} updates, {dt:.1f} s)"}
        # one core, for comparison with the paper's sequential runs (Table 3)
        p1, dt1, b1, _, _ = oracle_sample(w, min(3.0, args.cpu_seconds), seed=rank + 1,
                                          bw=(hs_h, ht_h) if adaptive else None, nthreads=1)
        cpu["single_core"] = {"value": p1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{len(b1)} tiles, {p1} updates, {dt1:.1f} s"}
        scale = max(r.max() for r, _ in res)
        for f, buf in [(args.form, out)] + [(k, v["_out"]) for k, v in forms.items() if "_out" in v]:
            worst = 0.0
            for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, res):
                got = buf[x0:x1, y0:y1, t0:t1].double().cpu().numpy()
                ex = np.maximum(np.abs(got - ref) - slack, 0.0).max()
                worst = max(worst, float(ex / scale))
            errs[f] = worst
            forms[f]["max_rel_err"] = worst
            forms[f]["err_gate"] = ERR_GATE[f] if ERR_GATE[f] is not None else "report only"
    for v in forms.values():
        v.pop("_out", None)
    if medium is not None:
        medium.pop("_out", None)

    # ---- batched workload and serving loop (rank 0, N = 1)
    batch = serve = serve_load = tune = None
    if rank == 0 and world == 1 and args.medium and not adaptive:
        tune = run_tune(pkg, torch, dev)
    if rank == 0 and world == 1 and args.batch_count > 0:
        batch = run_batch(pkg, torch, args.form, args.batch_count)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        serve = run_serve(args.form, args.serve_requests, args.serve_rate)
    if rank == 0 and world == 1 and args.serve_load_requests > 0:
        serve_load = run_serve(args.form, args.serve_load_requests, args.serve_load_rate)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.form],
            "data": "synthetic",
            "config": {"workload": wname, "n": w.n, "grid": [w.gx, w.gy, w.gt], "hs": w.hs,
                       "ht": w.ht, "bandwidth": bandwidth_label(args),
                       "form": args.form, "updates_per_grid": updates,
                       "l2": "flushed before each step (256 MiB write); output 2.1 GB > L2",
                       "parallelism": f"{world} independent instance(s), one per GPU"},
            "roofline": roof,
            "phase_ms": phase_ms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "forms": forms,
            "medium": medium,
            "batch": batch,
            "tune": tune,
            "serve": serve,
            "serve_load": serve_load,
            "max_rel_err": errs.get(args.form),
            "peaks": peaks_src,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def densest_tiles(w, k):
    """The k 16 x 8 x gt tile boxes holding the most events (input statistics)."""
    cx = np.floor((w.points[:, 0] - w.x0) / w.sres / 16).astype(np.int64)
    cy = np.floor((w.points[:, 1] - w.y0) / w.sres / 8).astype(np.int64)
    nx, ny = (w.gx + 15) // 16, (w.gy + 7) // 8
    ok = (cx >= 0) & (cx < nx) & (cy >= 0) & (cy < ny)
    h = np.bincount(cx[ok] * ny + cy[ok], minlength=nx * ny)
    return [(int(c // ny) * 16, min(w.gx, int(c // ny) * 16 + 16), int(c % ny) * 8,
             min(w.gy, int(c % ny) * 8 + 8), 0, w.gt) for c in np.argsort(h)[::-1][:k]]


def run_medium(pkg, torch, dev, stream, form, peaks, peaks_src, flush, steps=10):
    """The medium workload (n = 200,000, 512 x 512 x 256, hs 10, ht 8) in the main
    form: ms per grid with the L2 flushed before each step (CUDA events), the
    tile kernel's time from the library's phase events, its output write rate
    and the fraction of the HBM floor (the 268 MB grid written once at the
    measured copy bandwidth).  The grid is kept (key "_out") for medium_error."""
    w = synth.medium()
    dims = (w.gx, w.gy, w.gt)
    pts = torch.from_numpy(w.points).to(dev)
    out = torch.empty(dims, dtype=torch.float32, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with pkg.Context(device=dev.index, stream=stream, form=form) as c:
        updates = c.count_updates(pts, dims, w.hs, w.ht)
        for _ in range(3):
            c.compute(pts, dims, w.hs, w.ht, out=out)
        c.synchronize()
        for i in range(steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            c.compute(pts, dims, w.hs, w.ht, out=out)
            ends[i].record(stream)
        c.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in zip(starts, ends))
    tiles = []
    with pkg.Context(device=dev.index, stream=stream, form=form, profile=True) as c:
        for i in range(steps):
            flush.fill_(float(i))
            c.compute(pts, dims, w.hs, w.ht, out=out)
            tiles.append(c.phase_times()[3])
        c.synchronize()
    tile_ms = statistics.mean(tiles)
    grid_bytes = 4 * w.gx * w.gy * w.gt
    floor_ms = 1e3 * grid_bytes / (peaks["hbm_gbs"] * 1e9)
    res = {"workload": w.name, "form": form, "updates_per_grid": int(updates), "ms_per_grid": ms,
           "updates_per_s": updates / (ms * 1e-3), "tile_kernel_ms": tile_ms,
           "hbm_write_gbs": grid_bytes / (tile_ms * 1e-3) / 1e9,
           "hbm_floor_ms": floor_ms, "frac_of_hbm_floor": floor_ms / tile_ms,
           "peak_source": peaks_src, "l2": "flushed before each step (256 MiB write)"}
    if form in TENSOR_FORMS:
        res["tensor_tflops"] = 2.0 * PRODUCTS[form] * updates / (tile_ms * 1e-3) / 1e12
    res["_out"] = out
    return res


def medium_error(medium):
    """Max error of the medium grid against the FP64 oracle on 24 sampled tiles
    (the 8 densest, 16 random), part of the CPU-oracle leg."""
    import oracle
    w = synth.medium()
    out = medium["_out"]
    rng = np.random.default_rng(7)
    boxes = densest_tiles(w, 8)
    allb = tile_boxes(w, seed=7)
    for k in rng.permutation(len(allb))[:16]:
        if allb[k] not in boxes:
            boxes.append(allb[k])
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht)
    refs = oracle.pb_boxes(w.points, p, boxes, with_slack=True)
    scale = max(r.max() for r, _ in refs)
    worst = 0.0
    for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, refs):
        got = out[x0:x1, y0:y1, t0:t1].double().cpu().numpy()
        worst = max(worst, float(np.maximum(np.abs(got - ref) - slack, 0.0).max() / scale))
    f = medium["form"]
    medium["max_rel_err"] = worst
    medium["err_gate"] = ERR_GATE[f] if ERR_GATE[f] is not None else "report only"
    medium["err_sample"] = f"{len(boxes)} tiles of 16x8x{w.gt}"


def run_batch(pkg, torch, form, count):
    """The batched workload: `count` uneven instances in one stkde_compute_batch
    call against the same problems in one stkde_compute call each, and the batch
    captured once into a CUDA graph and replayed (CUDA events, 3 repetitions after
    2 warm-up batches, no L2 flush: the instances are small)."""
    ws = synth.batched(count=count)
    pts = [torch.from_numpy(w.points).cuda() for w in ws]
    outs = [torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda") for w in ws]
    probs = [(p, (w.gx, w.gy, w.gt), w.hs, w.ht, o) for p, w, o in zip(pts, ws, outs)]
    stream = torch.cuda.Stream()  # capture needs a stream other than the legacy one
    with pkg.Context(stream=stream, form=form) as c:
        for _ in range(2):
            c.compute_batch(probs)
        c.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(3):
            c.compute_batch(probs)
        s1.record(stream)
        c.synchronize()
        t_batch = s0.elapsed_time(s1) / 3
        launches = c.last_launch_count()
        s0.record(stream)
        for _ in range(3):
            for p, w, o in zip(pts, ws, outs):
                c.compute(p, (w.gx, w.gy, w.gt), w.hs, w.ht, out=o)
        s1.record(stream)
        c.synchronize()
        t_single = s0.elapsed_time(s1) / 3
        # the batch as a CUDA graph: captured once, replayed
        c.compute_batch(probs)
        c.synchronize()
        direct = [o.clone() for o in outs]
        g = torch.cuda.CUDAGraph()
        # no garbage collection inside the capture: destroying stray CUDA objects
        # there would invalidate a global-mode capture
        gc.collect()
        gc.disable()
        try:
            with torch.cuda.graph(g, stream=stream):
                c.compute_batch(probs)
        finally:
            gc.enable()
        with torch.cuda.stream(stream):  # replays run on torch's current stream
            for o in outs:
                o.fill_(float("nan"))
            g.replay()
            stream.synchronize()
            identical = all(torch.equal(o, d) for o, d in zip(outs, direct))
            s0.record(stream)
            for _ in range(3):
                g.replay()
            s1.record(stream)
            stream.synchronize()
        t_graph = s0.elapsed_time(s1) / 3
        # host time to enqueue one batch (what the graph removes)
        torch.cuda.synchronize()
        t = time.perf_counter()
        c.compute_batch(probs)
        t_enqueue = 1e3 * (time.perf_counter() - t)
        c.synchronize()
        updates = sum(c.count_updates(p, (w.gx, w.gy, w.gt), w.hs, w.ht) for p, w in zip(pts, ws))
    # the fp32 form's batch (one tile launch over all problems), one warm-up, two timed
    fp32_ms = None
    if form != "fp32":
        with pkg.Context(stream=stream, form="fp32") as c:
            c.compute_batch(probs)
            c.synchronize()
            s0.record(stream)
            for _ in range(2):
                c.compute_batch(probs)
            s1.record(stream)
            c.synchronize()
            fp32_ms = s0.elapsed_time(s1) / 2
    return {"workload": f"{count} uneven instances (n log-uniform 1e3..5e5, grids 64^3..512x512x128)",
            "form": form,
            "events": int(sum(w.n for w in ws)), "voxels": int(sum(w.gx * w.gy * w.gt for w in ws)),
            "updates": int(updates), "ms_per_batch": t_batch, "ms_single_calls": t_single,
            "ms_per_batch_graph_replay": t_graph, "graph_replay_bit_identical": identical,
            "host_enqueue_ms": t_enqueue, "fp32_ms_per_batch": fp32_ms,
            "updates_per_s": updates / (t_batch * 1e-3), "launches_per_batch": launches}


def run_tune(pkg, torch, dev):
    """The autotuner on the medium workload (accuracy target 2e-5): every candidate
    (form x bin slab) timed on the problem, the winner, and the default
    configuration's time from the same table (no L2 flush between repetitions)."""
    from paper_1705_09366_gb300 import autotune

    w = synth.medium()
    pts = torch.from_numpy(w.points).to(dev)
    dims = (w.gx, w.gy, w.gt)
    t = autotune.Tuner(device=dev.index or 0, reps=3)
    try:
        cfg, key = t.config(pts, dims, w.hs, w.ht)
        e = t.table.entries[key]
    finally:
        t.close()
    return {"workload": w.name, "candidates": len(e["timings"]), "chosen": {"form": cfg[0], "slab": cfg[1]},
            "chosen_ms": e["ms"], "default_ms": e["timings"].get("bf16x3/0"), "timings_ms": e["timings"]}


def run_serve(form, n_requests, rate):
    """The serving loop over the resident sets: seeded Poisson arrivals, continuous
    batching; latency = completion - arrival."""
    from paper_1705_09366_gb300 import serve as srvmod

    sets = synth.resident_sets()
    srv = srvmod.Server(sets, form=form)
    srv.run(srvmod.request_stream(8, 1000.0, len(sets), seed=99))
    stats, _, _, _ = srv.run(srvmod.request_stream(n_requests, rate, len(sets), seed=0))
    srv.close()
    stats.update({"rate_hz": rate, "offered": n_requests, "sets": [int(s.shape[0]) for s in sets]})
    stats["dropped"] = len(stats["dropped"])
    return stats


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
