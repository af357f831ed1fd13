"""Serving loop for interactive density queries over resident event sets.

The paper's goal is near-real-time exploratory analysis: many density queries
(different grids and bandwidths) over the same event sets.  This module keeps
the event sets resident on the GPU and serves a stream of requests with
continuous batching: a small number of slots, each with its own library context
(workspace) and CUDA stream, run batches concurrently.  Whenever a slot is free,
the queued requests that fit the memory available right now -- free device
memory (cudaMemGetInfo) less a reserve, and at most the configured cap less the
bytes already in flight -- are admitted, in arrival order, into one
``stkde_compute_batch`` call on that slot's stream; requests that arrive while
others run join the next free slot, so batches overlap on the device (the small
kernels of one batch run beside another batch's tile kernel, and a tile kernel
of few tiles leaves most SMs to the others).  Each batch is bracketed by CUDA
events, from which the overlap of batches on the device is measured.

Each request's grid is bit-identical to computing it alone (the batched call
guarantees it, whatever runs beside it), so batching changes only latency.  A
queued request can be cancelled, or carry a deadline after which it is dropped
unserved (a request already on the device always completes).

The scheduler is plain host logic over the library's C ABI; all density work
runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Optional, Sequence

import numpy as np


@dataclasses.dataclass(frozen=True)
class Request:
    """One density query: event set, grid (voxels and domain extent), bandwidths
    in voxels, its arrival time in seconds from the start of the stream, and an
    optional deadline (seconds after arrival) by which it must be admitted."""

    rid: int
    set_id: int
    gx: int
    gy: int
    gt: int
    sres: float
    tres: float
    hs_vox: float
    ht_vox: float
    arrival: float
    deadline: Optional[float] = None

    @property
    def out_bytes(self) -> int:
        return 4 * self.gx * self.gy * self.gt

    @property
    def hs(self) -> float:
        return self.hs_vox * self.sres

    @property
    def ht(self) -> float:
        return self.ht_vox * self.tres


def request_stream(n_requests: int, rate_hz: float, n_sets: int, seed: int,
                   domain=(512.0, 512.0, 256.0)) -> list[Request]:
    """Seeded Poisson arrivals; each request picks a resident set, a grid with
    G_x = G_y in {128, 256, 512} and G_t in {128, 256} over the fixed domain
    (sres = domain_x / G_x, tres = domain_t / G_t), and bandwidths hs in {5, 10,
    20}, ht in {4, 8, 16} voxels."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_requests):
        gxy = int(rng.choice([128, 256, 512]))
        gt = int(rng.choice([128, 256]))
        out.append(Request(i, int(rng.integers(0, n_sets)), gxy, gxy, gt, domain[0] / gxy,
                           domain[2] / gt, float(rng.choice([5.0, 10.0, 20.0])),
                           float(rng.choice([4.0, 8.0, 16.0])), float(t[i])))
    return out


def form_batch(queue: Sequence[Request], budget_bytes: int, set_bytes: Callable[[int], int],
               max_batch: int = 64, force_first: bool = True) -> list[Request]:
    """Admits queued requests in arrival order while the batch's memory (its
    output grids plus a workspace estimate of 72 bytes per event of every
    request) stays within ``budget_bytes``; admission stops at the first request
    that does not fit, so arrival order is kept.  With ``force_first`` the first
    request is admitted whatever its size (nothing else is on the device), so an
    oversized request is served alone rather than starved."""
    batch, used = [], 0
    for r in queue:
        need = r.out_bytes + set_bytes(r.set_id)
        if len(batch) >= max_batch:
            break
        if used + need > budget_bytes and (batch or not force_first):
            break
        batch.append(r)
        used += need
    return batch


def expire(queue: list[Request], now: float, cancelled: set) -> list[Request]:
    """Removes from ``queue`` (in place) the cancelled requests and those whose
    deadline has passed; returns the removed ones."""
    keep, gone = [], []
    for r in queue:
        late = r.deadline is not None and now > r.arrival + r.deadline
        (gone if (r.rid in cancelled or late) else keep).append(r)
    queue[:] = keep
    return gone


def percentiles(lat_s: Sequence[float]) -> dict:
    a = np.sort(np.asarray(lat_s, dtype=np.float64)) * 1e3
    if a.size == 0:
        return {"p50_ms": math.nan, "p99_ms": math.nan, "max_ms": math.nan}
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "max_ms": float(a[-1])}


def overlap(intervals: Sequence[tuple]) -> dict:
    """Concurrency of [start, end) intervals: the largest number active at once
    and the total time (same unit) during which at least two are active."""
    pts = sorted([(s, 1) for s, _ in intervals] + [(e, -1) for _, e in intervals],
                 key=lambda x: (x[0], x[1]))
    active, peak, both, last = 0, 0, 0.0, None
    for t, d in pts:
        if last is not None and active >= 2:
            both += t - last
        active += d
        peak = max(peak, active)
        last = t
    return {"max_concurrent": peak, "overlap_time": both}


class Server:
    """Resident event sets plus a continuous-batching loop on one GPU."""

    WORKSPACE_BYTES_PER_EVENT = 72  # events, sort keys and scratch of a batch

    def __init__(self, sets: Sequence[np.ndarray], budget_bytes: int = 8 << 30,
                 form: str = "bf16x3", device: int = 0, max_batch: int = 64, slots: int = 3,
                 reserve_bytes: int = 1 << 30):
        import torch
        import paper_1705_09366_gb300 as pkg

        self.torch, self.pkg = torch, pkg
        self.device = device
        self.budget = int(budget_bytes)
        self.reserve = int(reserve_bytes)
        self.max_batch = int(max_batch)
        self.sets = [torch.from_numpy(np.ascontiguousarray(s, dtype=np.float64)).to(f"cuda:{device}")
                     for s in sets]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.ctxs = [pkg.Context(device=device, stream=s, form=form) for s in self.streams]
        self.cancelled: set = set()
        self.inflight_bytes = 0  # bytes of the batches on the device now (run() keeps it)

    def set_bytes(self, set_id: int) -> int:
        return self.WORKSPACE_BYTES_PER_EVENT * int(self.sets[set_id].shape[0])

    def batch_bytes(self, batch: Sequence[Request]) -> int:
        return sum(r.out_bytes + self.set_bytes(r.set_id) for r in batch)

    def cancel(self, rid: int) -> None:
        """Drops request ``rid`` if it has not been admitted yet."""
        self.cancelled.add(rid)

    def free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return int(free)

    def admission_budget(self, inflight_bytes: int) -> int:
        """Bytes a new batch may take now: free device memory less the reserve,
        and at most the cap less the bytes already in flight."""
        return max(0, min(self.free_bytes() - self.reserve, self.budget - inflight_bytes))

    def close(self):
        for c in self.ctxs:
            c.close()

    def _launch(self, slot: int, batch: Sequence[Request]):
        torch = self.torch
        stream = self.streams[slot]
        with torch.cuda.stream(stream):
            outs = [torch.empty((r.gx, r.gy, r.gt), dtype=torch.float32, device=f"cuda:{self.device}")
                    for r in batch]
        probs = []
        for r, o in zip(batch, outs):
            pts = self.sets[r.set_id]
            probs.append(self.pkg.Problem(self.pkg._ptr(pts), int(pts.shape[0]),
                                          self.pkg.make_grid(r.gx, r.gy, r.gt, sres=r.sres, tres=r.tres),
                                          r.hs, r.ht, self.pkg._ptr(o)))
        begin, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            begin.record(stream)
            self.pkg.stkde_compute_batch(self.ctxs[slot].handle, probs)
            end.record(stream)
        return outs, begin, end

    def compute_alone(self, r: Request):
        """The request computed by itself (for the alone-vs-mix check)."""
        outs, _, end = self._launch(0, [r])
        end.synchronize()
        self.ctxs[0].synchronize()
        return outs[0]

    def run(self, requests: Sequence[Request], keep_outputs: Callable[[Request], bool] = lambda r: False,
            on_arrival: Optional[Callable[["Server", Request], None]] = None):
        """Serves the stream in real time (arrivals relative to the start of the
        call); returns statistics, per-request latencies (completion - arrival),
        the batches (request ids) and any outputs selected by ``keep_outputs``.
        ``on_arrival`` is called for each request as it arrives (it may cancel
        requests).  Dropped requests (cancelled or past their deadline before
        admission) have no latency; their ids are in stats["dropped"]."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        lat, kept, batches, dropped = {}, {}, [], []
        inflight: list = [None] * len(self.ctxs)  # per slot: (batch, outs, begin, end, bytes)
        intervals_ev = []
        max_admitted = 0
        i = 0
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        while i < len(pending) or queue or any(f is not None for f in inflight):
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                if on_arrival is not None:
                    on_arrival(self, pending[i])
                i += 1
            dropped += [r.rid for r in expire(queue, now, self.cancelled)]
            # retire finished batches
            for s, f in enumerate(inflight):
                if f is not None and f[3].query():
                    done = time.perf_counter() - t0
                    for r, o in zip(f[0], f[1]):
                        lat[r.rid] = done - r.arrival
                        if keep_outputs(r):
                            kept[r.rid] = o
                    inflight[s] = None
            self.inflight_bytes = sum(f[4] for f in inflight if f is not None)
            # admit into free slots while memory allows
            launched = False
            for s in range(len(inflight)):
                if inflight[s] is not None or not queue:
                    continue
                busy = sum(f[4] for f in inflight if f is not None)
                nothing_running = all(f is None for f in inflight)
                batch = form_batch(queue, self.admission_budget(busy), self.set_bytes, self.max_batch,
                                   force_first=nothing_running)
                if not batch:
                    break
                del queue[:len(batch)]
                nbytes = self.batch_bytes(batch)
                max_admitted = max(max_admitted, busy + nbytes)
                outs, begin, end = self._launch(s, batch)
                inflight[s] = (batch, outs, begin, end, nbytes)
                self.inflight_bytes = busy + nbytes
                intervals_ev.append((begin, end))
                batches.append([r.rid for r in batch])
                launched = True
            if launched:
                continue
            if all(f is None for f in inflight) and not queue and i < len(pending):
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.002)))
            else:
                time.sleep(0.0001)
        for c in self.ctxs:
            c.synchronize()
        wall = time.perf_counter() - t0
        intervals = [(ref.elapsed_time(b) * 1e-3, ref.elapsed_time(e) * 1e-3) for b, e in intervals_ev]
        ov = overlap(intervals)
        stats = percentiles(list(lat.values()))
        stats.update({"requests": len(lat), "dropped": sorted(dropped), "batches": len(batches),
                      "mean_batch": float(np.mean([len(b) for b in batches])) if batches else 0.0,
                      "grids_per_s": len(lat) / wall if wall > 0 else math.nan,
                      "wall_s": wall, "max_admitted_bytes": int(max_admitted),
                      "budget_bytes": self.budget, "slots": len(self.ctxs),
                      "max_concurrent_batches": ov["max_concurrent"],
                      "overlap_s": ov["overlap_time"],
                      "device_busy_s": float(sum(e - b for b, e in intervals))})
        return stats, lat, batches, kept


def main(argv=None):
    import argparse
    import json

    from paper_1705_09366_gb300 import synth

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--form", default="bf16x3")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    sets = synth.resident_sets()
    srv = Server(sets, budget_bytes=int(a.budget_gb * (1 << 30)), form=a.form, slots=a.slots)
    warm = request_stream(8, 1000.0, len(sets), seed=a.seed + 99)
    srv.run(warm)
    reqs = request_stream(a.requests, a.rate, len(sets), seed=a.seed)
    stats, _, _, _ = srv.run(reqs)
    srv.close()
    stats.update({"rate_hz": a.rate, "form": a.form, "sets": [int(s.shape[0]) for s in sets]})
    stats["dropped"] = len(stats["dropped"])
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
