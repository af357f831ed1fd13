"""Serving loop for interactive density queries over resident event sets.

The paper's goal is near-real-time exploratory analysis: many density queries
(different grids and bandwidths) over the same event sets.  This module keeps
the event sets resident on the GPU and serves a stream of requests with
continuous batching: whenever the device is free, every queued request that fits
the memory budget (output grid bytes plus the batch's workspace estimate) is
admitted, in arrival order, into one ``stkde_compute_batch`` call; the next
batch is formed while the previous one runs.  Each request's grid is
bit-identical to computing it alone (the batched call guarantees it), so mixing
requests changes only their latency.

The scheduler is plain host logic over the library's C ABI; all density work
runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Sequence

import numpy as np


@dataclasses.dataclass(frozen=True)
class Request:
    """One density query: event set, grid (voxels and domain extent), bandwidths
    in voxels, and its arrival time in seconds from the start of the stream."""

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
               max_batch: int = 64) -> list[Request]:
    """Admits queued requests in arrival order while the batch's memory (its
    output grids plus a workspace estimate of 72 bytes per event of every
    request) stays within ``budget_bytes``.  The first request is always
    admitted, so an oversized request is served alone rather than starved."""
    batch, used = [], 0
    for r in queue:
        need = r.out_bytes + set_bytes(r.set_id)
        if batch and (used + need > budget_bytes or len(batch) >= max_batch):
            break
        batch.append(r)
        used += need
    return batch


def percentiles(lat_s: Sequence[float]) -> dict:
    a = np.sort(np.asarray(lat_s, dtype=np.float64)) * 1e3
    if a.size == 0:
        return {"p50_ms": math.nan, "p99_ms": math.nan, "max_ms": math.nan}
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "max_ms": float(a[-1])}


class Server:
    """Resident event sets plus a continuous-batching loop on one GPU."""

    WORKSPACE_BYTES_PER_EVENT = 72  # events, sort keys and scratch of a batch

    def __init__(self, sets: Sequence[np.ndarray], budget_bytes: int = 8 << 30,
                 form: str = "bf16x3", device: int = 0, max_batch: int = 64):
        import torch
        import paper_1705_09366_gb300 as pkg

        self.torch, self.pkg = torch, pkg
        self.device = device
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.sets = [torch.from_numpy(np.ascontiguousarray(s, dtype=np.float64)).to(f"cuda:{device}")
                     for s in sets]
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = pkg.Context(device=device, stream=self.stream, form=form)

    def set_bytes(self, set_id: int) -> int:
        return self.WORKSPACE_BYTES_PER_EVENT * int(self.sets[set_id].shape[0])

    def close(self):
        self.ctx.close()

    def _launch(self, batch: Sequence[Request]):
        torch = self.torch
        outs = [torch.empty((r.gx, r.gy, r.gt), dtype=torch.float32, device=f"cuda:{self.device}")
                for r in batch]
        probs = []
        for r, o in zip(batch, outs):
            pts = self.sets[r.set_id]
            probs.append(self.pkg.Problem(self.pkg._ptr(pts), int(pts.shape[0]),
                                          self.pkg.make_grid(r.gx, r.gy, r.gt, sres=r.sres, tres=r.tres),
                                          r.hs, r.ht, self.pkg._ptr(o)))
        with torch.cuda.stream(self.stream):
            self.pkg.stkde_compute_batch(self.ctx.handle, probs)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        return outs, ev

    def compute_alone(self, r: Request):
        """The request computed by itself (for the alone-vs-mix check)."""
        outs, ev = self._launch([r])
        ev.synchronize()
        self.ctx.synchronize()
        return outs[0]

    def run(self, requests: Sequence[Request], keep_outputs: Callable[[Request], bool] = lambda r: False):
        """Serves the stream in real time (arrivals relative to the start of the
        call); returns per-request latencies (completion - arrival), the batches
        and any outputs selected by ``keep_outputs``."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        lat = {}
        kept = {}
        batches = []
        inflight = None  # (batch, outputs, event)
        max_admitted = 0
        i = 0
        t0 = time.perf_counter()
        while i < len(pending) or queue or inflight is not None:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                i += 1
            if inflight is not None and inflight[2].query():
                done = time.perf_counter() - t0
                for r, o in zip(inflight[0], inflight[1]):
                    lat[r.rid] = done - r.arrival
                    if keep_outputs(r):
                        kept[r.rid] = o
                inflight = None
            if inflight is None and queue:
                batch = form_batch(queue, self.budget, self.set_bytes, self.max_batch)
                del queue[:len(batch)]
                admitted = sum(r.out_bytes + self.set_bytes(r.set_id) for r in batch)
                max_admitted = max(max_admitted, admitted)
                outs, ev = self._launch(batch)
                inflight = (batch, outs, ev)
                batches.append([r.rid for r in batch])
                continue
            if inflight is None and not queue and i < len(pending):
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.002)))
            else:
                time.sleep(0.0001)
        self.ctx.synchronize()
        wall = time.perf_counter() - t0
        stats = percentiles(list(lat.values()))
        stats.update({"requests": len(lat), "batches": len(batches),
                      "mean_batch": float(np.mean([len(b) for b in batches])) if batches else 0.0,
                      "grids_per_s": len(lat) / wall if wall > 0 else math.nan,
                      "wall_s": wall, "max_admitted_bytes": int(max_admitted),
                      "budget_bytes": self.budget})
        return stats, lat, batches, kept


def main(argv=None):
    import argparse
    import json

    from paper_1705_09366_gb300 import synth

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--form", default="bf16x3")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    sets = synth.resident_sets()
    srv = Server(sets, budget_bytes=int(a.budget_gb * (1 << 30)), form=a.form)
    warm = request_stream(8, 1000.0, len(sets), seed=a.seed + 99)
    srv.run(warm)
    reqs = request_stream(a.requests, a.rate, len(sets), seed=a.seed)
    stats, _, _, _ = srv.run(reqs)
    srv.close()
    stats.update({"rate_hz": a.rate, "form": a.form, "sets": [int(s.shape[0]) for s in sets]})
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
