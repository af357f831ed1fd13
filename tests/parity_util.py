"""Helpers shared by the GPU parity tests (no STKDE arithmetic here)."""
from __future__ import annotations

import contextlib
import gc

import numpy as np

# Gates from the accuracy targets: max |gpu - oracle| / max(oracle), after the
# binary32 tie slack of the oracle (pairs on the cylinder wall may go either way).
TOL = {"fp32": 1e-5, "bf16x3": 2e-5, "fp16x3": 1e-5, "scatter": 1e-5, "tf32x3": 1e-5}
# the one-product tf32 form is reported, not gated: about 2^-11 per term; this
# bound only catches a broken kernel
REPORT_ONLY_BOUND = {"tf32x1": 2e-3}


def excess_error(got, ref, slack, scale=None):
    """max over voxels of max(|got - ref| - slack, 0) / scale (scale = max ref)."""
    got = np.asarray(got, dtype=np.float64)
    ex = np.abs(got - ref)
    if slack is not None:
        ex = np.maximum(ex - slack, 0.0)
    s = float(ref.max()) if scale is None else float(scale)
    if s == 0.0:
        return float(ex.max()) if ex.size else 0.0
    return float(ex.max() / s) if ex.size else 0.0


def densest_cells(points, gx, gy, cell=(16, 8), k=8):
    """Indices (cx, cy) of the k cells holding the most events (input statistics)."""
    cx = np.floor(points[:, 0] / cell[0]).astype(np.int64)
    cy = np.floor(points[:, 1] / cell[1]).astype(np.int64)
    nx, ny = (gx + cell[0] - 1) // cell[0], (gy + cell[1] - 1) // cell[1]
    ok = (cx >= 0) & (cx < nx) & (cy >= 0) & (cy < ny)
    h = np.bincount(cx[ok] * ny + cy[ok], minlength=nx * ny)
    top = np.argsort(h)[::-1][:k]
    return [(int(t // ny), int(t % ny)) for t in top]


def sample_tile_boxes(points, gx, gy, gt, n_random=48, seed=0, cell=(16, 8)):
    """Tile-shaped boxes (full T) for sampled parity: the densest tiles, the four
    corners, edge tiles and random tiles."""
    nx, ny = (gx + cell[0] - 1) // cell[0], (gy + cell[1] - 1) // cell[1]
    cells = set(densest_cells(points, gx, gy, cell, k=8))
    cells |= {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, 0), (0, ny // 2),
              (nx - 1, ny // 2), (nx // 2, ny - 1)}
    rng = np.random.default_rng(seed)
    while len(cells) < 16 + n_random:
        cells.add((int(rng.integers(0, nx)), int(rng.integers(0, ny))))
    boxes = []
    for cx, cy in sorted(cells):
        boxes.append((cx * cell[0], min(gx, (cx + 1) * cell[0]), cy * cell[1],
                      min(gy, (cy + 1) * cell[1]), 0, gt))
    return boxes


@contextlib.contextmanager
def captured(torch, graph, stream, **kw):
    """torch.cuda.graph with Python's garbage collector held off.  A collection
    inside the capture could destroy CUDA objects left by earlier tests (events,
    graphs, streams); an ongoing global-mode capture forbids those calls and
    would be invalidated for reasons outside the code under test."""
    gc.collect()
    torch.cuda.synchronize()
    was = gc.isenabled()
    gc.disable()
    try:
        with torch.cuda.graph(graph, stream=stream, **kw):
            yield
    finally:
        if was:
            gc.enable()
