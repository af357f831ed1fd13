"""Seeded synthetic event sets for STKDE (inputs only).

This module draws event coordinates and nothing else: it holds none of the
density arithmetic, so both the CUDA path and the FP64 oracle can take their
inputs from it without sharing any of the method's code.

The paper's datasets (Dengue, PollenUS, Flu, eBird; Section 6.1) are not
available here, so clustered Gaussian mixtures of the same character stand in
for them: events concentrate in space around a few centres and in time around
per-cluster bursts, with a share of uniform background noise.  Coordinates are
FP64 in voxel units (grid origin 0, sres = tres = 1), shaped ``(n, 3)`` as
``x, y, t`` rows.  Events that fall outside the grid are kept: they still count
in ``n`` and still reach voxels inside their bandwidth cylinder.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1705_09366


@dataclasses.dataclass(frozen=True)
class Workload:
    """One STKDE problem: events plus grid and bandwidths (domain units)."""

    name: str
    points: np.ndarray          # (n, 3) float64, rows (x, y, t)
    gx: int
    gy: int
    gt: int
    hs: float
    ht: float
    x0: float = 0.0
    y0: float = 0.0
    t0: float = 0.0
    sres: float = 1.0
    tres: float = 1.0

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def grid_bytes(self) -> int:
        return 4 * self.gx * self.gy * self.gt


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def clustered_events(rng: np.random.Generator, n: int, gx: int, gy: int, gt: int,
                     n_clusters: int, sigma_xy=(6.0, 6.0), sigma_t=None,
                     background: float = 0.0) -> np.ndarray:
    """Gaussian space clusters with optional Gaussian time bursts.

    ``sigma_xy`` is a (lo, hi) range for the per-cluster isotropic spatial sigma
    (voxels).  ``sigma_t`` is None for times uniform over [0, gt), else a
    (lo, hi) range for the per-cluster burst sigma, the burst centre being
    uniform over [0, gt).  ``background`` is the share of events drawn uniformly
    over the whole grid.  Clusters have equal weight.
    """
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    cx = rng.uniform(0.0, gx, n_clusters)
    cy = rng.uniform(0.0, gy, n_clusters)
    sxy = rng.uniform(sigma_xy[0], sigma_xy[1], n_clusters)
    if sigma_t is not None:
        ct = rng.uniform(0.0, gt, n_clusters)
        st = rng.uniform(sigma_t[0], sigma_t[1], n_clusters)
    lab = rng.integers(0, n_clusters, n_cl)
    pts = np.empty((n, 3), dtype=np.float64)
    pts[:n_cl, 0] = cx[lab] + sxy[lab] * rng.standard_normal(n_cl)
    pts[:n_cl, 1] = cy[lab] + sxy[lab] * rng.standard_normal(n_cl)
    if sigma_t is None:
        pts[:n_cl, 2] = rng.uniform(0.0, gt, n_cl)
    else:
        pts[:n_cl, 2] = ct[lab] + st[lab] * rng.standard_normal(n_cl)
    if n_bg:
        pts[n_cl:, 0] = rng.uniform(0.0, gx, n_bg)
        pts[n_cl:, 1] = rng.uniform(0.0, gy, n_bg)
        pts[n_cl:, 2] = rng.uniform(0.0, gt, n_bg)
        # interleave background and cluster events so no index range is special
        pts = pts[rng.permutation(n)]
    return np.ascontiguousarray(pts)


def small(seed_offset: int = 0) -> Workload:
    """n = 2,000; 64x64x32 grid; hs = 4, ht = 3 voxels; 8 clusters (sigma 6), t uniform."""
    rng = _rng(SEED_BASE + 0 + 1000 * seed_offset)
    pts = clustered_events(rng, 2000, 64, 64, 32, 8, (6.0, 6.0), None, 0.0)
    return Workload("small-n2k-64x64x32-hs4-ht3", pts, 64, 64, 32, 4.0, 3.0)


def medium(seed_offset: int = 0) -> Workload:
    """n = 200,000; 512x512x256; hs = 10, ht = 8; 64 clusters, bursts, 10% background."""
    rng = _rng(SEED_BASE + 1 + 1000 * seed_offset)
    pts = clustered_events(rng, 200_000, 512, 512, 256, 64, (5.0, 30.0), (3.0, 20.0), 0.10)
    return Workload("medium-n200k-512x512x256-hs10-ht8", pts, 512, 512, 256, 10.0, 8.0)


def large(seed_offset: int = 0) -> Workload:
    """n = 2,000,000; 1024x1024x512; hs = 25, ht = 20; 256 clusters, bursts, 10% background."""
    rng = _rng(SEED_BASE + 2 + 1000 * seed_offset)
    pts = clustered_events(rng, 2_000_000, 1024, 1024, 512, 256, (5.0, 30.0), (3.0, 20.0), 0.10)
    return Workload("large-n2M-1024x1024x512-hs25-ht20", pts, 1024, 1024, 512, 25.0, 20.0)


def batched(count: int = 64, seed_offset: int = 0) -> list[Workload]:
    """Uneven instances: n log-uniform in [1e3, 5e5], grids 64^3 .. 512x512x128,
    hs ~ U[2, 30], ht ~ U[2, 20] voxels; each instance its own seeded clustered set."""
    rng = _rng(SEED_BASE + 3 + 1000 * seed_offset)
    out = []
    sides_xy = [64, 128, 256, 512]
    sides_t = [64, 128]
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e5)))))
        gxy = int(rng.choice(sides_xy))
        gt = int(rng.choice(sides_t))
        hs = float(rng.uniform(2.0, 30.0))
        ht = float(rng.uniform(2.0, 20.0))
        ncl = int(rng.integers(4, 65))
        irng = _rng(SEED_BASE + 3 + 1000 * seed_offset + 7919 * (i + 1))
        pts = clustered_events(irng, n, gxy, gxy, gt, ncl, (3.0, 20.0), (2.0, 12.0), 0.10)
        out.append(Workload(f"batch{i}-n{n}-{gxy}x{gxy}x{gt}", pts, gxy, gxy, gt, hs, ht))
    return out


def resident_sets(seed_offset: int = 0, sizes=(50_000, 200_000, 1_000_000, 2_000_000)):
    """Point sets kept resident by the serving loop: clustered events in a
    512 x 512 x 256 domain (domain units)."""
    rng = _rng(SEED_BASE + 4 + 1000 * seed_offset)
    return [clustered_events(rng, n, 512, 512, 256, 64, (5.0, 30.0), (3.0, 20.0), 0.10)
            for n in sizes]


def adaptive_bandwidths(n: int, hs: float, ht: float, spread: float = 2.0,
                        seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Per-event bandwidths (domain units) log-uniform in [h / spread, h * spread]
    around the fixed pair (hs, ht), drawn independently per event and axis: a
    stand-in for bandwidths adapted to the local population density, which the
    caller would derive from data this module does not have."""
    rng = _rng(SEED_BASE + 5 + 7 * seed)
    ls = math.log(spread)
    hsi = hs * np.exp(rng.uniform(-ls, ls, n))
    hti = ht * np.exp(rng.uniform(-ls, ls, n))
    return np.ascontiguousarray(hsi), np.ascontiguousarray(hti)


def tiny(rng: np.random.Generator, n: int, gx: int, gy: int, gt: int, spill: float = 0.25) -> np.ndarray:
    """Uniform events over the grid widened by ``spill`` of each side, so some
    fall outside it (for brute-force comparisons on tiny inputs)."""
    lo = np.array([-spill * gx, -spill * gy, -spill * gt])
    hi = np.array([(1 + spill) * gx, (1 + spill) * gy, (1 + spill) * gt])
    return np.ascontiguousarray(rng.uniform(lo, hi, size=(n, 3)))


WORKLOADS = {"small": small, "medium": medium, "large": large}
