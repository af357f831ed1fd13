"""Pins for the FP64 oracle, each against something other than the oracle itself.

The paper prints no density values, so the oracle is pinned by closed-form
integrals of the kernels (tests/golden/kernel_integrals.json, re-derived here by
quadrature), by a library routine that computes the temporal factor
(scikit-learn's 1-D Epanechnikov KDE), by symmetries and invariants the density
equation of Section 2.1 implies, by the cylinder geometry of Figure 2, and by
brute force: Algorithm 1 (VB) against Algorithm 2 (PB) on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1705_09366_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _golden(golden_dir):
    with open(os.path.join(golden_dir, "kernel_integrals.json")) as f:
        return json.load(f)


def test_golden_integrals_match_quadrature(golden_dir):
    """The hand-derived kernel integrals agree with scipy quadrature."""
    integrate = pytest.importorskip("scipy.integrate")
    g = _golden(golden_dir)
    lo = lambda u: -math.sqrt(max(0.0, 1 - u * u))
    hi = lambda u: math.sqrt(max(0.0, 1 - u * u))
    mass, _ = integrate.dblquad(lambda v, u: (1 - u * u) * (1 - v * v), -1, 1, lo, hi)
    m2, _ = integrate.dblquad(lambda v, u: u * u * (1 - u * u) * (1 - v * v), -1, 1, lo, hi)
    assert mass == pytest.approx(g["spatial_mass_per_cs"]["value"], rel=1e-9)
    assert m2 == pytest.approx(g["spatial_second_moment_u2_per_cs"]["value"], rel=1e-9)
    assert m2 / mass == pytest.approx(g["spatial_mean_u2"]["value"], rel=1e-9)
    assert oracle.CS_UNIT_MASS * mass == pytest.approx(1.0, rel=1e-12)
    assert g["cs_unit_mass"]["value"] == pytest.approx(oracle.CS_UNIT_MASS, rel=1e-15)
    assert oracle.CS_PRINTED * mass == pytest.approx(g["spatial_mass_printed_cs"]["value"], rel=1e-12)
    tm, _ = integrate.quad(lambda w: 0.75 * (1 - w * w), -1, 1)
    tw2, _ = integrate.quad(lambda w: 0.75 * w * w * (1 - w * w), -1, 1)
    assert tm == pytest.approx(g["temporal_mass_printed_ct"]["value"], rel=1e-12)
    assert tw2 == pytest.approx(g["temporal_mean_w2"]["value"], rel=1e-12)


def _centred_events(rng, m, G, h):
    c = G / 2.0
    return np.column_stack([c + rng.uniform(-1, 1, m), c + rng.uniform(-1, 1, m),
                            c + rng.uniform(-1, 1, m)])


@pytest.mark.parametrize("h,tol", [(12, 2.5e-3), (24, 6e-4), (48, 2e-4)])
def test_mass_integrates_to_one(h, tol):
    """With c_s = 24/(13 pi) and every cylinder inside the grid, the density's
    Riemann sum over the grid tends to 1 (shrinking error as h grows)."""
    rng = np.random.default_rng(h)
    G = 2 * h + 8
    pts = _centred_events(rng, 4, G, h)
    p = oracle.params(G, G, G, h, h, cs=oracle.CS_UNIT_MASS, round_fp32=False)
    out = oracle.pb(pts, p)
    assert abs(out.sum() * p.sres ** 2 * p.tres - 1.0) < tol


def test_mass_with_printed_constants(golden_dir):
    """With the printed c_s = pi/2 the mass is 13 pi^2 / 48, also in domain
    units with non-unit resolutions and a shifted origin."""
    g = _golden(golden_dir)
    rng = np.random.default_rng(7)
    h = 30
    G = 2 * h + 8
    sres, tres = 0.25, 3.0
    x0, y0, t0 = -17.0, 4.5, 1000.0
    vox = _centred_events(rng, 3, G, h)
    pts = np.column_stack([x0 + vox[:, 0] * sres, y0 + vox[:, 1] * sres, t0 + vox[:, 2] * tres])
    p = oracle.params(G, G, G, h * sres, h * tres, x0=x0, y0=y0, t0=t0, sres=sres, tres=tres,
                      round_fp32=False)
    out = oracle.pb(pts, p)
    mass = out.sum() * sres * sres * tres
    assert mass == pytest.approx(g["spatial_mass_printed_cs"]["value"], rel=5e-4)


@pytest.mark.parametrize("h", [24, 48])
def test_second_moments(golden_dir, h):
    """Spatial E[u^2] = 19/104 and temporal E[w^2] = 1/5 under the kernels."""
    g = _golden(golden_dir)
    pts = np.array([[h + 4 + 0.37, h + 4 - 0.21, h + 4 + 0.13]])
    G = 2 * h + 8
    p = oracle.params(G, G, G, h, h, round_fp32=False)
    out = oracle.pb(pts, p)
    X = np.arange(G) + 0.5
    u2 = ((X - pts[0, 0]) / h) ** 2
    v2 = ((X - pts[0, 1]) / h) ** 2
    w2 = ((X - pts[0, 2]) / h) ** 2
    tot = out.sum()
    tol = 3e-3 if h == 24 else 1e-3
    assert (out * u2[:, None, None]).sum() / tot == pytest.approx(g["spatial_mean_u2"]["value"], abs=tol)
    assert (out * v2[None, :, None]).sum() / tot == pytest.approx(g["spatial_mean_u2"]["value"], abs=tol)
    assert (out * w2[None, None, :]).sum() / tot == pytest.approx(g["temporal_mean_w2"]["value"], abs=tol)


def test_temporal_profile_matches_library_epanechnikov_kde():
    """Events that share one planar position reduce the density to
    k_s(0,0)/hs^2 times a 1-D Epanechnikov KDE in time, which scikit-learn
    computes independently (kernel 3/(4h) (1 - (d/h)^2))."""
    kd_mod = pytest.importorskip("sklearn.neighbors")
    rng = np.random.default_rng(11)
    gx, gy, gt = 9, 7, 120
    hs, ht = 3.3, 6.7
    X0, Y0 = 4, 3
    n = 40
    t = rng.uniform(-10, gt + 10, n)
    pts = np.column_stack([np.full(n, X0 + 0.5), np.full(n, Y0 + 0.5), t])
    p = oracle.params(gx, gy, gt, hs, ht, round_fp32=False)
    out = oracle.pb(pts, p)
    kde = kd_mod.KernelDensity(kernel="epanechnikov", bandwidth=ht).fit(t[:, None])
    tc = (np.arange(gt) + 0.5)[:, None]
    with np.errstate(divide="ignore"):
        ref = np.exp(kde.score_samples(tc)) * oracle.CS_PRINTED / hs ** 2
    np.testing.assert_allclose(out[X0, Y0, :], ref, rtol=1e-12, atol=1e-15)
    # and against VB, which evaluates the same events by the other loop order
    np.testing.assert_allclose(oracle.vb(pts, p)[X0, Y0, :], ref, rtol=1e-12, atol=1e-15)


def test_support_is_the_bandwidth_cylinder():
    """A single event lights exactly the voxels whose centre lies strictly inside
    the cylinder of radius hs and half-height ht around it (Figure 2)."""
    G = 40
    pts = np.array([[20.31, 19.77, 20.42]])
    hs, ht = 7.3, 4.6
    p = oracle.params(G, G, G, hs, ht, round_fp32=False)
    out = oracle.pb(pts, p)
    X = np.arange(G) + 0.5
    d2 = (X[:, None, None] - pts[0, 0]) ** 2 + (X[None, :, None] - pts[0, 1]) ** 2
    dt = np.abs(X[None, None, :] - pts[0, 2])
    inside = (d2 < hs * hs) & (dt < ht)
    assert np.array_equal(out > 0, inside)
    assert (out >= 0).all()


def test_single_event_closed_form():
    """n = 1 at a sub-voxel offset in a 64^3 grid: each voxel equals
    c_s (1-u^2)(1-v^2) c_t (1-w^2) / (hs^2 ht) inside the cylinder, 0 outside."""
    G = 64
    pts = np.array([[31.3, 30.8, 33.6]])
    hs, ht = 9.5, 6.25
    p = oracle.params(G, G, G, hs, ht, round_fp32=False)
    out = oracle.pb(pts, p)
    c = np.arange(G) + 0.5
    u = (c[:, None, None] - pts[0, 0]) / hs
    v = (c[None, :, None] - pts[0, 1]) / hs
    w = (c[None, None, :] - pts[0, 2]) / ht
    ref = np.where((u * u + v * v < 1) & (np.abs(w) <= 1),
                   (math.pi / 2) * (1 - u * u) * (1 - v * v) * 0.75 * (1 - w * w) / (hs * hs * ht), 0.0)
    np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-300)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(axis):
    """Adding the mirror image of every event about the grid's mid-plane makes
    the grid symmetric under X -> G-1-X (resp. Y, T): the kernels are even and
    voxels are sampled at their centres."""
    rng = np.random.default_rng(100 + axis)
    dims = [30, 26, 22]
    x0 = [2.0, -3.0, 10.0]
    res = [0.5, 0.5, 2.0]
    n = 60
    vox = np.column_stack([rng.uniform(-3, d + 3, n) for d in dims])
    pts = np.column_stack([x0[k] + vox[:, k] * res[k] for k in range(3)])
    mir = pts.copy()
    mir[:, axis] = 2 * x0[axis] + dims[axis] * res[axis] - pts[:, axis]
    both = np.vstack([pts, mir])
    p = oracle.params(*dims, 2.6, 3.4, x0=x0[0], y0=x0[1], t0=x0[2], sres=res[0], tres=res[2],
                      round_fp32=False)
    out = oracle.pb(both, p)
    flipped = np.flip(out, axis=axis)
    assert np.abs(out - flipped).max() <= 1e-12 * out.max()
    assert out.max() > 0


def test_translation_by_whole_voxels():
    """Moving every event and the grid origin by whole voxels leaves the grid unchanged."""
    rng = np.random.default_rng(5)
    pts = synth.tiny(rng, 50, 20, 18, 16)
    p = oracle.params(20, 18, 16, 3.1, 2.2, round_fp32=False)
    a = oracle.pb(pts, p)
    shift = np.array([7.0, -5.0, 13.0])
    q = oracle.params(20, 18, 16, 3.1, 2.2, x0=7.0, y0=-5.0, t0=13.0, round_fp32=False)
    b = oracle.pb(pts + shift, q)
    assert np.abs(a - b).max() <= 1e-13 * a.max()


def test_additivity():
    """n f(A u B) = |A| f(A) + |B| f(B): the estimate is a normalised sum over events."""
    rng = np.random.default_rng(9)
    A = synth.tiny(rng, 37, 16, 16, 12)
    B = synth.tiny(rng, 21, 16, 16, 12)
    p = oracle.params(16, 16, 12, 2.7, 1.9, round_fp32=False)
    fa, fb, fab = oracle.pb(A, p), oracle.pb(B, p), oracle.pb(np.vstack([A, B]), p)
    lhs = 58 * fab
    rhs = 37 * fa + 21 * fb
    assert np.abs(lhs - rhs).max() <= 1e-12 * lhs.max()


@pytest.mark.parametrize("seed", range(8))
def test_vb_equals_pb_on_tiny_inputs(seed):
    """Brute force: Algorithm 1 (voxel loop, domain units) and Algorithm 2
    (event loop over the clipped voxel box, voxel units) agree to 1e-12 on tiny
    random problems with non-integer bandwidths, non-unit resolutions, a shifted
    origin, events outside the grid, and both sampling conventions."""
    rng = np.random.default_rng(1000 + seed)
    gx, gy, gt = (int(v) for v in rng.integers(3, 25, 3))
    n = int(rng.integers(1, 51))
    sres = float(rng.uniform(0.3, 3.0))
    tres = float(rng.uniform(0.3, 3.0))
    x0, y0, t0 = (float(v) for v in rng.uniform(-50, 50, 3))
    hs = float(rng.uniform(0.4, 6.0)) * sres
    ht = float(rng.uniform(0.4, 6.0)) * tres
    vox = synth.tiny(rng, n, gx, gy, gt, spill=0.3)
    pts = np.column_stack([x0 + vox[:, 0] * sres, y0 + vox[:, 1] * sres, t0 + vox[:, 2] * tres])
    for off in (0.5, 0.0):
        for r32 in (False, True):
            p = oracle.params(gx, gy, gt, hs, ht, x0=x0, y0=y0, t0=t0, sres=sres, tres=tres,
                              sample_off=off, round_fp32=r32)
            a = oracle.vb(pts, p)
            b = oracle.pb(pts, p)
            scale = max(a.max(), 1e-300)
            assert np.abs(a - b).max() <= 1e-12 * scale, (off, r32)


def test_empty_input_is_zero():
    p = oracle.params(5, 6, 7, 1.5, 1.5)
    z = np.zeros((0, 3))
    assert not oracle.pb(z, p).any()
    assert not oracle.vb(z, p).any()
    assert oracle.count_updates(z, p) == 0


def test_sampled_boxes_equal_full_grid():
    """PB restricted to boxes equals the same voxels of the full-grid PB, and
    VB at sampled voxels agrees too."""
    w = synth.small()
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht)
    full, slack = oracle.pb(w.points, p, with_slack=True)
    boxes = [(0, 16, 0, 8, 0, 32), (48, 64, 56, 64, 0, 32), (20, 37, 11, 30, 5, 17)]
    for (vals, sl), b in zip(oracle.pb_boxes(w.points, p, boxes), boxes):
        np.testing.assert_array_equal(vals, full[b[0]:b[1], b[2]:b[3], b[4]:b[5]])
        np.testing.assert_array_equal(sl, slack[b[0]:b[1], b[2]:b[3], b[4]:b[5]])
    rng = np.random.default_rng(3)
    vox = np.column_stack([rng.integers(0, d, 200) for d in (w.gx, w.gy, w.gt)])
    vals = oracle.vb_voxels(w.points, p, vox)
    np.testing.assert_allclose(vals, full[vox[:, 0], vox[:, 1], vox[:, 2]], rtol=1e-12,
                               atol=1e-12 * full.max())


def test_update_count_by_enumeration():
    """The work count equals the number of (event, voxel) pairs with a nonzero
    term, enumerated event by event (k_t vanishes only at |w| = 1, which random
    times never hit)."""
    rng = np.random.default_rng(21)
    pts = synth.tiny(rng, 30, 20, 17, 15)
    p = oracle.params(20, 17, 15, 3.7, 2.9, round_fp32=False)
    total = 0
    for i in range(pts.shape[0]):
        total += int((oracle.pb(pts[i:i + 1], p) > 0).sum())
    assert oracle.count_updates(pts, p) == total


def test_tie_slack_marks_only_wall_pairs():
    """Slack is zero away from the cylinder wall and covers the term of an event
    placed exactly on it."""
    G = 20
    hs = 5.0
    # event at a voxel centre offset so that voxel (X=13, Y=10) is exactly hs away:
    # dx = 13.5 - 10.5 = 3, dy = 14.5 - 10.5 = 4 -> d = 5 = hs (tie; strictly outside)
    pts = np.array([[10.5, 10.5, 10.5]])
    p = oracle.params(G, G, G, hs, 3.0, round_fp32=False)
    out, slack = oracle.pb(pts, p, with_slack=True)
    assert out[13, 14, 10] == 0.0
    assert slack[13, 14, 10] > 0.0
    assert slack[10, 10, 10] == 0.0
    assert (slack > 0).sum() < (out > 0).sum()


def test_box_pair_counts_add_up_to_the_update_count():
    """Pair counts of boxes that tile the grid sum to the whole-grid update count."""
    rng = np.random.default_rng(31)
    pts = synth.tiny(rng, 40, 24, 20, 18)
    p = oracle.params(24, 20, 18, 3.2, 2.6)
    boxes = [(x, min(24, x + 7), y, min(20, y + 9), t, min(18, t + 10))
             for x in range(0, 24, 7) for y in range(0, 20, 9) for t in range(0, 18, 10)]
    _, counts = oracle.pb_boxes(pts, p, boxes, pair_counts=True)
    assert int(counts.sum()) == oracle.count_updates(pts, p)
