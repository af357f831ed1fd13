"""Pins for the oracle's per-event (adaptive) bandwidth functions.

The conclusion names a bandwidth that adapts to the local population density as
the next step; with per-event bandwidths hs_i, ht_i each event still adds one
separable cylinder of unit-scaled mass, normalised by 1/(n hs_i^2 ht_i).  These
functions are pinned by reduction to the fixed-bandwidth density (already pinned
by closed forms and quadrature): equal bandwidths give the fixed density, and
the adaptive grid is the mean of one-event fixed-bandwidth grids.  Brute force
(Algorithm 1 against Algorithm 2 with the per-event test), a closed form for
one event, unit mass and mirror symmetry close the remaining gaps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1705_09366_gb300 import synth


def _random_problem(rng, n, spill=0.3):
    gx, gy, gt = (int(v) for v in rng.integers(3, 25, 3))
    sres = float(rng.uniform(0.3, 3.0))
    tres = float(rng.uniform(0.3, 3.0))
    x0, y0, t0 = (float(v) for v in rng.uniform(-50, 50, 3))
    vox = synth.tiny(rng, n, gx, gy, gt, spill=spill)
    pts = np.column_stack([x0 + vox[:, 0] * sres, y0 + vox[:, 1] * sres, t0 + vox[:, 2] * tres])
    hs = rng.uniform(0.4, 6.0, n) * sres
    ht = rng.uniform(0.4, 6.0, n) * tres
    return (gx, gy, gt), (x0, y0, t0), (sres, tres), pts, hs, ht


def test_equal_bandwidths_give_the_fixed_density():
    rng = np.random.default_rng(11)
    dims, org, res, pts, _, _ = _random_problem(rng, 40)
    hs, ht = 2.9 * res[0], 3.7 * res[1]
    p = oracle.params(*dims, hs, ht, x0=org[0], y0=org[1], t0=org[2], sres=res[0], tres=res[1],
                      round_fp32=False)
    a = oracle.pb(pts, p)
    b = oracle.pb_adaptive(pts, np.full(40, hs), np.full(40, ht), p)
    c = oracle.vb_adaptive(pts, np.full(40, hs), np.full(40, ht), p)
    assert a.max() > 0
    assert np.abs(a - b).max() <= 1e-13 * a.max()
    assert np.abs(a - c).max() <= 1e-12 * a.max()


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_is_the_mean_of_one_event_fixed_densities(seed):
    """f = (1/n) sum_i f_fixed({e_i}; hs_i, ht_i): each event keeps its own
    bandwidth and its own normalisation, and n counts every event."""
    rng = np.random.default_rng(200 + seed)
    n = 12
    dims, org, res, pts, hs, ht = _random_problem(rng, n)
    kw = dict(x0=org[0], y0=org[1], t0=org[2], sres=res[0], tres=res[1], round_fp32=False)
    p = oracle.params(*dims, 1.0, 1.0, **kw)
    got = oracle.pb_adaptive(pts, hs, ht, p)
    ref = np.zeros(dims)
    for i in range(n):
        ref += oracle.pb(pts[i:i + 1], oracle.params(*dims, hs[i], ht[i], **kw))
    ref /= n
    scale = max(ref.max(), 1e-300)
    assert np.abs(got - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("seed", range(8))
def test_vb_equals_pb_on_tiny_inputs(seed):
    """Algorithm 1 with the per-event test (domain units) against Algorithm 2
    with a per-event box (voxel units), both sampling conventions, with and
    without binary32 re-centring."""
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(1, 51))
    dims, org, res, pts, hs, ht = _random_problem(rng, n)
    for off in (0.5, 0.0):
        for r32 in (False, True):
            p = oracle.params(*dims, 1.0, 1.0, x0=org[0], y0=org[1], t0=org[2], sres=res[0],
                              tres=res[1], sample_off=off, round_fp32=r32)
            a = oracle.vb_adaptive(pts, hs, ht, p)
            b = oracle.pb_adaptive(pts, hs, ht, p)
            scale = max(a.max(), 1e-300)
            assert np.abs(a - b).max() <= 1e-12 * scale, (off, r32)


def test_two_event_closed_form():
    """Two events with different bandwidths in a 48^3 grid: every voxel is the
    mean of the two printed-constant kernel products, each over its own
    hs_i^2 ht_i."""
    G = 48
    pts = np.array([[20.3, 22.8, 25.6], [27.1, 24.4, 20.2]])
    hs = np.array([6.5, 11.25])
    ht = np.array([9.0, 4.75])
    p = oracle.params(G, G, G, 1.0, 1.0, round_fp32=False)
    out = oracle.pb_adaptive(pts, hs, ht, p)
    c = np.arange(G) + 0.5
    ref = np.zeros((G, G, G))
    for (x, y, t), h, k in zip(pts, hs, ht):
        u = (c[:, None, None] - x) / h
        v = (c[None, :, None] - y) / h
        w = (c[None, None, :] - t) / k
        ref += np.where((u * u + v * v < 1) & (np.abs(w) <= 1),
                        (math.pi / 2) * (1 - u * u) * (1 - v * v) * 0.75 * (1 - w * w) / (h * h * k), 0.0)
    ref /= 2
    np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-300)


def test_unit_mass_with_mixed_bandwidths():
    """With c_s = 24/(13 pi) every event contributes mass 1/n whatever its
    bandwidth, so the Riemann sum tends to 1."""
    rng = np.random.default_rng(77)
    G = 120
    m = 5
    pts = np.column_stack([G / 2 + rng.uniform(-1, 1, m) for _ in range(3)])
    hs = rng.uniform(24, 48, m)
    ht = rng.uniform(24, 48, m)
    p = oracle.params(G, G, G, 1.0, 1.0, cs=oracle.CS_UNIT_MASS, round_fp32=False)
    out = oracle.pb_adaptive(pts, hs, ht, p)
    assert abs(out.sum() - 1.0) < 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(axis):
    """Each event's mirror image carries the same bandwidths: the grid is
    symmetric about the mid-plane of the mirrored axis."""
    rng = np.random.default_rng(400 + axis)
    dims = [28, 24, 20]
    x0 = [1.0, -2.0, 6.0]
    res = [0.5, 0.5, 2.0]
    n = 40
    vox = np.column_stack([rng.uniform(-3, d + 3, n) for d in dims])
    pts = np.column_stack([x0[k] + vox[:, k] * res[k] for k in range(3)])
    mir = pts.copy()
    mir[:, axis] = 2 * x0[axis] + dims[axis] * res[axis] - pts[:, axis]
    hs = rng.uniform(0.8, 3.0, n)
    ht = rng.uniform(1.0, 8.0, n)
    p = oracle.params(*dims, 1.0, 1.0, x0=x0[0], y0=x0[1], t0=x0[2], sres=res[0], tres=res[2],
                      round_fp32=False)
    out = oracle.pb_adaptive(np.vstack([pts, mir]), np.r_[hs, hs], np.r_[ht, ht], p)
    assert out.max() > 0
    assert np.abs(out - np.flip(out, axis=axis)).max() <= 1e-12 * out.max()


def test_boxes_equal_full_grid():
    rng = np.random.default_rng(5)
    n = 60
    dims, org, res, pts, hs, ht = _random_problem(rng, n)
    p = oracle.params(*dims, 1.0, 1.0, x0=org[0], y0=org[1], t0=org[2], sres=res[0], tres=res[1])
    full, slack = oracle.pb_adaptive(pts, hs, ht, p, with_slack=True)
    gx, gy, gt = dims
    boxes = [(0, gx, 0, gy, 0, gt), (1, max(2, gx // 2), 0, gy, 1, max(2, gt - 1)),
             (gx - 1, gx, gy // 3, gy, 0, 1)]
    for b, (v, s) in zip(boxes, oracle.pb_adaptive_boxes(pts, hs, ht, p, boxes)):
        np.testing.assert_array_equal(v, full[b[0]:b[1], b[2]:b[3], b[4]:b[5]])
        np.testing.assert_array_equal(s, slack[b[0]:b[1], b[2]:b[3], b[4]:b[5]])


def test_empty_input_is_zero():
    p = oracle.params(5, 6, 7, 1.0, 1.0)
    z = np.zeros((0, 3))
    assert not oracle.pb_adaptive(z, np.zeros(0), np.zeros(0), p).any()
    assert not oracle.vb_adaptive(z, np.zeros(0), np.zeros(0), p).any()


def test_box_pair_counts_equal_per_event_update_counts():
    """The in-cylinder pairs the adaptive boxes count add up to the sum of the
    fixed-bandwidth update counts of each event with its own bandwidths."""
    rng = np.random.default_rng(31)
    n = 30
    dims, org, res, pts, hs, ht = _random_problem(rng, n)
    kw = dict(x0=org[0], y0=org[1], t0=org[2], sres=res[0], tres=res[1])
    p = oracle.params(*dims, 1.0, 1.0, **kw)
    gx, gy, gt = dims
    boxes = [(0, gx // 2, 0, gy, 0, gt), (gx // 2, gx, 0, gy, 0, gt)]
    _, counts = oracle.pb_adaptive_boxes(pts, hs, ht, p, boxes, pair_counts=True)
    ref = sum(oracle.count_updates(pts[i:i + 1], oracle.params(*dims, hs[i], ht[i], **kw))
              for i in range(n))
    assert int(counts.sum()) == ref


# ---- bandwidths from a pilot density (Abramson's square-root law)

def _clustered(seed, n=400, G=40):
    rng = np.random.default_rng(seed)
    return synth.clustered_events(rng, n, G, G, G, 3, (2.0, 6.0), (2.0, 6.0), 0.3), G


def test_abramson_alpha_zero_gives_the_pilot_bandwidths():
    pts, G = _clustered(1)
    p = oracle.params(G, G, G, 3.0, 2.5)
    hs, ht, lam = oracle.abramson(pts, p, alpha=0.0)
    assert np.all(lam == 1.0) and np.all(hs == 3.0) and np.all(ht == 2.5)


def test_abramson_geometric_mean_is_one():
    """lambda_i = (f_i / g)^-alpha with g the geometric mean of the f_i: the
    unclamped factors have geometric mean exactly 1."""
    pts, G = _clustered(2)
    p = oracle.params(G, G, G, 3.0, 2.5)
    _, _, lam = oracle.abramson(pts, p, alpha=0.5, lam_min=1e-9, lam_max=1e9)
    assert abs(np.exp(np.mean(np.log(lam))) - 1.0) < 1e-12


def test_abramson_is_invariant_to_the_pilot_scale():
    """Scaling the pilot (here: unit-mass instead of printed kernel constants)
    leaves the factors unchanged."""
    pts, G = _clustered(3)
    a = oracle.abramson(pts, oracle.params(G, G, G, 3.0, 2.5), alpha=0.5)[2]
    b = oracle.abramson(pts, oracle.params(G, G, G, 3.0, 2.5, cs=oracle.CS_UNIT_MASS), alpha=0.5)[2]
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_abramson_denser_means_narrower():
    """The factor is a non-increasing function of the pilot value at the event's
    voxel, with exponent -alpha."""
    pts, G = _clustered(4)
    p = oracle.params(G, G, G, 3.0, 2.5)
    pilot = oracle.pb(pts, p)
    _, _, lam = oracle.abramson(pts, p, alpha=0.5, lam_min=1e-9, lam_max=1e9, pilot=pilot)
    vox = np.clip(np.floor(pts).astype(int), 0, G - 1)
    f = pilot[vox[:, 0], vox[:, 1], vox[:, 2]]
    f = np.maximum(f, 1e-6 * f.max())
    order = np.argsort(f)
    assert np.all(np.diff(lam[order]) <= 1e-15)
    np.testing.assert_allclose(lam[order[-1]] / lam[order[0]], (f[order[-1]] / f[order[0]]) ** -0.5,
                               rtol=1e-12)


def test_abramson_cluster_against_a_lone_event():
    """m coincident events and one lone event far away, same sub-voxel offset: the
    pilot at the cluster is m times the pilot at the lone event, so the lone
    event's factor is m^alpha times the cluster's, and the geometric mean is 1."""
    m, G = 9, 48
    # dyadic offsets: the binary32 re-centring keeps them exact
    pts = np.array([[10.25, 10.625, 10.125]] * m + [[38.25, 37.625, 38.125]])
    p = oracle.params(G, G, G, 4.0, 3.0)
    _, _, lam = oracle.abramson(pts, p, alpha=0.5, lam_min=1e-9, lam_max=1e9)
    assert lam[-1] / lam[0] == pytest.approx(m ** 0.5, rel=1e-12)
    assert lam[0] ** m * lam[-1] == pytest.approx(1.0, rel=1e-12)


def test_abramson_clamps():
    pts, G = _clustered(5)
    p = oracle.params(G, G, G, 3.0, 2.5)
    _, _, lam = oracle.abramson(pts, p, alpha=1.0, lam_min=0.8, lam_max=1.25)
    assert lam.min() == 0.8 and lam.max() == 1.25
