"""GPU: per-event (adaptive) bandwidths through stkde_compute_adaptive.

Each event carries its own hs_i, ht_i and normalisation 1/(n hs_i^2 ht_i), the
density-adaptive bandwidth that the conclusion (Section 8) leaves as future
work.  The CUDA path is compared element by element with the FP64 oracle's
adaptive PB on full grids that span several tiles with ragged edges, and on
sampled tiles of the clustered 200k-event workload; equal bandwidths must
reproduce stkde_compute within the parity tolerance; host and device
bandwidth arrays must give the same bits; invalid bandwidths are rejected
before any launch.
"""
import ctypes
import zlib

import numpy as np
import pytest

import oracle
import paper_1705_09366_gb300 as pkg
import parity_util as pu
from paper_1705_09366_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = ["bf16x3", "fp16x3", "fp32"]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.lib()
    yield


def _case(name, spread=2.0):
    """A few thousand events over a grid of 3 x 5 tiles in the plane with ragged
    edges, some events outside it, per-event bandwidths around (hs, ht)."""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    gx, gy, gt = 45, 37, 300
    n = 3000
    sres, tres = 0.5, 2.0
    org = (-20.0, 13.5, 100.0)
    vox = np.vstack([synth.clustered_events(rng, n - 600, gx, gy, gt, 6, (3.0, 8.0), (5.0, 30.0)),
                     synth.tiny(rng, 600, gx, gy, gt, spill=0.2)])
    pts = np.column_stack([org[0] + vox[:, 0] * sres, org[1] + vox[:, 1] * sres,
                           org[2] + vox[:, 2] * tres])
    hs, ht = synth.adaptive_bandwidths(n, 5.0 * sres, 9.0 * tres, spread=spread,
                                       seed=zlib.crc32(name.encode()) % 1000)
    return dict(pts=np.ascontiguousarray(pts), hs=hs, ht=ht, dims=(gx, gy, gt), org=org,
                sres=sres, tres=tres)


def _oracle(c):
    p = oracle.params(*c["dims"], 1.0, 1.0, x0=c["org"][0], y0=c["org"][1], t0=c["org"][2],
                      sres=c["sres"], tres=c["tres"])
    return oracle.pb_adaptive(c["pts"], c["hs"], c["ht"], p, with_slack=True)


def _gpu(form, c, host_bw=False, host_pts=False):
    pts = torch.from_numpy(c["pts"])
    hs, ht = torch.from_numpy(c["hs"]), torch.from_numpy(c["ht"])
    if not host_pts:
        pts = pts.cuda()
    if not host_bw:
        hs, ht = hs.cuda(), ht.cuda()
    with pkg.Context(form=form) as ctx:
        out = torch.full(c["dims"], float("nan"), dtype=torch.float32, device="cuda")
        ctx.compute_adaptive(pts, c["dims"], hs, ht, out, origin=c["org"], sres=c["sres"],
                             tres=c["tres"])
        ctx.synchronize()
        return out.cpu().numpy()


@pytest.fixture(scope="module")
def case():
    c = _case("adaptive-small")
    c["ref"], c["slack"] = _oracle(c)
    return c


@pytest.mark.parametrize("form", FORMS)
def test_adaptive_full_grid_parity(form, case):
    got = _gpu(form, case)
    assert not np.isnan(got).any()
    err = pu.excess_error(got, case["ref"], case["slack"])
    assert err <= pu.TOL[form], err


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_adaptive_wide_bandwidth_range(form):
    """Bandwidths spread over a factor of 36 (spatial) and 36 (temporal): the
    per-event weights reach 36^3 relative to the largest bandwidth."""
    c = _case("adaptive-wide", spread=6.0)
    ref, slack = _oracle(c)
    got = _gpu(form, c)
    assert pu.excess_error(got, ref, slack) <= pu.TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_equal_bandwidths_match_stkde_compute(form, case):
    c = dict(case)
    n = c["pts"].shape[0]
    hs, ht = 2.6, 17.0
    c["hs"], c["ht"] = np.full(n, hs), np.full(n, ht)
    got = _gpu(form, c)
    with pkg.Context(form=form) as ctx:
        ref = ctx.compute(torch.from_numpy(c["pts"]).cuda(), c["dims"], hs, ht, origin=c["org"],
                          sres=c["sres"], tres=c["tres"])
        ctx.synchronize()
        ref = ref.cpu().numpy()
    assert np.abs(got.astype(np.float64) - ref).max() <= pu.TOL[form] * ref.max()


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_host_and_device_arrays_give_the_same_bits(form, case):
    a = _gpu(form, case)
    b = _gpu(form, case, host_bw=True, host_pts=True)
    assert np.array_equal(a, b)


def test_sampled_tiles_of_the_clustered_workload():
    """The 200k-event clustered workload on 512 x 512 x 256 with bandwidths
    log-uniform in [5, 20] x [4, 16] voxels, on sampled tiles (densest, edges,
    corners, random) against the oracle evaluated box by box."""
    w = synth.medium()
    hs, ht = synth.adaptive_bandwidths(w.n, w.hs, w.ht, spread=2.0, seed=1)
    with pkg.Context(form="bf16x3") as ctx:
        out = ctx.compute_adaptive(torch.from_numpy(w.points).cuda(), (w.gx, w.gy, w.gt),
                                   torch.from_numpy(hs).cuda(), torch.from_numpy(ht).cuda())
        ctx.synchronize()
    p = oracle.params(w.gx, w.gy, w.gt, 1.0, 1.0)
    boxes = pu.sample_tile_boxes(w.points, w.gx, w.gy, w.gt, n_random=8, seed=3)[:16]
    refs = oracle.pb_adaptive_boxes(w.points, hs, ht, p, boxes)
    scale = max(r.max() for r, _ in refs)
    err = 0.0
    for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, refs):
        sub = out[x0:x1, y0:y1, t0:t1].cpu().numpy()
        err = max(err, pu.excess_error(sub, ref, slack, scale=scale))
    assert err <= pu.TOL["bf16x3"], err


def test_invalid_bandwidths_and_forms(case):
    lib = pkg.lib()
    c = case
    n = c["pts"].shape[0]
    g = pkg.make_grid(*c["dims"], *c["org"], sres=c["sres"], tres=c["tres"])
    pts = torch.from_numpy(c["pts"]).cuda()
    out = torch.empty(c["dims"], dtype=torch.float32, device="cuda")
    call = lambda ctx, hs, ht, m=n: lib.stkde_compute_adaptive(
        ctx.handle, pkg._ptr(pts), m, ctypes.byref(g), pkg._ptr(hs), pkg._ptr(ht), pkg._ptr(out))
    with pkg.Context(form="bf16x3") as ctx:
        bad = c["hs"].copy()
        bad[17] = -1.0
        assert call(ctx, bad, c["ht"]) == pkg.ERR_INVALID_ARGUMENT
        dbad = torch.from_numpy(c["ht"]).cuda()
        dbad[n - 1] = float("nan")
        assert call(ctx, torch.from_numpy(c["hs"]).cuda(), dbad) == pkg.ERR_INVALID_ARGUMENT
        dzero = torch.from_numpy(c["hs"]).cuda()
        dzero[0] = 0.0
        assert call(ctx, dzero, c["ht"]) == pkg.ERR_INVALID_ARGUMENT
        assert call(ctx, None, c["ht"]) == pkg.ERR_INVALID_ARGUMENT
        assert call(ctx, c["hs"], c["ht"], -1) == pkg.ERR_INVALID_ARGUMENT
        out.fill_(1.0)
        assert call(ctx, None, None, 0) == pkg.OK
        ctx.synchronize()
        assert not out.any().item()
    for form in ("scatter", "tf32x3", "tf32x1"):  # fixed bandwidths only
        with pkg.Context(form=form) as ctx:
            assert call(ctx, c["hs"], c["ht"]) == pkg.ERR_UNSUPPORTED
    with pkg.Context(form="fp16x3") as ctx:
        wide = c["hs"].copy()
        wide[0] = wide.max() * 200.0
        assert call(ctx, wide, c["ht"]) == pkg.ERR_UNSUPPORTED


def test_update_count_matches_the_oracle(case):
    """The per-event update count equals the sum of the oracle's exact one-event
    counts, each with its own bandwidths (binary32 re-centred events)."""
    c = case
    m = 400
    pts, hs, ht = c["pts"][:m], c["hs"][:m], c["ht"][:m]
    kw = dict(x0=c["org"][0], y0=c["org"][1], t0=c["org"][2], sres=c["sres"], tres=c["tres"])
    ref = sum(oracle.count_updates(pts[i:i + 1], oracle.params(*c["dims"], hs[i], ht[i], **kw))
              for i in range(m))
    with pkg.Context() as ctx:
        got_dev = ctx.count_updates_adaptive(torch.from_numpy(pts).cuda(), c["dims"],
                                             torch.from_numpy(hs).cuda(), torch.from_numpy(ht).cuda(),
                                             origin=c["org"], sres=c["sres"], tres=c["tres"])
        got_host = ctx.count_updates_adaptive(pts, c["dims"], hs, ht, origin=c["org"], sres=c["sres"],
                                              tres=c["tres"])
        fixed = ctx.count_updates(pts, c["dims"], 2.5, 17.0, origin=c["org"], sres=c["sres"],
                                  tres=c["tres"])
        same = ctx.count_updates_adaptive(pts, c["dims"], np.full(m, 2.5), np.full(m, 17.0),
                                          origin=c["org"], sres=c["sres"], tres=c["tres"])
    assert ref > 0
    assert got_dev == ref and got_host == ref
    assert same == fixed


def _edge_cases():
    rng = np.random.default_rng(zlib.crc32(b"adaptive-edges"))
    cases = []
    # one event, sub-voxel bandwidths
    cases.append(("one-tiny", np.array([[10.3, 7.6, 4.4]]), np.array([0.7]), np.array([0.6]), (24, 20, 12)))
    # events far outside the grid whose large cylinders reach in, beside small ones inside
    far = np.array([[-30.0, 5.0, 10.0], [70.0, 40.0, 3.0], [20.0, -25.0, 60.0]])
    near = synth.tiny(rng, 200, 40, 36, 50, spill=0.0)
    pts = np.vstack([far, near])
    hs = np.r_[np.array([34.0, 40.0, 30.0]), rng.uniform(0.8, 3.0, 200)]
    ht = np.r_[np.array([12.0, 9.0, 15.0]), rng.uniform(0.8, 4.0, 200)]
    cases.append(("far-reach", pts, hs, ht, (40, 36, 50)))
    # a single time slice
    pts = synth.tiny(rng, 300, 50, 30, 1, spill=0.2)
    cases.append(("gt1", pts, rng.uniform(1.0, 8.0, 300), rng.uniform(0.3, 2.0, 300), (50, 30, 1)))
    # bandwidths over a factor of 100 (more halvings than bandwidth classes)
    pts = synth.tiny(rng, 800, 48, 40, 70, spill=0.1)
    hs = np.where(rng.random(800) < 0.5, 0.3, 30.0) * rng.uniform(0.9, 1.1, 800)
    ht = rng.uniform(0.5, 12.0, 800)
    cases.append(("ratio-100", pts, hs, ht, (48, 40, 70)))
    return cases


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
@pytest.mark.parametrize("case", _edge_cases(), ids=lambda c: c[0])
def test_adaptive_edge_cases(form, case):
    name, pts, hs, ht, dims = case
    p = oracle.params(*dims, 1.0, 1.0)
    ref, slack = oracle.pb_adaptive(pts, hs, ht, p, with_slack=True)
    with pkg.Context(form=form) as ctx:
        out = ctx.compute_adaptive(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), dims,
                                   torch.from_numpy(hs).cuda(), torch.from_numpy(ht).cuda())
        ctx.synchronize()
        got = out.cpu().numpy()
    assert ref.max() > 0, name
    assert pu.excess_error(got, ref, slack) <= pu.TOL[form], name
