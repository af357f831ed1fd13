"""GPU parity: every form of the CUDA path against the FP64 oracle.

Element by element on the same seeded inputs: the full grid for the small
(64x64x32) and medium (512x512x256) workloads, and 64 sampled tiles (the
densest, corners, edges, random) of the large 1024x1024x512 workload in the
launch configuration the benchmark times.  Gates: max |gpu - oracle| over the
grid maximum, after the oracle's binary32 tie slack, <= 1e-5 (fp32, fp16x3,
tf32x3, scatter) and <= 2e-5 (bf16x3); the one-product tf32x1 form is reported
against a loose bound only.
"""
import zlib

import numpy as np
import pytest

import oracle
import paper_1705_09366_gb300 as pkg
import parity_util as pu
from paper_1705_09366_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE_FORMS = ["bf16x3", "fp16x3", "tf32x3", "fp32"]
ALL_FORMS = TILE_FORMS + ["scatter"]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.lib()
    yield


def run(form, w, *, kernel_constants=0, out=None, t_block=0, slab=0, host=False):
    with pkg.Context(form=form, kernel_constants=kernel_constants, t_block=t_block,
                     slab=slab) as c:
        pts = torch.from_numpy(w.points) if host else torch.from_numpy(w.points).cuda()
        if out is None:
            out = torch.full((w.gx, w.gy, w.gt), float("nan"), dtype=torch.float32,
                             device="cpu" if host else "cuda")
        c.compute(pts, (w.gx, w.gy, w.gt), w.hs, w.ht, out=out, origin=(w.x0, w.y0, w.t0),
                  sres=w.sres, tres=w.tres)
        c.synchronize()
    return out


def oracle_full(w, cs=oracle.CS_PRINTED):
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht, x0=w.x0, y0=w.y0, t0=w.t0, sres=w.sres,
                      tres=w.tres, cs=cs)
    return oracle.pb(w.points, p, with_slack=True)


@pytest.mark.parametrize("form", ALL_FORMS)
def test_small_full_grid(form):
    w = synth.small()
    ref, slack = oracle_full(w)
    got = run(form, w).cpu().numpy()
    assert np.isfinite(got).all()
    err = pu.excess_error(got, ref, slack)
    assert err <= pu.TOL[form], err


@pytest.mark.parametrize("form", ALL_FORMS)
def test_medium_full_grid(form):
    w = synth.medium()
    ref, slack = oracle_full(w)
    got = run(form, w).cpu().numpy()
    assert np.isfinite(got).all()
    err = pu.excess_error(got, ref, slack)
    assert err <= pu.TOL[form], err


@pytest.mark.parametrize("name", ["small", "medium"])
def test_tf32x1_reported(name):
    w = getattr(synth, name)()
    ref, slack = oracle_full(w)
    got = run("tf32x1", w).cpu().numpy()
    assert np.isfinite(got).all()
    err = pu.excess_error(got, ref, slack)
    print(f"tf32x1 {name}: max error {err:.3e} of the grid maximum (reported, not gated)")
    assert err <= pu.REPORT_ONLY_BOUND["tf32x1"], err


@pytest.fixture(scope="module")
def large_case():
    w = synth.large()
    boxes = pu.sample_tile_boxes(w.points, w.gx, w.gy, w.gt, n_random=48, seed=1)
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht)
    return w, boxes, oracle.pb_boxes(w.points, p, boxes)


@pytest.mark.parametrize("form", TILE_FORMS)
def test_large_sampled_tiles(form, large_case):
    w, boxes, refs = large_case
    out = run(form, w)
    scale = max(r.max() for r, _ in refs)
    worst = 0.0
    for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, refs):
        got = out[x0:x1, y0:y1, t0:t1].cpu().numpy()
        assert np.isfinite(got).all()
        worst = max(worst, pu.excess_error(got, ref, slack, scale=scale))
    assert worst <= pu.TOL[form], worst
    # every voxel written (no NaN left from the prefill) and none negative
    assert not torch.isnan(out).any().item()
    assert (out >= 0).all().item()


@pytest.mark.parametrize("form", TILE_FORMS)
def test_bitwise_deterministic(form):
    w = synth.medium()
    a = run(form, w)
    b = run(form, w)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with pkg.Context(form=form, stream=s) as c:
            cc = torch.empty_like(a)
            c.compute(torch.from_numpy(w.points).cuda(), (w.gx, w.gy, w.gt), w.hs, w.ht, out=cc)
            c.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a, cc)


def _case(name, rng, n, dims, hs, ht, origin=(0.0, 0.0, 0.0), sres=1.0, tres=1.0, spill=0.25):
    vox = synth.tiny(rng, n, *dims, spill=spill)
    pts = np.column_stack([origin[0] + vox[:, 0] * sres, origin[1] + vox[:, 1] * sres,
                           origin[2] + vox[:, 2] * tres])
    return synth.Workload(name, np.ascontiguousarray(pts), *dims, hs, ht, *origin, sres, tres)


EDGE = [
    ("ragged", 400, (37, 13, 45), 3.3, 2.2, (0, 0, 0), 1.0, 1.0),
    ("gt1", 300, (40, 33, 1), 4.5, 1.7, (0, 0, 0), 1.0, 1.0),
    ("h_below_voxel", 500, (30, 30, 20), 0.45, 0.3, (0, 0, 0), 1.0, 1.0),
    ("origin_res", 600, (50, 44, 70), 2.1, 9.0, (-1234.5, 77.25, 5000.0), 0.37, 3.0),
    ("wide_t", 800, (24, 24, 700), 3.0, 90.0, (0, 0, 0), 1.0, 1.0),
    ("wide_s", 200, (80, 80, 10), 60.0, 2.0, (0, 0, 0), 1.0, 1.0),
    ("single_tile", 50, (16, 8, 16), 2.5, 2.5, (0, 0, 0), 1.0, 1.0),
]


@pytest.mark.parametrize("form", ALL_FORMS)
@pytest.mark.parametrize("case", EDGE, ids=[e[0] for e in EDGE])
def test_edge_cases(form, case):
    name, n, dims, hs, ht, origin, sres, tres = case
    w = _case(name, np.random.default_rng(zlib.crc32(name.encode())), n, dims, hs * sres, ht * tres,
              origin, sres, tres)
    ref, slack = oracle_full(w)
    got = run(form, w).cpu().numpy()
    assert np.isfinite(got).all()
    assert pu.excess_error(got, ref, slack) <= pu.TOL[form]


@pytest.mark.parametrize("form", ALL_FORMS)
def test_empty_and_single_event(form):
    w0 = synth.Workload("empty", np.zeros((0, 3)), 20, 17, 9, 3.0, 2.0)
    got = run(form, w0)
    assert (got == 0).all().item()
    w1 = synth.Workload("one", np.array([[10.3, 8.6, 4.2]]), 20, 17, 9, 3.0, 2.0)
    ref, slack = oracle_full(w1)
    assert pu.excess_error(run(form, w1).cpu().numpy(), ref, slack) <= pu.TOL[form]
    far = synth.Workload("far", np.array([[1e7, -3e6, 4.0]]), 20, 17, 9, 3.0, 2.0)
    assert (run(form, far) == 0).all().item()


@pytest.mark.parametrize("form", TILE_FORMS)
def test_unit_mass_constants(form):
    w = synth.small()
    ref, slack = oracle_full(w, cs=oracle.CS_UNIT_MASS)
    got = run(form, w, kernel_constants=pkg.KERNEL_UNIT_MASS).cpu().numpy()
    assert pu.excess_error(got, ref, slack) <= pu.TOL[form]


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_host_buffers_match_device_buffers(form):
    w = synth.small()
    dev = run(form, w)
    host = run(form, w, host=True)
    assert torch.equal(dev.cpu(), host)


def test_nonfinite_event_is_reported():
    pts = synth.small().points.copy()
    pts[17, 1] = np.nan
    with pkg.Context(form="fp32") as c:
        out = torch.empty((64, 64, 32), dtype=torch.float32, device="cuda")
        c.compute(torch.from_numpy(pts).cuda(), (64, 64, 32), 4.0, 3.0, out=out)
        with pytest.raises(pkg.StkdeError) as ei:
            c.synchronize()
        assert ei.value.status == pkg.ERR_NONFINITE
        c.synchronize()  # the error was cleared


def test_invalid_arguments_on_device():
    with pkg.Context(form="fp32") as c:
        pts = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
        out = torch.empty((4, 4, 4), dtype=torch.float32, device="cuda")
        for hs, ht, dims in [(0.0, 1.0, (4, 4, 4)), (1.0, -1.0, (4, 4, 4)),
                             (float("nan"), 1.0, (4, 4, 4)), (1.0, 1.0, (0, 4, 4))]:
            with pytest.raises(pkg.StkdeError) as ei:
                c.compute(pts, dims, hs, ht, out=out)
            assert ei.value.status == pkg.ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("wname", ["small", "medium"])
def test_update_count_matches_oracle(wname):
    w = synth.WORKLOADS[wname]()
    p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht)
    with pkg.Context(form="fp32") as c:
        got = c.count_updates(torch.from_numpy(w.points).cuda(), (w.gx, w.gy, w.gt), w.hs, w.ht)
    assert got == oracle.count_updates(w.points, p)


@pytest.mark.parametrize("form", ["bf16x3", "fp16x3", "tf32x3", "fp32", "scatter"])
def test_output_only_4_byte_aligned(form):
    """An output that starts 4 bytes past a 16-byte boundary (G_t a multiple of 4,
    so only the base breaks the vector path's alignment) gives the same grid."""
    w = synth.small()
    dims = (w.gx, w.gy, w.gt)
    n = w.gx * w.gy * w.gt
    ref = run(form, w)
    raw = torch.full((n + 4,), float("nan"), dtype=torch.float32, device="cuda")
    shifted = raw[1:1 + n].view(dims)
    assert shifted.data_ptr() % 16 == 4
    run(form, w, out=shifted)
    if form == "scatter":  # atomics: the last bits vary from run to run
        scale = float(ref.abs().max())
        assert float((shifted - ref).abs().max()) <= 1e-6 * scale
    else:
        assert torch.equal(shifted, ref)
    assert torch.isnan(raw[0]).item() and torch.isnan(raw[1 + n:]).all().item()


@pytest.mark.parametrize("form", ["bf16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("slab", [1, 2, 8, 32, 64, 1000])
def test_explicit_slabs(form, slab):
    """Every bin slab (the T extent of an event bin, including one longer than the
    grid's T extent) gives the density within the gate: the slab changes the
    binning and the summation order, never the set of events a voxel sums."""
    for name in ("ragged", "wide_t", "origin_res"):
        case = next(e for e in EDGE if e[0] == name)
        _, n, dims, hs, ht, origin, sres, tres = case
        w = _case(name, np.random.default_rng(zlib.crc32(name.encode())), n, dims, hs * sres,
                  ht * tres, origin, sres, tres)
        ref, slack = oracle_full(w)
        got = run(form, w, slab=slab).cpu().numpy()
        assert pu.excess_error(got, ref, slack) <= pu.TOL[form], (name, slab)
