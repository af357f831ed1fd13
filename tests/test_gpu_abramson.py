"""GPU: per-event bandwidths from a pilot density (stkde_abramson_bandwidths).

With the GPU's own pilot grid handed to the oracle, the sampling at the events,
the floor, the geometric mean and the law must agree with the FP64 oracle to
rounding; the pilot itself is stkde_compute, parity-tested elsewhere.  The
bandwidths then drive stkde_compute_adaptive, compared with the oracle's
adaptive PB on the same bandwidths.
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


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.lib()
    yield


def _case():
    rng = np.random.default_rng(zlib.crc32(b"abramson"))
    G = (60, 52, 80)
    pts = np.vstack([synth.clustered_events(rng, 2500, *G, 5, (2.0, 7.0), (3.0, 12.0)),
                     synth.tiny(rng, 500, *G, spill=0.15)])
    return np.ascontiguousarray(pts), G


@pytest.mark.parametrize("alpha,lam", [(0.5, (0.125, 8.0)), (1.0, (0.5, 2.0)), (0.0, (1.0, 1.0))])
def test_bandwidths_match_the_oracle_on_the_same_pilot(alpha, lam):
    pts, G = _case()
    hs, ht = 3.0, 4.0
    with pkg.Context(form="bf16x3") as c:
        pilot = torch.empty(G, dtype=torch.float32, device="cuda")
        hs_i, ht_i = c.abramson_bandwidths(torch.from_numpy(pts).cuda(), G, hs, ht, alpha=alpha,
                                           lam_min=lam[0], lam_max=lam[1], pilot=pilot)
        c.synchronize()
    p = oracle.params(*G, hs, ht)
    ref_hs, ref_ht, _ = oracle.abramson(pts, p, alpha=alpha, lam_min=lam[0], lam_max=lam[1],
                                        pilot=pilot.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(hs_i.cpu().numpy(), ref_hs, rtol=1e-12)
    np.testing.assert_allclose(ht_i.cpu().numpy(), ref_ht, rtol=1e-12)


def test_adaptive_density_from_gpu_bandwidths():
    pts, G = _case()
    with pkg.Context(form="bf16x3") as c:
        dpts = torch.from_numpy(pts).cuda()
        hs_i, ht_i = c.abramson_bandwidths(dpts, G, 3.0, 4.0)
        out = c.compute_adaptive(dpts, G, hs_i, ht_i)
        c.synchronize()
    hs_h, ht_h = hs_i.cpu().numpy(), ht_i.cpu().numpy()
    assert hs_h.min() < 3.0 < hs_h.max()  # the law spread the bandwidths
    ref, slack = oracle.pb_adaptive(pts, hs_h, ht_h, oracle.params(*G, 1.0, 1.0), with_slack=True)
    assert pu.excess_error(out.cpu().numpy(), ref, slack) <= pu.TOL["bf16x3"]


def test_own_pilot_buffer_and_host_events_give_the_same_bits():
    pts, G = _case()
    with pkg.Context(form="bf16x3") as c:
        a = c.abramson_bandwidths(torch.from_numpy(pts).cuda(), G, 3.0, 4.0)
        b = c.abramson_bandwidths(pts, G, 3.0, 4.0,
                                  pilot=torch.empty(G, dtype=torch.float32, device="cuda"))
        c.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_invalid_arguments():
    pts, G = _case()
    lib = pkg.lib()
    g = pkg.make_grid(*G)
    d = torch.from_numpy(pts).cuda()
    n = pts.shape[0]
    hs_o = torch.empty(n, dtype=torch.float64, device="cuda")
    ht_o = torch.empty(n, dtype=torch.float64, device="cuda")
    host_o = np.empty(n)
    with pkg.Context() as c:
        call = lambda alpha=0.5, lmin=0.125, lmax=8.0, hso=hs_o, hto=ht_o: lib.stkde_abramson_bandwidths(
            c.handle, pkg._ptr(d), n, ctypes.byref(g), 3.0, 4.0, alpha, lmin, lmax, None,
            pkg._ptr(hso), pkg._ptr(hto))
        assert call() == pkg.OK
        assert call(alpha=-0.1) == pkg.ERR_INVALID_ARGUMENT
        assert call(lmin=0.0) == pkg.ERR_INVALID_ARGUMENT
        assert call(lmin=1.5) == pkg.ERR_INVALID_ARGUMENT
        assert call(lmax=0.5) == pkg.ERR_INVALID_ARGUMENT
        assert call(hso=host_o) == pkg.ERR_INVALID_ARGUMENT
        assert call(hso=None) == pkg.ERR_INVALID_ARGUMENT
        c.synchronize()


def _event_voxels(pts, G):
    """Voxel of each event, clamped into the grid (the sampling rule of the law)."""
    v = np.floor(pts).astype(np.int64)
    return tuple(np.clip(v[:, k], 0, G[k] - 1) for k in range(3))


@pytest.mark.parametrize("alpha,lam", [(0.5, (0.125, 8.0)), (1.0, (0.5, 2.0))])
def test_chain_against_the_oracle_with_its_own_pilot(alpha, lam):
    """The whole chain against the oracle end to end: the oracle computes its own
    FP64 pilot, its bandwidths from it, and the adaptive density on them.

    Bandwidths: the GPU pilot is a sum of non-negative terms, each carried with
    about 2^-16 relative error by the split-bf16 products, so at an event whose
    pilot value is at least 1e-3 of the largest sampled value both sides' f_i
    agree to about 1e-5 relative, and lambda_i = (f_i / g)^-alpha to rtol 1e-4
    (the clamp and the floor are 1-Lipschitz in log space and cannot widen
    this).  Events below 1e-3 of the largest value are excluded from that
    bound (the parity gate bounds the pilot's error relative to the grid
    maximum only): they are checked to lie in [lam_min, lam_max] and, where the
    oracle's pilot is exactly zero without tie slack (no event reaches the
    voxel), to get exactly zero from the GPU too.  Density: the GPU's adaptive
    density on the oracle's bandwidths against the oracle's adaptive PB, within
    the bf16x3 parity gate after the tie slack."""
    pts, G = _case()
    hs, ht = 3.0, 4.0
    p = oracle.params(*G, hs, ht)
    ref_hs, ref_ht, ref_lam = oracle.abramson(pts, p, alpha=alpha, lam_min=lam[0], lam_max=lam[1])
    pil_ref, pil_slack = oracle.pb(pts, p, with_slack=True)
    d = torch.from_numpy(pts).cuda()
    with pkg.Context(form="bf16x3") as c:
        pilot = torch.empty(G, dtype=torch.float32, device="cuda")
        hs_i, ht_i = c.abramson_bandwidths(d, G, hs, ht, alpha=alpha, lam_min=lam[0],
                                           lam_max=lam[1], pilot=pilot)
        c.synchronize()
    lam_gpu = hs_i.cpu().numpy() / hs
    np.testing.assert_allclose(ht_i.cpu().numpy() / ht, lam_gpu, rtol=1e-15)
    vx = _event_voxels(pts, G)
    f_ref = pil_ref[vx]
    dense = f_ref >= 1e-3 * f_ref.max()
    assert dense.mean() > 0.8  # the bound covers most events
    rel = np.abs(lam_gpu / ref_lam - 1.0)
    assert rel[dense].max() <= 1e-4, rel[dense].max()
    assert lam_gpu.min() >= lam[0] and lam_gpu.max() <= lam[1]
    empty = (f_ref == 0.0) & (pil_slack[vx] == 0.0)
    assert (pilot.cpu().numpy()[vx][empty] == 0.0).all()

    # the density on the oracle's own bandwidths
    with pkg.Context(form="bf16x3") as c:
        out = c.compute_adaptive(d, G, torch.from_numpy(ref_hs).cuda(), torch.from_numpy(ref_ht).cuda())
        c.synchronize()
    ref, slack = oracle.pb_adaptive(pts, ref_hs, ref_ht, p, with_slack=True)
    assert pu.excess_error(out.cpu().numpy(), ref, slack) <= pu.TOL["bf16x3"]
