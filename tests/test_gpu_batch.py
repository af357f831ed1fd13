"""GPU: the batched entry point stkde_compute_batch.

One re-centre, one sort and one bounds pass over the concatenated events of all
problems, then one tile-kernel launch whose queue holds the tiles of every
problem (tensor forms; one fp32 launch per problem).  Each problem must come out
bit-identical to its own stkde_compute with the same form (the same kernels see
the same events in the same order), and within the parity tolerance of the FP64
oracle on sampled tiles.  The batch mixes the uneven instances of the batched
workload (n log-uniform, grids 64^3 .. 512x512x128, hs and ht drawn per
instance) with an empty problem, a one-event problem, host-resident events and a
shifted origin with non-unit resolution.
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

FORMS = ["bf16x3", "fp16x3", "tf32x3", "tf32x1", "fp32"]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.lib()
    yield


def _workloads():
    ws = synth.batched(count=8)
    rng = np.random.default_rng(zlib.crc32(b"batch-edges"))
    empty = synth.Workload("empty", np.zeros((0, 3)), 40, 24, 30, 3.0, 2.0)
    one = synth.Workload("one", np.array([[10.3, 7.9, 12.2]]), 32, 32, 32, 5.0, 4.0)
    vox = synth.tiny(rng, 700, 50, 44, 70)
    sres, tres, org = 0.37, 3.0, (-1234.5, 77.25, 5000.0)
    pts = np.column_stack([org[0] + vox[:, 0] * sres, org[1] + vox[:, 1] * sres, org[2] + vox[:, 2] * tres])
    shifted = synth.Workload("shifted", np.ascontiguousarray(pts), 50, 44, 70, 2.1 * sres, 9.0 * tres,
                             *org, sres, tres)
    return ws[:4] + [empty, one, shifted] + ws[4:]


HOST_INDEX = 2  # this problem's events stay in host memory


def _grid(w):
    return pkg.make_grid(w.gx, w.gy, w.gt, w.x0, w.y0, w.t0, sres=w.sres, tres=w.tres)


def _single(ctx, w):
    out = torch.full((w.gx, w.gy, w.gt), float("nan"), dtype=torch.float32, device="cuda")
    pts = torch.from_numpy(w.points).cuda()
    pkg.stkde_compute(ctx.handle, pts if w.n else None, w.n, _grid(w), w.hs, w.ht, out)
    return out


def _batch(ctx, ws):
    outs, probs, keep = [], [], []
    for i, w in enumerate(ws):
        out = torch.full((w.gx, w.gy, w.gt), float("nan"), dtype=torch.float32, device="cuda")
        pts = torch.from_numpy(w.points) if i == HOST_INDEX else torch.from_numpy(w.points).cuda()
        keep.append(pts)
        outs.append(out)
        probs.append(pkg.Problem(pkg._ptr(pts) if w.n else None, w.n, _grid(w), w.hs, w.ht,
                                 pkg._ptr(out)))
    pkg.stkde_compute_batch(ctx.handle, probs)
    ctx.synchronize()
    return outs


@pytest.fixture(scope="module")
def workloads():
    return _workloads()


@pytest.mark.parametrize("form", FORMS)
def test_batch_bitwise_equals_single_calls(form, workloads):
    with pkg.Context(form=form) as c:
        got = _batch(c, workloads)
        for w, g in zip(workloads, got):
            ref = _single(c, w)
            c.synchronize()
            assert not torch.isnan(g).any().item(), w.name
            assert torch.equal(g, ref), w.name


@pytest.mark.parametrize("form", ["bf16x3", "tf32x3", "fp32"])
def test_batch_against_oracle(form, workloads):
    with pkg.Context(form=form) as c:
        got = _batch(c, workloads)
    for k, (w, g) in enumerate(zip(workloads, got)):
        p = oracle.params(w.gx, w.gy, w.gt, w.hs, w.ht, x0=w.x0, y0=w.y0, t0=w.t0, sres=w.sres,
                          tres=w.tres)
        if w.gx * w.gy * w.gt <= 200_000:
            ref, slack = oracle.pb(w.points, p, with_slack=True)
            err = pu.excess_error(g.cpu().numpy(), ref, slack)
        else:
            boxes = pu.sample_tile_boxes(w.points, w.gx, w.gy, w.gt, n_random=4, seed=k)[:10]
            refs = oracle.pb_boxes(w.points, p, boxes)
            scale = max(max(r.max() for r, _ in refs), 1e-300)
            err = 0.0
            for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, refs):
                sub = g[x0:x1, y0:y1, t0:t1].cpu().numpy()
                err = max(err, pu.excess_error(sub, ref, slack, scale=scale))
        if w.n == 0:
            assert not g.any().item()
        assert err <= pu.TOL[form], (w.name, err)


def test_batch_invalid_arguments(workloads):
    w = workloads[0]
    lib = pkg.lib()
    pts = torch.from_numpy(w.points).cuda()
    with pkg.Context(form="scatter") as c:
        out = torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda")
        arr = (pkg.Problem * 1)(pkg.Problem(pkg._ptr(pts), w.n, _grid(w), w.hs, w.ht, pkg._ptr(out)))
        assert lib.stkde_compute_batch(c.handle, arr, 1) == pkg.ERR_UNSUPPORTED
    with pkg.Context(form="bf16x3") as c:
        hout = np.empty((w.gx, w.gy, w.gt), dtype=np.float32)
        arr = (pkg.Problem * 1)(pkg.Problem(pkg._ptr(pts), w.n, _grid(w), w.hs, w.ht, hout.ctypes.data))
        assert lib.stkde_compute_batch(c.handle, arr, 1) == pkg.ERR_INVALID_ARGUMENT
        bad = (pkg.Problem * 1)(pkg.Problem(pkg._ptr(pts), w.n, _grid(w), -1.0, w.ht, pkg._ptr(out)))
        assert lib.stkde_compute_batch(c.handle, bad, 1) == pkg.ERR_INVALID_ARGUMENT
        assert lib.stkde_compute_batch(c.handle, None, 0) == pkg.OK
        assert lib.stkde_compute_batch(c.handle, ctypes.cast(None, ctypes.POINTER(pkg.Problem)), 2) == \
            pkg.ERR_INVALID_ARGUMENT
