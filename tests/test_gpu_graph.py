"""GPU: capturing stkde_compute and stkde_compute_batch in a CUDA graph.

After one warm-up call has sized the context's workspace, a call with device
events and a device output enqueues only kernels, memsets and copies on the
context's stream, so it can be captured (here with torch.cuda.graph on that
stream) and replayed: each replay recomputes the grid from the current contents
of the event buffer, bit-identical to a direct call.  Replays remove the host
cost of the ~15 launches per call, which matters for small problems.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_graph_replay_matches_direct_calls(form):
    w = synth.small()
    w2 = synth.small(seed_offset=1)
    dims = (w.gx, w.gy, w.gt)
    s = torch.cuda.Stream()
    pts = torch.from_numpy(w.points).cuda()
    out = torch.empty(dims, dtype=torch.float32, device="cuda")
    grid = pkg.make_grid(*dims)
    with pkg.Context(form=form, stream=s) as c:
        with torch.cuda.stream(s):
            pkg.stkde_compute(c.handle, pts, w.n, grid, w.hs, w.ht, out)   # warm-up: workspace
        c.synchronize()
        ref1 = out.clone()
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            pkg.stkde_compute(c.handle, pts, w.n, grid, w.hs, w.ht, out)
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref1)
        # new events in the same buffer: the replay follows them
        pts.copy_(torch.from_numpy(w2.points))
        g.replay()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            direct = torch.empty_like(out)
            pkg.stkde_compute(c.handle, pts, w2.n, grid, w2.hs, w2.ht, direct)
        c.synchronize()
        assert torch.equal(out, direct)
        assert not torch.equal(out, ref1)


def _batch_case(count, seed):
    rng = np.random.default_rng(seed)
    ws = []
    for i in range(count):
        n = int(rng.integers(0, 3000)) if i % 11 else 0  # some empty problems
        dims = (int(rng.integers(8, 70)), int(rng.integers(8, 40)), int(rng.integers(1, 300)))
        vox = synth.tiny(rng, n, *dims, spill=0.2)
        ws.append((np.ascontiguousarray(vox), dims, float(rng.uniform(0.6, 6.0)),
                   float(rng.uniform(0.6, 12.0))))
    return ws


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_graph_replay_of_a_batch(form):
    """70 problems (two kernel-parameter chunks of the problem table) captured as
    one stkde_compute_batch; each replay equals the direct batch bit for bit and
    follows new event values written into the same buffers."""
    ws = _batch_case(70, 5)
    s = torch.cuda.Stream()
    pts = [torch.from_numpy(p).cuda() for p, _, _, _ in ws]
    outs = [torch.empty(d, dtype=torch.float32, device="cuda") for _, d, _, _ in ws]
    probs = [(p, d, hs, ht, o) for p, (_, d, hs, ht), o in zip(pts, ws, outs)]
    with pkg.Context(form=form, stream=s) as c:
        c.compute_batch(probs)   # warm-up: sizes the workspace
        c.synchronize()
        ref = [o.clone() for o in outs]
        # each problem alone gives the same grid
        for (p, d, hs, ht, _), r in zip(probs, ref):
            alone = c.compute(p, d, hs, ht)
            c.synchronize()
            assert torch.equal(alone, r)
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            c.compute_batch(probs)
        for o in outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
        # new event values in the same buffers (same counts): the replay follows them
        rng = np.random.default_rng(6)
        for p, (_, d, _, _) in zip(pts, ws):
            if p.shape[0]:
                p.copy_(torch.from_numpy(synth.tiny(rng, p.shape[0], *d, spill=0.2)))
        g.replay()
        torch.cuda.synchronize()
        got = [o.clone() for o in outs]
        c.compute_batch(probs)
        c.synchronize()
        for o, r in zip(outs, got):
            assert torch.equal(o, r)


def test_capture_refuses_host_events_in_a_batch():
    w = synth.small()
    s = torch.cuda.Stream()
    out = torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda")
    dpts = torch.from_numpy(w.points).cuda()
    with pkg.Context(stream=s) as c:
        c.compute_batch([(dpts, (w.gx, w.gy, w.gt), w.hs, w.ht, out)])
        c.synchronize()
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            out.zero_()
            with pytest.raises(pkg.StkdeError) as e:
                c.compute_batch([(w.points, (w.gx, w.gy, w.gt), w.hs, w.ht, out)])
            assert e.value.status == pkg.ERR_UNSUPPORTED
        g.replay()
        torch.cuda.synchronize()


def test_reserve_lets_a_larger_problem_be_captured():
    """stkde_reserve grows the workspace up front: after a warm-up on a small
    problem, a larger one (whose workspace would otherwise have to grow, which a
    capture refuses) is captured and replayed to the direct call's bits, and the
    call allocates no device memory."""
    small, big = synth.small(), synth.medium()
    s = torch.cuda.Stream()
    with pkg.Context(stream=s) as c:
        c.compute(torch.from_numpy(small.points).cuda(), (small.gx, small.gy, small.gt),
                  small.hs, small.ht, out=torch.empty((small.gx, small.gy, small.gt),
                                                      dtype=torch.float32, device="cuda"))
        c.synchronize()
        pts = torch.from_numpy(big.points).cuda()
        dims = (big.gx, big.gy, big.gt)
        out = torch.empty(dims, dtype=torch.float32, device="cuda")
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            out.zero_()
            with pytest.raises(pkg.StkdeError) as e:  # the workspace would have to grow
                c.compute(pts, dims, big.hs, big.ht, out=out)
            assert e.value.status == pkg.ERR_UNSUPPORTED
        c.reserve(64 << 20)  # 56 B per event and 4 B per 512 voxels fit in 64 MB
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        c.compute(pts, dims, big.hs, big.ht, out=out)  # a direct call allocates nothing now
        c.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            c.compute(pts, dims, big.hs, big.ht, out=out)
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        replayed = out.clone()
        c.compute(pts, dims, big.hs, big.ht, out=out)
        c.synchronize()
        assert torch.equal(replayed, out)
