"""GPU: capturing stkde_compute in a CUDA graph.

After one warm-up call has sized the context's workspace, a call with device
events and a device output enqueues only kernels, memsets and copies on the
context's stream, so it can be captured (here with torch.cuda.graph on that
stream) and replayed: each replay recomputes the grid from the current contents
of the event buffer, bit-identical to a direct call.  Replays remove the host
cost of the ~15 launches per call, which matters for small problems.
"""
import pytest

import paper_1705_09366_gb300 as pkg
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
        with torch.cuda.graph(g, stream=s):
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
