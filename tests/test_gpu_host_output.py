"""GPU: host output buffers.

With a host output grid of at least two 64 MB slabs, the tensor forms compute the
grid slab by slab along X and copy each slab to the host on a second stream while
the later slabs compute.  The result must be bit-identical to the same call with a
device output (the slabs' tile kernels see the same events in the same order),
for pinned and pageable host memory, for the fixed and the per-event bandwidth
entry points, and stay stream-ordered with later work.
"""
import numpy as np
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


@pytest.fixture(scope="module")
def medium():
    return synth.medium()


@pytest.mark.parametrize("form", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("pinned", [True, False])
def test_slabbed_host_output_is_bitwise_equal(form, pinned, medium):
    w = medium
    dims = (w.gx, w.gy, w.gt)
    pts = torch.from_numpy(w.points).cuda()
    with pkg.Context(form=form) as c:
        ref = c.compute(pts, dims, w.hs, w.ht)
        c.synchronize()
        ref = ref.cpu()
        host = torch.full(dims, float("nan"), dtype=torch.float32, pin_memory=pinned)
        c.compute(pts, dims, w.hs, w.ht, out=host)
        c.synchronize()
        assert c.last_launch_count() > 15  # several slab launches
    assert torch.equal(host, ref)


def test_host_output_is_ordered_before_later_work(medium):
    """A second call into the same host buffer right after the first: the stream
    waits for the first call's slab copies, so the buffer ends with the second
    result, whole."""
    w = medium
    dims = (w.gx, w.gy, w.gt)
    pts = torch.from_numpy(w.points).cuda()
    host = torch.empty(dims, dtype=torch.float32, pin_memory=True)
    with pkg.Context(form="bf16x3") as c:
        c.compute(pts, dims, w.hs, w.ht, out=host)
        c.compute(pts, dims, 2.0 * w.hs, w.ht, out=host)
        ref = c.compute(pts, dims, 2.0 * w.hs, w.ht)
        c.synchronize()
        assert torch.equal(host, ref.cpu())


def test_adaptive_host_output(medium):
    w = medium
    dims = (w.gx, w.gy, w.gt)
    hs, ht = synth.adaptive_bandwidths(w.n, w.hs, w.ht, spread=2.0, seed=4)
    pts = torch.from_numpy(w.points).cuda()
    with pkg.Context(form="bf16x3") as c:
        ref = c.compute_adaptive(pts, dims, torch.from_numpy(hs).cuda(), torch.from_numpy(ht).cuda())
        c.synchronize()
        host = np.full(dims, np.nan, dtype=np.float32)
        c.compute_adaptive(w.points, dims, hs, ht, out=host)
        c.synchronize()
    assert np.array_equal(host, ref.cpu().numpy())
