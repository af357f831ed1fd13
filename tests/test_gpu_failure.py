"""GPU: failure paths, injected on the host side or as a wait nothing satisfies
(include/stkde_testing.h); no test makes the device fault.

- A bounded wait that expires: block 0 of the tensor tile kernel withholds the
  arrival of its first staging page (issuing no copy into it) and every wait of
  that launch is bounded at 200 us.  The call must report STKDE_ERR_TIMEOUT from
  stkde_synchronize within the wait bound plus the drain bound, and the same
  context must then compute the grid bit for bit as before.
- A device allocation that fails: the workspace, the result buffer for host
  outputs and the staging of host bandwidth arrays each fail once; the call must
  return STKDE_ERR_OOM before enqueueing anything, hold no device memory it did
  not hold before, and the context must then compute correctly.
- Stream capture: a call that would have to grow a buffer is refused with
  STKDE_ERR_UNSUPPORTED and leaves the capture intact.
"""
import time

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


def _status(exc_info):
    return exc_info.value.status


@pytest.mark.parametrize("form", ["bf16x3", "fp16x3", "tf32x3"])
def test_withheld_page_times_out_and_the_context_recovers(form):
    w = synth.medium()
    pts = torch.from_numpy(w.points).cuda()
    dims = (w.gx, w.gy, w.gt)
    with pkg.Context(form=form) as c:
        ref = c.compute(pts, dims, w.hs, w.ht)
        c.synchronize()
        out = torch.zeros_like(ref)
        c.inject_fault(pkg.FAULT_WITHHOLD_PAGE, 200)  # 200 us bound on every wait
        t0 = time.perf_counter()
        c.compute(pts, dims, w.hs, w.ht, out=out)
        with pytest.raises(pkg.StkdeError) as e:
            c.synchronize()
        dt = time.perf_counter() - t0
        assert _status(e) == pkg.ERR_TIMEOUT
        # wait bound, then at most the drain bound (200 ms) per pending page wait
        assert dt < 1.5, dt
        # the error is cleared and the hook was one-shot: the same context is correct again
        c.synchronize()
        again = c.compute(pts, dims, w.hs, w.ht)
        c.synchronize()
        assert torch.equal(again, ref)


def test_withheld_page_in_a_batch():
    ws = [synth.small(), synth.medium()]
    pts = [torch.from_numpy(w.points).cuda() for w in ws]
    with pkg.Context(form="bf16x3") as c:
        outs = [torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda") for w in ws]
        probs = [(p, (w.gx, w.gy, w.gt), w.hs, w.ht, o) for p, w, o in zip(pts, ws, outs)]
        c.compute_batch(probs)
        c.synchronize()
        refs = [o.clone() for o in outs]
        c.inject_fault(pkg.FAULT_WITHHOLD_PAGE, 200)
        c.compute_batch(probs)
        with pytest.raises(pkg.StkdeError) as e:
            c.synchronize()
        assert _status(e) == pkg.ERR_TIMEOUT
        c.compute_batch(probs)
        c.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


# allocations of stkde_compute in order: result buffer (host output only), workspace
@pytest.mark.parametrize("host_out,nth", [(False, 1), (True, 1), (True, 2)])
def test_failed_allocation_reports_oom_and_leaks_nothing(host_out, nth):
    w = synth.medium()
    pts = torch.from_numpy(w.points).cuda()
    dims = (w.gx, w.gy, w.gt)
    with pkg.Context(form="bf16x3") as good:
        ref = good.compute(pts, dims, w.hs, w.ht).cpu()
        good.synchronize()
    c = pkg.Context(form="bf16x3")
    try:
        before = _free()
        c.inject_fault(pkg.FAULT_ALLOC, nth)
        out = np.full(dims, np.nan, dtype=np.float32) if host_out else \
            torch.full(dims, float("nan"), dtype=torch.float32, device="cuda")
        with pytest.raises(pkg.StkdeError) as e:
            c.compute(pts, dims, w.hs, w.ht, out=out)
        assert _status(e) == pkg.ERR_OOM
        c.synchronize()  # nothing latched
        # nothing was enqueued (the output is untouched); the context holds only
        # the buffers that did grow (the result buffer when the workspace failed)
        got = out if host_out else out.cpu().numpy()
        assert np.isnan(got).all()
        held = 4 * w.gx * w.gy * w.gt if (host_out and nth == 2) else 0
        assert _free() >= before - held - (2 << 20)
        # the context works afterwards
        c.compute(pts, dims, w.hs, w.ht, out=out)
        c.synchronize()
        got = torch.from_numpy(out) if host_out else out.cpu()
        assert torch.equal(got, ref)
    finally:
        c.close()
    # destroying the context returns what it held (allocation granularity aside)
    assert _free() >= before - (4 << 20)


def test_failed_bandwidth_staging_reports_oom():
    w = synth.small()
    pts = torch.from_numpy(w.points).cuda()
    dims = (w.gx, w.gy, w.gt)
    hs, ht = synth.adaptive_bandwidths(w.n, w.hs, w.ht, spread=2.0, seed=3)
    with pkg.Context(form="bf16x3") as c:
        c.inject_fault(pkg.FAULT_ALLOC, 1)  # the staging buffer of the host arrays
        with pytest.raises(pkg.StkdeError) as e:
            c.compute_adaptive(pts, dims, hs, ht)
        assert _status(e) == pkg.ERR_OOM
        a = c.compute_adaptive(pts, dims, hs, ht)
        b = c.compute_adaptive(pts, dims, torch.from_numpy(hs).cuda(), torch.from_numpy(ht).cuda())
        c.synchronize()
        assert torch.equal(a, b)


def test_fault_arguments_are_checked():
    with pkg.Context() as c:
        for fault, arg in ((pkg.FAULT_ALLOC, 0), (pkg.FAULT_WITHHOLD_PAGE, 0),
                           (pkg.FAULT_WITHHOLD_PAGE, 2_000_001), (17, 1)):
            with pytest.raises(pkg.StkdeError) as e:
                c.inject_fault(fault, arg)
            assert _status(e) == pkg.ERR_INVALID_ARGUMENT
        c.inject_fault(pkg.FAULT_ALLOC, 1)
        c.inject_fault(pkg.FAULT_NONE)  # disarmed: the next call allocates normally
        w = synth.small()
        c.compute(torch.from_numpy(w.points).cuda(), (w.gx, w.gy, w.gt), w.hs, w.ht)
        c.synchronize()


def test_capture_refuses_growth_and_keeps_the_capture_valid():
    w = synth.small()
    pts = torch.from_numpy(w.points).cuda()
    out = torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with pkg.Context(stream=s) as c:  # fresh: empty workspace
        g = torch.cuda.CUDAGraph()
        with pu.captured(torch, g, s):
            out.zero_()
            with pytest.raises(pkg.StkdeError) as e:
                c.compute(pts, (w.gx, w.gy, w.gt), w.hs, w.ht, out=out)
            assert _status(e) == pkg.ERR_UNSUPPORTED
            with pytest.raises(pkg.StkdeError) as e:  # synchronous entry points too
                c.count_updates(pts, (w.gx, w.gy, w.gt), w.hs, w.ht)
            assert _status(e) == pkg.ERR_UNSUPPORTED
        out.fill_(1.0)
        g.replay()  # the capture stayed valid: it holds the zero fill
        torch.cuda.synchronize()
        assert not out.any().item()
        c.compute(pts, (w.gx, w.gy, w.gt), w.hs, w.ht, out=out)
        c.synchronize()
