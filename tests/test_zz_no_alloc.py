"""The allocation-free entry point stkde_compute_static.

It serves callers that cannot call cudaMalloc (another component owns every
device allocation, or their loop must not take cudaMalloc's device-wide
synchronisation).  Checked here through the C ABI: two calls in a row, each
compared with the allocating stkde_compute on the same inputs within the
tolerances of the parity tests; the device's free memory is the same before and
after a call; a call captured into a CUDA graph in global capture mode (where a
cudaMalloc would invalidate the capture) replays to the same bits; a call with
sync = 0 on a side stream completes with that stream; and the size limits are
refused before any launch.
This file is collected last, so a run that stops at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import ctypes

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


def _allocating(form, w, pts):
    with pkg.Context(form=form) as c:
        out = c.compute(pts, (w.gx, w.gy, w.gt), w.hs, w.ht)
        c.synchronize()
    return out


@pytest.mark.parametrize("wname,form", [("small", "bf16x3"), ("small", "fp32"),
                                        ("small", "fp16x3"), ("small", "tf32x3"),
                                        ("small", "scatter"), ("medium", "bf16x3")])
def test_static_entry_matches_allocating_entry_twice(wname, form):
    w = synth.WORKLOADS[wname]()
    pts = torch.from_numpy(w.points).cuda()
    ref = _allocating(form, w, pts).double()
    scale = float(ref.max())
    grid = pkg.make_grid(w.gx, w.gy, w.gt)
    for _ in range(2):
        out = torch.full((w.gx, w.gy, w.gt), float("nan"), dtype=torch.float32, device="cuda")
        pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, form=form, sync=True)
        assert not torch.isnan(out).any().item()
        err = float((out.double() - ref).abs().max()) / scale
        assert err <= pu.TOL[form], err


def test_static_entry_allocates_nothing():
    w = synth.small()
    pts = torch.from_numpy(w.points).cuda()
    grid = pkg.make_grid(w.gx, w.gy, w.gt)
    out = torch.empty((w.gx, w.gy, w.gt), dtype=torch.float32, device="cuda")
    pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, sync=True)  # modules loaded
    ref = out.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, sync=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, ref)

    # captured in global mode (any cudaMalloc in the call would invalidate the capture)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pu.captured(torch, g, s, capture_error_mode="global"):
        pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, stream=s, sync=False)
    out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # a captured call cannot wait for its stream
    g2 = torch.cuda.CUDAGraph()
    with pu.captured(torch, g2, s, capture_error_mode="global"):
        out.zero_()
        with pytest.raises(pkg.StkdeError) as e:
            pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, stream=s, sync=True)
        assert e.value.status == pkg.ERR_UNSUPPORTED

    # sync = 0 on a side stream: the result is there once that stream is done
    side = torch.cuda.Stream()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    pkg.stkde_compute_static(pts, w.n, grid, w.hs, w.ht, out, stream=side, sync=False)
    side.synchronize()
    assert torch.equal(out, ref)


def test_static_entry_refuses_sizes_beyond_its_scratch():
    lib = pkg.lib()
    out = torch.empty((64, 64, 32), dtype=torch.float32, device="cuda")
    too_many = torch.zeros((pkg.STATIC_MAX_EVENTS + 1, 3), dtype=torch.float64, device="cuda")
    g = pkg.make_grid(64, 64, 32)
    st = lib.stkde_compute_static(too_many.data_ptr(), too_many.shape[0], ctypes.byref(g), 4.0, 3.0,
                                  out.data_ptr(), pkg.FORM_TENSOR_BF16X3, 0, None, 1)
    assert st == pkg.ERR_UNSUPPORTED
    # a grid needing more bins than the scratch holds (2048 x 2048 x 512 voxels)
    big = pkg.make_grid(2048, 2048, 512)
    pts = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    st = lib.stkde_compute_static(pts.data_ptr(), 4, ctypes.byref(big), 4.0, 3.0, out.data_ptr(),
                                  pkg.FORM_TENSOR_BF16X3, 0, None, 1)
    assert st == pkg.ERR_UNSUPPORTED
    # host buffers are refused
    hout = np.empty((64, 64, 32), dtype=np.float32)
    st = lib.stkde_compute_static(pts.data_ptr(), 4, ctypes.byref(g), 4.0, 3.0, hout.ctypes.data,
                                  pkg.FORM_TENSOR_BF16X3, 0, None, 1)
    assert st == pkg.ERR_INVALID_ARGUMENT
