"""GPU: the autotuner times every candidate on the caller's problem once per
shape, caches the winner, and its result is bit-identical to a direct call
with the chosen form and slab."""
import pytest

import paper_1705_09366_gb300 as pkg
from paper_1705_09366_gb300 import autotune, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.lib()
    yield


def test_tuned_result_equals_direct_call_and_is_cached(tmp_path):
    w = synth.small()
    pts = torch.from_numpy(w.points).cuda()
    dims = (w.gx, w.gy, w.gt)
    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(cache=path, reps=2)
    try:
        out = t.compute(pts, dims, w.hs, w.ht)
        t.synchronize()
        key = autotune.shape_key(t.name, w.n, dims, w.hs, w.ht)
        entry = t.table.entries[key]
        assert len(entry["timings"]) == len(autotune.candidates(2e-5))
        cfg = (entry["form"], entry["slab"])
        with pkg.Context(form=cfg[0], slab=cfg[1]) as c:
            ref = c.compute(pts, dims, w.hs, w.ht)
            c.synchronize()
        assert torch.equal(out, ref)
    finally:
        t.close()
    # a new tuner reads the table and times nothing
    t2 = autotune.Tuner(cache=path, reps=2)
    try:
        def no_timing(*a, **k):
            raise AssertionError("cached shape was timed again")
        t2._time = no_timing
        again = t2.compute(pts, dims, w.hs, w.ht)
        t2.synchronize()
        assert torch.equal(again, ref)
    finally:
        t2.close()
