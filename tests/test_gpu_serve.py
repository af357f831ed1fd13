"""GPU: the serving loop over resident event sets.

- Every request is served; each kept output equals the same request computed
  alone (bit for bit: a mix changes latency, never values) and the oracle on
  sampled tiles (parity tolerance and the binary32 tie slack); the admitted
  bytes stay within the budget.
- Continuous batching: a batch admitted while another runs goes to a second
  slot (its own context and stream) and the two are resident on the device at
  once (CUDA event timestamps of both intervals overlap).
- Host-side cancellation and deadlines: a cancelled request and one whose
  deadline passes while the slots are busy are dropped unserved.
"""
import numpy as np
import pytest

import oracle
import parity_util as pu
from paper_1705_09366_gb300 import serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DOMAIN = (512.0, 512.0, 256.0)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


@pytest.fixture(scope="module")
def sets():
    return synth.resident_sets(sizes=(20_000, 60_000, 150_000))


def _req(rid, set_id, g, gt, hs, ht, arrival, deadline=None):
    return serve.Request(rid, set_id, g, g, gt, DOMAIN[0] / g, DOMAIN[2] / gt, hs, ht, arrival,
                         deadline)


def _check_against_oracle(r, out, points, seed):
    p = oracle.params(r.gx, r.gy, r.gt, r.hs, r.ht, sres=r.sres, tres=r.tres)
    vox = points / np.array([r.sres, r.sres, r.tres])
    boxes = pu.sample_tile_boxes(vox, r.gx, r.gy, r.gt, n_random=8, seed=seed)
    refs = oracle.pb_boxes(points, p, boxes)
    scale = max(float(ref.max()) for ref, _ in refs)
    worst = 0.0
    for (x0, x1, y0, y1, t0, t1), (ref, slack) in zip(boxes, refs):
        got = out[x0:x1, y0:y1, t0:t1].cpu().numpy()
        worst = max(worst, pu.excess_error(got, ref, slack, scale=scale))
    assert worst <= pu.TOL["bf16x3"], (r, worst)


def test_serving_stream_alone_equals_mix_and_the_oracle(sets):
    budget = 3 << 30
    srv = serve.Server(sets, budget_bytes=budget)
    try:
        reqs = serve.request_stream(48, 400.0, len(sets), seed=11)
        stats, lat, batches, kept = srv.run(reqs, keep_outputs=lambda r: r.rid % 8 == 0)
        assert stats["requests"] == len(reqs) and sorted(lat) == [r.rid for r in reqs]
        assert not stats["dropped"]
        assert all(v > 0 for v in lat.values())
        assert np.isfinite(stats["p50_ms"]) and stats["p99_ms"] >= stats["p50_ms"]
        assert stats["max_admitted_bytes"] <= budget
        assert sorted(sum(batches, [])) == [r.rid for r in reqs]
        by_id = {r.rid: r for r in reqs}
        assert len(kept) == 6
        for rid, out in kept.items():
            r = by_id[rid]
            alone = srv.compute_alone(r)
            assert torch.equal(out, alone), rid
            _check_against_oracle(r, out, sets[r.set_id], seed=rid)
    finally:
        srv.close()


def test_a_second_batch_runs_beside_the_first(sets):
    srv = serve.Server(sets, budget_bytes=3 << 30, slots=2)
    try:
        srv.run([_req(0, 0, 128, 128, 5.0, 4.0, 0.0)])  # warm-up
        # three heavy requests arrive together (one batch, several ms of device
        # work), a light one 0.1 ms later: it cannot join the running batch
        reqs = [_req(i, 2, 512, 256, 20.0, 16.0, 0.0) for i in range(3)]
        reqs.append(_req(3, 0, 128, 128, 5.0, 4.0, 1e-4))
        stats, lat, batches, kept = srv.run(reqs, keep_outputs=lambda r: r.rid == 3)
        assert sorted(lat) == [0, 1, 2, 3]
        assert [0, 1, 2] in batches and [3] in batches
        assert stats["max_concurrent_batches"] >= 2, stats
        assert stats["overlap_s"] > 0.0, stats
        assert torch.equal(kept[3], srv.compute_alone(reqs[3]))
    finally:
        srv.close()


def test_cancelled_and_expired_requests_are_dropped(sets):
    srv = serve.Server(sets, budget_bytes=3 << 30, slots=1)
    try:
        srv.run([_req(0, 0, 128, 128, 5.0, 4.0, 0.0)])  # warm-up
        reqs = [_req(i, 2, 512, 256, 20.0, 16.0, 0.0) for i in range(3)]  # holds the only slot
        reqs.append(_req(3, 0, 128, 128, 5.0, 4.0, 1e-4, deadline=1e-3))  # expires while queued
        reqs.append(_req(4, 0, 128, 128, 5.0, 4.0, 2e-4))                  # cancelled on arrival of 3
        reqs.append(_req(5, 0, 128, 128, 5.0, 4.0, 3e-4, deadline=10.0))  # served

        def on_arrival(s, r):
            if r.rid == 3:
                s.cancel(4)

        stats, lat, batches, _ = srv.run(reqs, on_arrival=on_arrival)
        assert stats["dropped"] == [3, 4], stats
        assert sorted(lat) == [0, 1, 2, 5]
        assert all(3 not in b and 4 not in b for b in batches)
    finally:
        srv.close()


def test_admission_follows_free_device_memory(sets):
    """Device memory that batches in flight use up (600 MB above the reserve in
    all, as cudaMemGetInfo would report it without a caching allocator): the
    bytes in flight never exceed 600 MB, whatever the cap; every request is
    still served, several batches at a time."""
    srv = serve.Server(sets, budget_bytes=8 << 30, slots=3, reserve_bytes=1 << 30)
    try:
        srv.run([_req(0, 0, 128, 128, 5.0, 4.0, 0.0)])  # warm-up
        srv.free_bytes = lambda: srv.reserve + (600 << 20) - srv.inflight_bytes
        reqs = [_req(i, i % 3, 256, 256, 10.0, 8.0, 0.0) for i in range(12)]  # a burst
        stats, lat, batches, _ = srv.run(reqs)
        assert sorted(lat) == list(range(12))
        assert 0 < stats["max_admitted_bytes"] <= 600 << 20, stats["max_admitted_bytes"]
        assert len(batches) > 1
    finally:
        srv.close()
