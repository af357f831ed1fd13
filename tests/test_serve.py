"""Serving loop host logic (no GPU): the seeded request stream and the
admission rule of continuous batching."""
import numpy as np

from paper_1705_09366_gb300 import serve


def test_request_stream_is_seeded_poisson_over_the_stated_choices():
    a = serve.request_stream(4000, 200.0, 4, seed=3)
    b = serve.request_stream(4000, 200.0, 4, seed=3)
    assert a == b
    t = np.array([r.arrival for r in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0          # exponential mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.06           # coefficient of variation 1
    assert {r.gx for r in a} == {128, 256, 512} and all(r.gx == r.gy for r in a)
    assert {r.gt for r in a} == {128, 256}
    assert {r.hs_vox for r in a} == {5.0, 10.0, 20.0} and {r.ht_vox for r in a} == {4.0, 8.0, 16.0}
    assert {r.set_id for r in a} == {0, 1, 2, 3}
    for r in a[:50]:
        assert r.gx * r.sres == 512.0 and r.gt * r.tres == 256.0
        assert r.hs == r.hs_vox * r.sres and r.out_bytes == 4 * r.gx * r.gy * r.gt


def _req(i, g, arrival=0.0):
    return serve.Request(i, 0, g, g, g, 1.0, 1.0, 5.0, 4.0, arrival)


def test_form_batch_admits_in_order_within_budget():
    q = [_req(i, 64) for i in range(10)]                       # 1 MiB outputs
    per = q[0].out_bytes + 100
    b = serve.form_batch(q, budget_bytes=4 * per, set_bytes=lambda s: 100)
    assert [r.rid for r in b] == [0, 1, 2, 3]
    b = serve.form_batch(q, budget_bytes=4 * per - 1, set_bytes=lambda s: 100)
    assert [r.rid for r in b] == [0, 1, 2]
    b = serve.form_batch(q, budget_bytes=100 * per, set_bytes=lambda s: 100, max_batch=6)
    assert len(b) == 6
    # an oversized request is served alone, never starved
    big = [_req(0, 512), _req(1, 64)]
    b = serve.form_batch(big, budget_bytes=1 << 20, set_bytes=lambda s: 0)
    assert [r.rid for r in b] == [0]
    # admission stops at the first request that does not fit (arrival order kept)
    mixed = [_req(0, 64), _req(1, 512), _req(2, 64)]
    b = serve.form_batch(mixed, budget_bytes=3 << 20, set_bytes=lambda s: 0)
    assert [r.rid for r in b] == [0]


def test_percentiles():
    p = serve.percentiles([0.001 * k for k in range(1, 101)])
    assert abs(p["p50_ms"] - 50.5) < 1e-9 and abs(p["p99_ms"] - 99.01) < 1e-9 and p["max_ms"] == 100.0


def test_form_batch_without_force_waits_for_room():
    # with batches already running, an oversized first request waits
    big = [_req(0, 512), _req(1, 64)]
    assert serve.form_batch(big, budget_bytes=1 << 20, set_bytes=lambda s: 0, force_first=False) == []
    assert [r.rid for r in serve.form_batch(big, budget_bytes=1 << 30, set_bytes=lambda s: 0,
                                            force_first=False)] == [0, 1]


def test_expire_drops_cancelled_and_late_requests_in_place():
    q = [serve.Request(0, 0, 8, 8, 8, 1.0, 1.0, 5.0, 4.0, 0.0, deadline=0.5),
         serve.Request(1, 0, 8, 8, 8, 1.0, 1.0, 5.0, 4.0, 0.2),
         serve.Request(2, 0, 8, 8, 8, 1.0, 1.0, 5.0, 4.0, 0.3, deadline=0.5),
         serve.Request(3, 0, 8, 8, 8, 1.0, 1.0, 5.0, 4.0, 0.4)]
    gone = serve.expire(q, now=0.6, cancelled={3})
    assert [r.rid for r in gone] == [0, 3]          # 0 is late (0.6 > 0.0 + 0.5); 3 cancelled
    assert [r.rid for r in q] == [1, 2]             # 2 is not late yet (0.6 <= 0.8), order kept
    assert serve.expire(q, now=0.81, cancelled=set())[0].rid == 2 and [r.rid for r in q] == [1]


def test_overlap_of_intervals():
    assert serve.overlap([]) == {"max_concurrent": 0, "overlap_time": 0.0}
    assert serve.overlap([(0.0, 1.0), (2.0, 3.0)]) == {"max_concurrent": 1, "overlap_time": 0.0}
    o = serve.overlap([(0.0, 2.0), (1.0, 3.0), (1.5, 1.75)])
    assert o["max_concurrent"] == 3 and abs(o["overlap_time"] - 1.0) < 1e-12
    # touching intervals do not overlap
    assert serve.overlap([(0.0, 1.0), (1.0, 2.0)])["max_concurrent"] == 1
