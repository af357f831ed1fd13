"""GPU: the serving loop over resident event sets.  Every request must be served,
each kept output must equal the same request computed alone (bit for bit: a mix
changes latency, never values), and the admitted bytes stay within the budget."""
import numpy as np
import pytest

from paper_1705_09366_gb300 import serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_serving_stream_alone_equals_mix():
    sets = synth.resident_sets(sizes=(20_000, 60_000, 150_000))
    budget = 3 << 30
    srv = serve.Server(sets, budget_bytes=budget)
    try:
        reqs = serve.request_stream(48, 400.0, len(sets), seed=11)
        stats, lat, batches, kept = srv.run(reqs, keep_outputs=lambda r: r.rid % 8 == 0)
        assert stats["requests"] == len(reqs) and sorted(lat) == [r.rid for r in reqs]
        assert all(v > 0 for v in lat.values())
        assert np.isfinite(stats["p50_ms"]) and stats["p99_ms"] >= stats["p50_ms"]
        assert stats["max_admitted_bytes"] <= budget
        assert sorted(sum(batches, [])) == [r.rid for r in reqs]
        by_id = {r.rid: r for r in reqs}
        for rid, out in kept.items():
            alone = srv.compute_alone(by_id[rid])
            assert torch.equal(out, alone), rid
    finally:
        srv.close()
