"""Autotuner host logic (no GPU): cache keys, candidate filtering by the
accuracy target, the choice of the fastest configuration and the JSON table."""
import json

from paper_1705_09366_gb300 import autotune


def test_shape_key_rounds_events_and_bandwidths():
    a = autotune.shape_key("GB300", 1_000_000, (512, 512, 256), 10.04, 8.0)
    b = autotune.shape_key("GB300", 1_040_000, (512, 512, 256), 10.01, 8.04)
    assert a == b
    assert a != autotune.shape_key("GB300", 2_000_000, (512, 512, 256), 10.0, 8.0)
    assert a != autotune.shape_key("GB300", 1_000_000, (512, 512, 128), 10.0, 8.0)
    assert a != autotune.shape_key("other", 1_000_000, (512, 512, 256), 10.0, 8.0)
    assert "n2^0" in autotune.shape_key("GB300", 0, (8, 8, 8), 1.0, 1.0)


def test_candidates_meet_the_accuracy_target():
    c = autotune.candidates(2e-5)
    assert {f for f, _ in c} == {"bf16x3", "fp16x3", "tf32x3", "fp32"}
    assert {s for _, s in c} == set(autotune.SLABS)
    c = autotune.candidates(1e-5)
    assert "bf16x3" not in {f for f, _ in c}
    assert autotune.candidates(1e-6) == []
    assert {f for f, _ in autotune.candidates(2e-5, forms=("bf16x3",))} == {"bf16x3"}


def test_pick_and_table_round_trip(tmp_path):
    t = {("bf16x3", 0): 2.0, ("fp16x3", 8): 1.5, ("fp32", 0): 9.0}
    assert autotune.pick(t) == ("fp16x3", 8)
    path = str(tmp_path / "tune.json")
    tab = autotune.Table(path)
    assert tab.get("k") is None
    tab.put("k", ("fp16x3", 8), t)
    again = autotune.Table(path)
    assert again.get("k") == ("fp16x3", 8)
    with open(path) as f:
        d = json.load(f)
    assert d["k"]["ms"] == 1.5 and d["k"]["timings"]["bf16x3/0"] == 2.0
