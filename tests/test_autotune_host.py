"""Host logic of the launch-parameter tuning cache (no GPU)."""
import json

import pytest

pytest.importorskip("torch")

from paper_2301_10622_gb300 import autotune  # noqa: E402


def test_tuning_cache_keys_reads_and_writes(tmp_path):
    """Host logic of the tuning cache (no GPU): a miss runs the tuner once and
    stores its choice; a hit returns it without tuning; keys separate GPUs,
    shapes, flags and sizes (rounded to a power of two)."""
    path = str(tmp_path / "tunings.json")
    calls = []

    def tune(v):
        def f():
            calls.append(v)
            return {"tiles_per_block": v, "bound_every": 4}
        return f

    k1 = autotune.tuning_key("GB300", 30522, 128, 1, 4096, 1_000_000, 10, 1000)
    t, hit = autotune.cached_tuning(path, k1, tune(2))
    assert (t["tiles_per_block"], hit, calls) == (2, False, [2])
    t, hit = autotune.cached_tuning(path, k1, tune(8))
    assert (t["tiles_per_block"], hit, calls) == (2, True, [2])
    assert autotune.tuning_key("GB300", 30522, 128, 1, 4096, 900_000, 10, 1000) == k1
    others = [autotune.tuning_key("B200", 30522, 128, 1, 4096, 1_000_000, 10, 1000),
              autotune.tuning_key("GB300", 30522, 128, 2, 4096, 1_000_000, 10, 1000),
              autotune.tuning_key("GB300", 30522, 128, 1, 2048, 1_000_000, 10, 1000),
              autotune.tuning_key("GB300", 30522, 128, 1, 4096, 1_000_000, 10, 1000, flags=2),
              autotune.tuning_key("GB300", 30522, 128, 1, 4096, 3_000_000, 10, 1000),
              autotune.tuning_key("GB300", 30522, 128, 1, 4096, 1_000_000, 10, 2000)]
    assert len(set(others + [k1])) == len(others) + 1
    t, hit = autotune.cached_tuning(path, others[0], tune(4))
    assert (t["tiles_per_block"], hit) == (4, False)
    with open(path) as f:
        assert set(json.load(f)) == {k1, others[0]}
