"""Launch tuning: every tuning returns the same results (the launch
parameters change only the fp32 summation order and the batching), invalid
tunings are rejected, and the autotuner leaves a valid, faster-or-equal
configuration in place."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def setup():
    w = synth.scaled(synth.WORKLOADS["text"], 30000, n=8000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=400)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=2048)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    q = (qs.indptr.astype(np.int64), qs.indices.astype(np.int32), qs.values)
    yield ix, q
    ix.close()


def _same(a, b):
    (ia, sa), (ib, sb) = a, b
    scale = np.maximum(np.abs(sa).max(axis=1, keepdims=True), 1e-30)
    assert np.all(np.abs(sa.astype(np.float64) - sb) <= REL * scale)
    diff = ia != ib
    assert np.all(np.abs(sa[diff].astype(np.float64) - sb[diff]) <= REL * scale.repeat(
        ia.shape[1], axis=1)[diff])


def _run(ix, q, kp=300):
    ids, sc = ix.search(*q, k=10, k_prime=kp)
    return ids.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("fields", [
    dict(max_batch=7), dict(max_batch=33, bound_every=1), dict(bound_every=64),
    dict(emit_min_batch=1, max_batch=40), dict(emit_min_batch=65535),
    dict(rerank_blocks=1), dict(rerank_blocks=1024, dense_blocks_per_sm=1), dict(rerank_blocks=0),
    dict(dense_blocks_per_sm=32, emit_min_batch=500), dict(tiles_per_block=1),
    dict(tiles_per_block=3, bound_every=5), dict(tiles_per_block=64, bound_every=1),
    dict(persistent_blocks_per_sm=4), dict(persistent_blocks_per_sm=1, tiles_per_block=2,
                                           max_batch=50),
    dict(array_walk=1), dict(array_walk=1, persistent_blocks_per_sm=2, tiles_per_block=3),
    dict(array_walk=1, max_batch=20, emit_min_batch=64)])
def test_every_tuning_gives_the_same_results(setup, fields):
    ix, q = setup
    base = ix.tuning()
    want = _run(ix, q)
    try:
        ix.set_tuning(**fields)
        assert all(ix.tuning()[f] == v for f, v in fields.items())
        _same(want, _run(ix, q))
    finally:
        ix.set_tuning(**base)


@pytest.mark.parametrize("field,value", [("bound_every", 0), ("bound_every", 65),
                                          ("emit_min_batch", 0), ("rerank_blocks", 1025),
                                          ("dense_blocks_per_sm", 0),
                                          ("dense_blocks_per_sm", 33), ("tiles_per_block", 0),
                                          ("tiles_per_block", 65),
                                          ("persistent_blocks_per_sm", 5), ("array_walk", 2)])
def test_invalid_tuning_is_rejected(setup, field, value):
    ix, _ = setup
    before = ix.tuning()
    with pytest.raises(sinnamon.SinnError):
        ix.set_tuning(**{field: value})
    assert ix.tuning() == before


def test_autotune_picks_a_valid_tuning(setup):
    ix, q = setup
    want = _run(ix, q)
    t = ix.autotune(*q, k=10, k_prime=300, reps=1)
    assert t == ix.tuning()
    assert 1 <= t["bound_every"] <= 64 and 0 <= t["rerank_blocks"] <= 1024
    assert 1 <= t["dense_blocks_per_sm"] <= 32 and 1 <= t["emit_min_batch"] <= 65535
    assert 1 <= t["tiles_per_block"] <= 64
    _same(want, _run(ix, q))


def test_tile_size_is_chosen_by_measurement():
    from paper_2301_10622_gb300 import autotune
    w = synth.scaled(synth.WORKLOADS["text"], 12000, n=6000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=120)
    best, res = autotune.choose_tile_docs(w.n, w.m, w.h, docs, qs, k=10, k_prime=200,
                                          candidates=(1024, 2048), reps=2,
                                          scratch_bytes=256 << 20)
    assert set(res) == {1024, 2048} and best in res
    assert all(r["ms"] > 0 for r in res.values())
    assert res[best]["ms"] == min(r["ms"] for r in res.values())



def test_cached_autotune_measures_once_then_reuses(tmp_path):
    """autotune_cached on a new key measures and stores the tuning; on the
    same key it sets the stored tuning without measuring."""
    from paper_2301_10622_gb300 import autotune
    w = synth.scaled(synth.WORKLOADS["text"], 9000, n=6000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=200)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    path = str(tmp_path / "tunings.json")
    msgs = []
    t1 = autotune.autotune_cached(ix, qs, 10, 300, path, reps=1, log=msgs.append)
    assert "measured" in msgs[-1]
    ix.set_tuning(tiles_per_block=1, bound_every=1)
    t2 = autotune.autotune_cached(ix, qs, 10, 300, path, reps=1, log=msgs.append)
    assert "from cache" in msgs[-1] and t2 == t1
    assert {f: ix.tuning()[f] for f in t1} == t1
    ix.close()


@pytest.mark.parametrize("h,tile", [(2, 1024), (1, 2048), (3, 1024)])
def test_spread_array_walk_matches_the_oracle(h, tile):
    """array_walk = 1 (array postings spread over the block) on thin,
    mixed-sign lists with h sketch rows: the search equals the oracle's, as
    with per-term chunks."""
    from tests.test_gpu_parity import _check_search, _pair
    w = synth.scaled(synth.WORKLOADS["mixed"], 9000, n=20000, h=h)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=48)
    gpu, ora = _pair(w, docs, tile_docs=tile)
    gpu.set_tuning(array_walk=1)
    _check_search(gpu, ora, qs, 10, 300)
    gpu.set_tuning(array_walk=0)
    _check_search(gpu, ora, qs, 10, 300)
