"""Recorded searches (CUDA graphs): a replay returns what the same search
returns when launched directly; the recording stays valid across inserts
and deletes that reuse ids and is made again after the index grows into a
new tile; the phases inside the graph are timed."""
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


def _data(n_docs=30000, nq=300):
    w = synth.scaled(synth.WORKLOADS["text"], n_docs + 6000, n=8000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=nq)
    return w, docs, qs


def _index(w, docs, rows):
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=2048)
    part = docs.slice(0, rows)
    ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    return ix


def _dev(qs):
    return (torch.from_numpy(qs.indptr.astype(np.int64)).cuda(),
            torch.from_numpy(qs.indices.astype(np.int32)).cuda(),
            torch.from_numpy(qs.values).cuda())


def _same(a, b):
    ia, sa = (x.cpu().numpy() for x in a)
    ib, sb = (x.cpu().numpy() for x in b)
    scale = np.maximum(np.abs(np.where(np.isfinite(sa), sa, 0)).max(axis=1, keepdims=True), 1e-30)
    fin = np.isfinite(sa)
    assert np.array_equal(fin, np.isfinite(sb))
    assert np.all(np.abs(np.where(fin, sa, 0).astype(np.float64) - np.where(fin, sb, 0))
                  <= REL * scale)
    diff = ia != ib
    assert np.all(np.abs(np.where(fin, sa, 0)[diff].astype(np.float64)
                         - np.where(fin, sb, 0)[diff]) <= REL * np.broadcast_to(scale, sa.shape)[diff])


def test_fixed_kprime_replay_matches_direct_search():
    w, docs, qs = _data()
    ix = _index(w, docs, 30000)
    q = _dev(qs)
    plan = sinnamon.Plan(ix, *q, k=10, k_prime_max=300, scratch_bytes=256 << 20)
    got = plan.run()
    _same(got, ix.search(*q, k=10, k_prime=300))
    got2 = tuple(x.clone() for x in plan.run())
    _same(got2, got)
    assert plan.recordings == 1


def test_per_query_kprime_and_learned_replays():
    w, docs, qs = _data()
    ix = _index(w, docs, 30000)
    q = _dev(qs)
    kp = torch.from_numpy(np.random.default_rng(2).integers(10, 700, qs.rows)
                          .astype(np.int32)).cuda()
    plan = sinnamon.Plan(ix, *q, k=10, k_prime_max=700, k_prime=kp, scratch_bytes=256 << 20)
    _same(plan.run(), ix.search(*q, k=10, k_prime=kp, k_prime_max=700))
    mlp = sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=11)
    mlp.set_normalizer(np.zeros(sinnamon.KP_FEATURES, np.float32),
                       np.full(sinnamon.KP_FEATURES, 4.0, np.float32))
    lp = sinnamon.Plan(ix, *q, k=10, k_prime_max=512, mlp=mlp, k_prime_min=10,
                       scratch_bytes=256 << 20)
    ids, sc = lp.run()
    e_ids, e_sc, e_kp = ix.search_learned(mlp, *q, 10, 10, 512)
    assert torch.equal(lp.out_kprime, e_kp)
    assert len(set(e_kp.cpu().numpy().tolist())) > 1
    _same((ids, sc), (e_ids, e_sc))


def test_replay_follows_inserts_deletes_and_growth():
    w, docs, qs = _data(n_docs=20000)
    ix = _index(w, docs, 20000)
    q = _dev(qs)
    rng = np.random.default_rng(4)
    # one churn step first: the append-only vector store doubles once
    first = rng.choice(20000, 300, replace=False).astype(np.int32)
    ix.delete(first)
    part = docs.slice(20000, 20300)
    ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    plan = sinnamon.Plan(ix, *q, k=10, k_prime_max=200, scratch_bytes=256 << 20)
    _same(plan.run(), ix.search(*q, k=10, k_prime=200))
    assert plan.recordings == 1
    # churn that reuses the freed ids: the recording stays valid
    dele = np.sort(rng.choice(20000, 300, replace=False)).astype(np.int32)
    ix.delete(dele)
    got = plan.run()
    assert not np.isin(got[0].cpu().numpy(), dele).any()
    _same(got, ix.search(*q, k=10, k_prime=200))
    part = docs.slice(0, 300)
    new = ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    assert np.array_equal(np.sort(new.cpu().numpy()), dele)
    _same(plan.run(), ix.search(*q, k=10, k_prime=200))
    assert plan.recordings == 1
    # new ids beyond the last tile in use: recorded again
    part = docs.slice(20300, 26000)
    ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    got = plan.run()
    assert plan.recordings >= 2
    _same(got, ix.search(*q, k=10, k_prime=200))
    assert (got[0].cpu().numpy() >= 20000).any()


def test_replay_sees_the_live_count():
    """k' above the live count: the replay takes the count at run time."""
    w, docs, qs = _data(n_docs=40, nq=5)
    ix = _index(w, docs, 40)
    q = _dev(qs)
    plan = sinnamon.Plan(ix, *q, k=10, k_prime_max=100, scratch_bytes=64 << 20)
    _same(plan.run(), ix.search(*q, k=10, k_prime=100))
    ix.delete(np.arange(0, 40, 2, dtype=np.int32))
    got = plan.run()
    assert plan.recordings == 1
    _same(got, ix.search(*q, k=10, k_prime=100))
    assert (got[0].cpu().numpy() % 2 == 1).all()


def test_phases_inside_the_graph_are_timed():
    w, docs, qs = _data(n_docs=20000, nq=100)
    ix = _index(w, docs, 20000)
    q = _dev(qs)
    plan = sinnamon.Plan(ix, *q, k=10, k_prime_max=200, scratch_bytes=256 << 20)
    plan.run()
    torch.cuda.synchronize()
    sinnamon.sinn_timing_start(ix.handle)
    for _ in range(3):
        plan.run()
    tm = sinnamon.sinn_timing_stop(ix.handle)
    assert tm["spans"]["score"] == 3 and tm["ms"]["score"] > 0
    assert tm["spans"]["rerank"] == 3 and tm["launches"] > 0
