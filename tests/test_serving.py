"""The continuous-batching serving loop: each query's result in the mix (a
batch in one of several overlapping search contexts, at its snapshot, while
later epochs of inserts and deletes are applied) is the same as the same
query run alone, with no snapshot, on an index that replays the loop's
calls up to exactly the epochs its snapshot counts.

Both sides are the CUDA path; alone the query is a batch of one, in the mix
one of a larger batch, so the scoring kernels sum in other orders.  Re-ranked
scores are exact inner products computed the same way on both sides, so the
top-k must agree rank by rank within the fp32 bar (1e-5 of the score),
except where fp32 rounding moved an id across the k'-th approximate score:
then every id in which the two differ must sit inside that tie band of the
boundary (scores here are sums of positive terms, so the band is relative to
the score itself)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_10622_gb300 import serving, sinnamon, synth  # noqa: E402

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _setup(n0=20000, pool=6000, nq=300):
    w = synth.scaled(synth.WORKLOADS["text"], n0 + pool, n=8000)
    docs = synth.make_docs(w)
    qs = synth.make_queries(w, n_q=nq)
    start = docs.slice(0, n0)
    extra = docs.slice(n0, n0 + pool)

    def fresh():
        ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=2048)
        ids = ix.insert(start.indptr.astype(np.int64), start.indices.astype(np.int32),
                        start.values).cpu().numpy()
        return ix, ids
    return w, qs, extra, fresh


def _stream(qs, extra, seconds=1.2, burst=300):
    reqs = serving.poisson_stream(seconds, {"insert": 2000.0, "delete": 300.0, "query": 1200.0},
                                  extra.rows, qs.rows, seed=4000)
    # a burst at the start: more queries than one slot takes, so slots overlap
    rng = np.random.default_rng(7)
    reqs = [serving.Request(0.0, "query", int(r)) for r in rng.integers(0, qs.rows, burst)] + reqs
    reqs.sort(key=lambda r: r.t)
    return reqs


def _compare(results, alone, approx, k):
    boundary_moves = 0
    for q, (ids_m, sc_m, kp_m) in results.items():
        ids_a, sc_a, kp_a = alone[q]
        assert kp_m == kp_a, (q, kp_m, kp_a)
        scale = max(float(np.abs(sc_a).max()), 1e-30)
        same_ranks = np.all(np.abs(sc_m.astype(np.float64) - sc_a) <= REL * scale)
        if same_ranks:
            # ids may differ only by swaps of equal exact scores
            for r in range(k):
                if ids_m[r] != ids_a[r]:
                    assert abs(float(sc_m[r]) - float(sc_a[r])) <= REL * scale
            continue
        boundary_moves += 1
        s = approx[q]
        live = np.isfinite(s)
        kq = min(kp_a, int(live.sum()))
        tau = np.sort(s[live])[::-1][kq - 1]
        for d in set(ids_m.tolist()) ^ set(ids_a.tolist()):
            if d < 0:
                continue
            assert abs(float(s[d]) - tau) <= 2 * REL * max(abs(float(s[d])), abs(tau)), (
                q, d, float(s[d]), tau)
    return boundary_moves


@pytest.mark.parametrize("learned", [False, True])
def test_same_alone_and_in_the_mix(learned):
    w, qs, extra, fresh = _setup()
    k, kp = 10, 200
    mlp = None
    if learned:
        mlp = sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=11)
        mlp.set_normalizer(np.zeros(sinnamon.KP_FEATURES, np.float32),
                           np.full(sinnamon.KP_FEATURES, 4.0, np.float32))
    ix, live = fresh()
    srv = serving.Server(ix, qs, extra, live, slots=3, slot_bytes=96 << 20, max_batch=64,
                         k=k, k_prime=kp, mlp=mlp, kp_max=512, mutation_delay=0.004)
    reqs = _stream(qs, extra)
    stats, results, log = srv.serve(reqs)
    n_q = sum(r.kind == "query" for r in reqs)
    assert stats["queries"] == n_q == len(results)
    assert stats["max_inflight"] >= 2, stats          # searches overlapped
    assert stats["mean_batch"] > 1.0, stats           # batches formed
    assert any(e[0] == "insert" for e in log) and any(e[0] == "delete" for e in log)
    assert stats["epochs_overlapped"] >= 1, stats     # an epoch ran beside searches
    assert any(e[0] == "reclaim" for e in log)
    k_primes = None
    if learned:
        assert len({v[2] for v in results.values()}) > 1  # k' varies per query
        # the network reads list lengths (tombstones included) as they stand
        # when the search runs, which later epochs may already have changed:
        # the alone run takes the k' the mix chose
        k_primes = {q: v[2] for q, v in results.items()}
        assert all(k <= v <= 512 for v in k_primes.values())

    ix2, live2 = fresh()
    assert np.array_equal(live, live2)
    alone, approx = serving.replay(ix2, qs, extra, log, k, kp, approx=True, k_primes=k_primes)
    assert set(alone) == set(results)
    moves = _compare(results, alone, approx, k)
    assert moves <= max(2, 0.02 * n_q), moves
    st1, st2 = ix.stats(), ix2.stats()
    st1.pop("bytes_scratch"), st2.pop("bytes_scratch")  # the replay searched via the index's own
    assert st1 == st2


def test_mutations_follow_arrival_order():
    """Snapshots follow arrival: a query counts only epochs whose requests
    all arrived no later than it, and never a later epoch than the last one
    logged before its launch; epochs are numbered 1, 2, ... in log order;
    reclaim horizons only grow and no query launched after a reclaim is
    older than its horizon; the log keeps every request exactly once."""
    w, qs, extra, fresh = _setup(n0=5000, pool=2000, nq=50)
    ix, live = fresh()
    srv = serving.Server(ix, qs, extra, live, slots=2, slot_bytes=32 << 20, max_batch=16,
                         k=10, k_prime=100, mutation_delay=0.002)
    reqs = serving.poisson_stream(0.5, {"insert": 1000.0, "delete": 400.0, "query": 800.0},
                                  extra.rows, qs.rows, seed=4001)
    stats, results, log = srv.serve(reqs)
    seen = [i for e in log for i in e[1]]
    assert sorted(seen) == list(range(len(reqs)))
    epoch_reqs, last_epoch, horizon = {}, 0, 0
    for kind, ri, rows, ids, seq in log:
        if kind in ("insert", "delete"):
            assert seq in (last_epoch, last_epoch + 1)
            last_epoch = seq
            epoch_reqs.setdefault(seq, []).extend(ri)
        elif kind == "reclaim":
            assert seq > horizon
            horizon = seq
        else:
            assert horizon <= seq <= last_epoch
            t = max(reqs[q].t for q in ri)
            for e in range(1, seq + 1):
                assert all(reqs[j].t <= t for j in epoch_reqs[e])
    assert last_epoch == stats["epochs"] >= 2
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert ix.stats()["live"] == len(srv.live)
