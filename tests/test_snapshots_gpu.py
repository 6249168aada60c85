"""Sequence-numbered mutations (Sec. 4.3 deletes and Alg. 5 inserts that
overlap searches): a search at snapshot s returns what the oracle returns on
exactly the vectors inserted at numbers <= s and not deleted at numbers <= s,
while later mutations are applied -- also while that search runs on another
stream.  Deleted ids keep scoring for older snapshots until sinn_reclaim,
and only then are they reused (ascending); a tile whose other copy an older
search may still read refuses a rebuild (SINN_EBUSY) and nothing changes.

The oracle for snapshot s is a fresh oracle index holding the visible
vectors in ascending id order (oracle id r = r-th visible id): Alg. 6 scores
and exact scores are per-vector, so the two id spaces differ by that map
only.  Bar as in the parity tests: ids equal except inside the fp32 tie
band (2e-5 of the score's magnitude) at the k-th score, scores within 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402

SEED = 0x5151


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


class Book:
    """Host record of every id's vector and (born, died) numbers."""

    def __init__(self):
        self.rows, self.born, self.died = {}, {}, {}

    def insert(self, ids, part, seq):
        for r, i in enumerate(ids):
            i = int(i)
            self.rows[i] = part.row(r)
            self.born[i], self.died[i] = seq, None

    def delete(self, ids, seq):
        for i in ids:
            assert self.died[int(i)] is None
            self.died[int(i)] = seq

    def visible(self, s):
        return np.array(sorted(i for i in self.rows if self.born[i] <= s and
                               (self.died[i] is None or self.died[i] > s)), np.int64)

    def oracle(self, w, s):
        vis = self.visible(s)
        ora = oracle.OracleIndex(w.n, w.m, w.h, seed=SEED)
        if vis.size:
            ip = np.zeros(vis.size + 1, np.uint64)
            ip[1:] = np.cumsum([self.rows[int(i)][0].size for i in vis])
            idx = np.concatenate([self.rows[int(i)][0] for i in vis]).astype(np.uint32)
            val = np.concatenate([self.rows[int(i)][1] for i in vis]).astype(np.float32)
            assert np.array_equal(ora.insert(ip, idx, val), np.arange(vis.size, dtype=np.uint32))
        return ora, vis


def _dev_csr(qs, dev):
    return (torch.from_numpy(qs.indptr.astype(np.int64)).to(dev),
            torch.from_numpy(qs.indices.astype(np.int32)).to(dev),
            torch.from_numpy(qs.values.astype(np.float32)).to(dev))


def _ctx_search(ctx, dq, k, kp, stream=None):
    n = dq[0].numel() - 1
    ids = torch.empty((n, k), dtype=torch.int32, device=dq[0].device)
    sc = torch.empty((n, k), dtype=torch.float32, device=dq[0].device)
    ctx.search(dq[0], dq[1], dq[2], k, kp, ids, sc, stream=stream)
    return ids, sc


def _check(ids, sc, book, w, s, qs, k, kp):
    """GPU top-k at snapshot s against the oracle on that snapshot's vectors."""
    ids = ids.cpu().numpy().astype(np.int64)
    sc = sc.cpu().numpy()
    ora, vis = book.oracle(w, s)
    inv = {int(g): r for r, g in enumerate(vis)}
    ref = ora.search(qs.indptr, qs.indices, qs.values, k=k, k_prime=kp, candidates=True)
    for q in range(qs.rows):
        qi, qv = qs.row(q)
        exact, emag = ora.exact_scores(qi, qv, with_magnitude=True)
        r_ = min(k, vis.size)
        got = [inv.get(int(g), -1) for g in ids[q][:r_]]
        assert min(got, default=0) >= 0, (q, "an id not visible at the snapshot")
        assert all(i < 0 for i in ids[q][r_:])
        for o, v in zip(got, sc[q][:r_]):
            assert abs(float(v) - exact[o]) <= 1e-5 * max(emag[o], 1e-30)
        want = [int(x) for x in ref["ids"][q][:r_]]
        if got != want:
            tau = ref["scores"][q][r_ - 1]
            for o in set(got) ^ set(want):
                assert abs(exact[o] - tau) <= 2e-5 * max(emag[o], 1e-30) or \
                    o not in set(int(x) for x in ref["cand_ids"][q]), (q, o)


def _setup(n0=5000, pool=4000, nq=24, n=3000):
    w = synth.scaled(synth.WORKLOADS["mixed"], n0, n=n)
    docs = synth.make_docs(w)
    extra = synth.make_docs(w, n_docs=pool, seed=91)
    qs = synth.make_queries(w, n_q=nq, seed=92)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024, seed=SEED)
    book = Book()
    ids = ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32),
                    docs.values).cpu().numpy()
    book.insert(ids, docs, 0)
    return w, ix, book, extra, qs


def _insert_at(ix, book, part, seq):
    ids = ix.insert_at(part.indptr.astype(np.int64), part.indices.astype(np.int32),
                       part.values, seq).cpu().numpy().astype(np.int64)
    book.insert(ids, part, seq)
    return ids


def _delete_at(ix, book, ids, seq):
    ix.delete_at(np.asarray(ids, np.int32), seq)
    book.delete(ids, seq)


@pytest.mark.parametrize("walk", [0, 1])
def test_snapshots_see_their_epoch_and_reclaim_reuses_ids(walk):
    w, ix, book, extra, qs = _setup()
    ix.set_tuning(array_walk=walk, emit_min_batch=1)  # batched scorers, either walk
    rng = np.random.default_rng(3)
    k, kp = 10, 150
    ctx = sinnamon.Context(ix, 64 << 20)
    dq = _dev_csr(qs, ix.device)

    # epoch 1: deletes stay scorable for snapshot 0; inserts take fresh ids
    d1 = rng.choice(book.visible(0), 300, replace=False)
    _delete_at(ix, book, d1, 1)
    new1 = _insert_at(ix, book, extra.slice(0, 800), 1)
    assert list(new1) == list(range(5000, 5800))    # nothing reclaimed: no reuse
    st = ix.stats()
    assert st["pending_deletes"] == 300 and st["live"] == 5500
    for s in (0, 1):
        ctx.set_snapshot(s)
        _check(*_ctx_search(ctx, dq, k, kp), book, w, s, qs, k, kp)
    _check(*ix.search(qs.indptr.astype(np.int64), qs.indices.astype(np.int32), qs.values,
                      k=k, k_prime=kp), book, w, 1, qs, k, kp)   # no snapshot: the latest

    # epoch 2: reclaim what only snapshot 0 counted, then reuse it ascending
    ix.reclaim(1)
    assert ix.stats()["pending_deletes"] == 0
    d2 = rng.choice(book.visible(1), 200, replace=False)
    _delete_at(ix, book, d2, 2)
    new2 = _insert_at(ix, book, extra.slice(800, 1500), 2)
    assert list(new2[:300]) == sorted(int(i) for i in d1)
    assert list(new2[300:]) == list(range(5800, 6200))
    for s in (1, 2):
        ctx.set_snapshot(s)
        _check(*_ctx_search(ctx, dq, k, kp), book, w, s, qs, k, kp)
    ctx.set_snapshot(sinnamon.SINN_SEQ_LATEST)
    _check(*_ctx_search(ctx, dq, k, kp), book, w, 2, qs, k, kp)

    # epoch 3: the fresh-id tile was rebuilt at 2 and snapshot 1 may still
    # read its other copy: refused, nothing changes; after reclaim(2) it goes
    before = ix.stats()
    lists = [ix.inverted_list(j) for j in range(0, w.n, 97)]
    part = extra.slice(1500, 1700)
    with pytest.raises(sinnamon.SinnError) as e:
        ix.insert_at(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values, 3)
    assert e.value.code == sinnamon.SINN_EBUSY
    assert ix.stats() == before
    assert all(np.array_equal(a, ix.inverted_list(j)) for a, j in zip(lists, range(0, w.n, 97)))
    ix.reclaim(2)
    new3 = _insert_at(ix, book, part, 3)
    assert list(new3) == sorted(int(i) for i in d2)
    for s in (2, 3):
        ctx.set_snapshot(s)
        _check(*_ctx_search(ctx, dq, k, kp), book, w, s, qs, k, kp)
    assert ix.stats()["live"] == book.visible(3).size


def test_a_running_search_keeps_its_snapshot():
    """A large batch at snapshot 1 runs on its own stream while epoch 2
    (reclaim, deletes, inserts that rebuild tiles) is applied on another;
    its results are snapshot 1's whatever the overlap was."""
    w, ix, book, extra, _ = _setup(n0=20000, pool=6000, nq=1)
    qs = synth.make_queries(w, n_q=3000, seed=93)
    rng = np.random.default_rng(4)
    k, kp = 10, 100
    d1 = rng.choice(book.visible(0), 1500, replace=False)
    _delete_at(ix, book, d1, 1)
    _insert_at(ix, book, extra.slice(0, 3000), 1)
    ctx = sinnamon.Context(ix, 512 << 20)
    ctx.set_snapshot(1)
    dq = _dev_csr(qs, ix.device)
    side = torch.cuda.Stream(device=ix.device)
    torch.cuda.synchronize(ix.device)
    ids, sc = _ctx_search(ctx, dq, k, kp, stream=side)   # asynchronous on `side`
    ix.reclaim(1)                                        # no search older than 1 runs
    d2 = rng.choice(book.visible(1), 2000, replace=False)
    _delete_at(ix, book, d2, 2)
    new2 = _insert_at(ix, book, extra.slice(3000, 6000), 2)
    assert sorted(int(i) for i in d1) == list(new2[:1500])   # reused while the search ran
    side.synchronize()
    pick = np.sort(rng.choice(qs.rows, 40, replace=False))
    sub = qs.take(pick)
    tp = torch.from_numpy(pick).to(ids.device)
    _check(ids[tp], sc[tp], book, w, 1, sub, k, kp)
    # the same queries afterwards at snapshot 2 and at snapshot 1 again
    ctx2 = sinnamon.Context(ix, 64 << 20)
    dsub = _dev_csr(sub, ix.device)
    for s in (1, 2):
        ctx2.set_snapshot(s)
        _check(*_ctx_search(ctx2, dsub, k, kp), book, w, s, sub, k, kp)


def test_sequence_arguments_are_checked():
    w, ix, book, extra, qs = _setup(n0=2000, pool=100, nq=2)
    part = extra.slice(0, 10)
    before = ix.stats()
    with pytest.raises(sinnamon.SinnError) as e:
        ix.insert_at(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values,
                     sinnamon.SINN_SEQ_LATEST + 1)
    assert e.value.code == sinnamon.SINN_EINVAL
    with pytest.raises(sinnamon.SinnError) as e:
        ix.delete_at(np.array([5, 5], np.int32), 1)        # a repeat
    assert e.value.code == sinnamon.SINN_EINVAL
    _delete_at(ix, book, [7], 1)
    with pytest.raises(sinnamon.SinnError) as e:
        ix.delete_at(np.array([7], np.int32), 2)           # already deleted
    assert e.value.code == sinnamon.SINN_ENOTFOUND
    assert ix.stats()["live"] == before["live"] - 1 and ix.stats()["pending_deletes"] == 1
    # a pending delete is not reusable, even by the stream-ordered insert
    got = ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32),
                    part.values).cpu().numpy()
    assert 7 not in set(got.tolist()) and list(got) == list(range(2000, 2010))
    book.insert(got, part, 0)
    ix.reclaim(sinnamon.SINN_SEQ_LATEST + 1)               # every search done
    assert ix.stats()["pending_deletes"] == 0
    ctx = sinnamon.Context(ix, 32 << 20)
    for s in (1, sinnamon.SINN_SEQ_LATEST):
        ctx.set_snapshot(s)
        _check(*_ctx_search(ctx, _dev_csr(qs, ix.device), 5, 50), book, w, 1, qs, 5, 50)


def test_reserve_makes_room_ahead():
    """sinn_reserve grows the id capacity and the vector store once; inserts
    within the reserved sizes then allocate neither, and the index holds and
    returns the same as without the reservation."""
    w, ix, book, extra, qs = _setup(n0=3000, pool=2000, nq=8)
    before = ix.stats()
    ix.reserve(2000, int(extra.nnz))
    st = ix.stats()
    assert st["capacity"] >= before["next_id"] + 2000 and st["bytes_store"] > before["bytes_store"]
    assert st["live"] == before["live"] and st["postings"] == before["postings"]
    ix.reserve(10, 10)                                 # already there: no change
    assert ix.stats() == st
    new = _insert_at(ix, book, extra.slice(0, 2000), 1)
    after = ix.stats()
    assert after["capacity"] == st["capacity"] and after["bytes_store"] == st["bytes_store"]
    assert list(new) == list(range(3000, 5000))
    ctx = sinnamon.Context(ix, 32 << 20)
    for s in (0, 1):
        ctx.set_snapshot(s)
        _check(*_ctx_search(ctx, _dev_csr(qs, ix.device), 10, 100), book, w, s, qs, 10, 100)
