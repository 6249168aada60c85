"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: bit-exact for ids, hash tables, sketch bins and inverted-list contents;
fp32 approximate and re-ranked scores within 1e-5 * magnitude of fp64;
candidate sets and top-k ids equal except inside that tie band.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402
from tests import parity  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _ip(c):
    return c.indptr.astype(np.int64)


def _ix(c):
    return c.indices.astype(np.int32)


def _pair(w, docs, tile_docs=1024, table=None, seed=0x5151, **cfg):
    gpu = sinnamon.Index(w.n, w.m, w.h, tile_docs=tile_docs, seed=seed, table=table, **cfg)
    ora = oracle.OracleIndex(w.n, w.m, w.h, seed=seed, table=table)
    if docs is not None and docs.rows:
        g = gpu.insert(_ip(docs), _ix(docs), docs.values).cpu().numpy().astype(np.uint32)
        o = ora.insert(docs.indptr, docs.indices, docs.values)
        assert np.array_equal(g, o)
    return gpu, ora


def _check_search(gpu, ora, qs, k, kp, budget=0):
    """The GPU index's search (with its own anytime budget, if any) against
    the oracle's at the same budget."""
    gi, gs = gpu.search(_ip(qs), _ix(qs), qs.values, k=k, k_prime=kp)
    gpu.sync()
    ci, cs, cnt = gpu.candidates(_ip(qs), _ix(qs), qs.values, kp)
    gi, gs = gi.cpu().numpy().astype(np.uint32), gs.cpu().numpy()
    ci, cs, cnt = ci.cpu().numpy().astype(np.uint32), cs.cpu().numpy(), cnt.cpu().numpy()
    ref = ora.search(qs.indptr, qs.indices, qs.values, k=k, k_prime=kp, candidates=True,
                     budget=budget)
    live = ora.live_mask()
    swaps = 0
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        kq = min(kp, int(live.sum()))
        assert cnt[r] == kq
        approx, amag = ora.scores(qi, qv, with_magnitude=True, budget=budget)
        exact, emag = ora.exact_scores(qi, qv, with_magnitude=True)
        # candidate approximate scores agree with the oracle's Alg. 6 scores
        for i, s in zip(ci[r][:kq], cs[r][:kq]):
            assert live[i]
            assert parity.score_close(s, approx[i], amag[i])
        swaps += parity.check_candidate_set(ci[r], ref["cand_ids"][r], approx, amag, kq)
        parity.check_topk(gi[r], gs[r], ci[r][:kq], exact, emag, k)
        # and the final top-k equals the oracle's except inside the band
        r_ = min(k, kq)
        if list(gi[r][:r_]) != list(ref["ids"][r][:r_]):
            tau = ref["scores"][r][r_ - 1]
            for i in set(gi[r][:r_]) ^ set(ref["ids"][r][:r_]):
                assert abs(exact[i] - tau) <= 2e-5 * max(emag[i], 1e-30) or \
                    i not in set(ref["cand_ids"][r]) or i not in set(ci[r][:kq])
    return swaps


# ---------------------------------------------------------------- mappings

@pytest.mark.parametrize("n,m,h,seed", [(1000, 64, 1, 0x5151), (30000, 64, 2, 7),
                                        (30522, 128, 1, 0x5151), (777, 5, 3, 99)])
def test_hash_table_bit_exact(n, m, h, seed):
    g = sinnamon.Index(n, m, h, seed=seed)
    o = oracle.OracleIndex(n, m, h, seed=seed)
    assert np.array_equal(g.hash_table(), o.hash_table())


# --------------------------------------------------------------- indexing

@pytest.mark.parametrize("name,n_docs,tile", [("tiny", 3500, 1024), ("mixed", 2600, 1024),
                                              ("text", 2100, 2048)])
def test_sketch_and_lists_bit_exact(name, n_docs, tile):
    """Alg. 5: every sketch bin equals the oracle's bit for bit (bins are copies
    of input values) and every inverted list holds the same ids."""
    w = synth.WORKLOADS[name]
    w = synth.scaled(w, n_docs, n=min(w.n, 3000))
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, None, tile_docs=tile)
    # two batches: the second lands partly in an already-built tile
    for part in (docs.slice(0, n_docs // 3), docs.slice(n_docs // 3, n_docs)):
        g = gpu.insert(_ip(part), _ix(part), part.values).cpu().numpy().astype(np.uint32)
        o = ora.insert(part.indptr, part.indices, part.values)
        assert np.array_equal(g, o)
    ids = np.arange(n_docs, dtype=np.int32)
    u, l = gpu.sketch_columns(ids)
    u, l = u.cpu().numpy(), l.cpu().numpy()
    for i in range(n_docs):
        ou, ol = ora.sketch_column(i)
        assert np.array_equal(u[i], ou.astype(np.float32)), i
        assert np.array_equal(l[i], ol.astype(np.float32)), i
    for j in range(w.n):
        assert np.array_equal(gpu.inverted_list(j), ora.inverted_list(j)), j
    st = gpu.stats()
    assert st["live"] == n_docs and st["tombstones"] == 0
    assert st["postings"] == int((docs.values != 0).sum())


# ---------------------------------------------------------------- scoring

@pytest.mark.parametrize("name,n_docs,tile,nq", [("tiny", 5000, 1024, 30),
                                                 ("mixed", 3300, 1024, 20),
                                                 ("text", 4100, 1024, 20)])
def test_scores_within_tolerance(name, n_docs, tile, nq):
    """Alg. 6 scores over every slot (several tiles and a ragged last tile)."""
    w = synth.scaled(synth.WORKLOADS[name], n_docs, n=min(synth.WORKLOADS[name].n, 4000))
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=nq)
    gpu, ora = _pair(w, docs, tile_docs=tile)
    s = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
    live = ora.live_mask()
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        ref, mag = ora.scores(qi, qv, with_magnitude=True)
        parity.check_dense_scores(s[r][: ref.size], ref, mag, live)
        assert np.all(np.isneginf(s[r][ref.size:]))


def test_injective_mapping_scores_are_exact():
    """m = n and a permutation mapping: no bin is shared, so Alg. 6 returns
    exact inner products (fp32)."""
    n = 512
    perm = np.random.default_rng(1).permutation(n).astype(np.uint32)
    w = synth.scaled(synth.WORKLOADS["tiny"], 2000, n=n, m=n)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=10)
    gpu, ora = _pair(w, docs, table=perm)
    s = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        ex, mag = ora.exact_scores(qi, qv, with_magnitude=True)
        assert np.all(parity.score_close(s[r][: ex.size], ex, mag))


# ----------------------------------------------------------------- search

@pytest.mark.parametrize("name,n_docs,tile,nq,k,kp", [
    ("tiny", 10_000, 1024, 100, 10, 100),      # the tiny workload at full size
    ("mixed", 6000, 2048, 25, 10, 500),        # small batch: dense scoring
    ("mixed", 9000, 1024, 48, 10, 500),        # batch: emitted candidates
    ("text", 6000, 4096, 25, 10, 300),
    ("text", 12000, 1024, 64, 10, 1000),
    ("tiny", 3000, 1024, 10, 1, 1),            # k = k' = 1
    ("tiny", 2500, 1024, 10, 32, 2500),        # k' = |X|: exact top-k
])
def test_search_matches_oracle(name, n_docs, tile, nq, k, kp):
    w = synth.scaled(synth.WORKLOADS[name], n_docs, n=min(synth.WORKLOADS[name].n, 5000))
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=nq)
    gpu, ora = _pair(w, docs, tile_docs=tile)
    # at k' >= |X| every live id is a candidate, so the tie-band check of the
    # top k against the candidates is the check against the exact top k
    _check_search(gpu, ora, qs, k, kp)


def test_per_query_kprime():
    w = synth.scaled(synth.WORKLOADS["tiny"], 4000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=12)
    gpu, ora = _pair(w, docs)
    kps = np.array([10, 20, 50, 100, 400, 5, 1000, 10, 11, 12, 99, 4000], np.int32)
    gi, gs = gpu.search(_ip(qs), _ix(qs), qs.values, k=10, k_prime=kps, k_prime_max=2000)
    gi = gi.cpu().numpy().astype(np.uint32)
    for r in range(qs.rows):
        kp = int(min(max(kps[r], 10), 2000))
        one = qs.take([r])
        ref = ora.search(one.indptr, one.indices, one.values, k=10, k_prime=kp)
        ai, _ = gpu.search(_ip(one), _ix(one), one.values, k=10, k_prime=kp)
        assert np.array_equal(gi[r], ai.cpu().numpy().astype(np.uint32)[0])
        qi, qv = one.row(0)
        exact, emag = ora.exact_scores(qi, qv, with_magnitude=True)
        tau = ref["scores"][0][-1]
        for i in set(gi[r]) ^ set(ref["ids"][0]):
            assert abs(exact[i] - tau) <= 2e-5 * emag[i] or kp < 100


def test_host_buffer_search_equals_device_search():
    w = synth.scaled(synth.WORKLOADS["tiny"], 3000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=16)
    gpu, _ = _pair(w, docs)
    di, ds = gpu.search(_ip(qs), _ix(qs), qs.values, k=10, k_prime=100)
    hi = np.zeros((qs.rows, 10), np.uint32)
    hs = np.zeros((qs.rows, 10), np.float32)
    sinnamon.sinn_search_host(gpu.handle, qs.indptr.astype(np.uint64), qs.indices, qs.values,
                              10, 100, hi, hs)
    assert np.array_equal(di.cpu().numpy().astype(np.uint32), hi)
    assert np.array_equal(ds.cpu().numpy(), hs)


# -------------------------------------------------------------- streaming

def test_streaming_insert_delete_search():
    """Interleaved inserts, deletes and searches replayed on both sides: ids,
    lists, sketch columns of live ids and search results agree throughout, and
    a reused id never scores through its previous owner's postings."""
    w = synth.scaled(synth.WORKLOADS["mixed"], 0, n=2000)
    pool = synth.make_docs(w, n_docs=9000, seed=5)
    qs = synth.make_queries(w, n_q=40, seed=6)
    gpu, ora = _pair(w, None, tile_docs=1024)
    rng = np.random.default_rng(0)
    pos = 0
    for step in range(8):
        nb = int(rng.integers(200, 1500))
        part = pool.slice(pos, min(pos + nb, pool.rows))
        pos += part.rows
        g = gpu.insert(_ip(part), _ix(part), part.values).cpu().numpy().astype(np.uint32)
        o = ora.insert(part.indptr, part.indices, part.values)
        assert np.array_equal(g, o)
        live = ora.live_ids()
        dele = rng.choice(live, size=min(live.size, int(rng.integers(50, 600))), replace=False)
        gpu.delete(dele.astype(np.int32))
        ora.delete(dele.astype(np.uint32))
        st = gpu.stats()
        assert st["live"] == ora.live_count
        _check_search(gpu, ora, qs, 10, 200)
    for j in range(0, w.n, 7):
        assert np.array_equal(gpu.inverted_list(j), ora.inverted_list(j))
    live = ora.live_ids()
    u, l = gpu.sketch_columns(live.astype(np.int32))
    u = u.cpu().numpy()
    for t, i in enumerate(live[:500]):
        assert np.array_equal(u[t], ora.sketch_column(int(i))[0].astype(np.float32))


def test_delete_leaves_stale_column_and_reuse_overwrites():
    w = synth.scaled(synth.WORKLOADS["tiny"], 1500)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs)
    before = gpu.sketch_columns([5])[0].cpu().numpy()
    gpu.delete([5, 700])
    ora.delete([5, 700])
    assert np.array_equal(gpu.sketch_columns([5])[0].cpu().numpy(), before)
    assert gpu.stats()["tombstones"] == int((docs.row(5)[1] != 0).sum() + (docs.row(700)[1] != 0).sum())
    new = synth.make_docs(w, n_docs=3, seed=77)
    g = gpu.insert(_ip(new), _ix(new), new.values).cpu().numpy()
    assert list(g) == [5, 700, 1500]
    ora.insert(new.indptr, new.indices, new.values)
    u = gpu.sketch_columns([5, 700])[0].cpu().numpy()
    assert np.array_equal(u[0], ora.sketch_column(5)[0].astype(np.float32))
    assert gpu.stats()["tombstones"] == 0  # the rebuilt tile compacted them
    for j in range(w.n):
        assert np.array_equal(gpu.inverted_list(j), ora.inverted_list(j))


@pytest.mark.parametrize("h", [1, 2])
def test_containers_around_the_bitmap_threshold(h):
    """Per-tile posting counts of a coordinate on both sides of every plausible
    array/bitmap switch (T/16, T/8, T/4 of a T-id tile, and T itself), with
    mixed signs, tombstones in both kinds of container and a rebuild: lists
    stay bit-exact and the Alg. 6 scores and searches match the oracle."""
    T, n = 1024, 64
    w = synth.scaled(synth.WORKLOADS["tiny"], 0, n=n, m=16, h=h)
    targets = [T // 16 - 1, T // 16, T // 8 - 1, T // 8, T // 4 - 1, T // 4, T // 2, T, 1, 3]
    n_docs = 2 * T + 300
    rng = np.random.default_rng(40 + h)
    dense = np.zeros((n_docs, n), bool)
    for t0 in range(0, n_docs, T):
        rows = min(T, n_docs - t0)
        for c, cnt in enumerate(targets):
            dense[t0 + rng.choice(rows, size=min(cnt, rows), replace=False), c] = True
    dense[:, n - 1] = True                                   # no empty vector
    extra = rng.random((n_docs, n)) < 0.02                   # sparse background
    extra[:, : len(targets)] = False                         # exact counts there
    dense |= extra
    idx = [np.flatnonzero(r).astype(np.uint32) for r in dense]
    indptr = np.concatenate([[0], np.cumsum([a.size for a in idx])]).astype(np.uint64)
    indices = np.concatenate(idx)
    values = rng.standard_normal(indices.size).astype(np.float32)
    values[values == 0] = 0.5
    docs = synth.CSR(indptr, indices, values)
    gpu, ora = _pair(w, docs, tile_docs=T)
    qrows = []
    for _ in range(16):
        c = np.sort(rng.choice(len(targets), size=6, replace=False)).astype(np.uint32)
        c = np.concatenate([c, np.sort(rng.choice(np.arange(len(targets), n), 3, replace=False)).astype(np.uint32)])
        qrows.append(np.sort(c))
    qip = np.concatenate([[0], np.cumsum([r.size for r in qrows])]).astype(np.uint64)
    qs = synth.CSR(qip, np.concatenate(qrows), rng.standard_normal(int(qip[-1])).astype(np.float32))

    def check():
        for j in range(n):
            assert np.array_equal(gpu.inverted_list(j), ora.inverted_list(j)), j
        s = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
        live = ora.live_mask()
        for r in range(qs.rows):
            qi, qv = qs.row(r)
            ref, mag = ora.scores(qi, qv, with_magnitude=True)
            parity.check_dense_scores(s[r][: ref.size], ref, mag, live)
        _check_search(gpu, ora, qs, 10, 200)

    check()
    dele = rng.choice(n_docs, size=n_docs // 7, replace=False)
    gpu.delete(dele.astype(np.int32))
    ora.delete(dele.astype(np.uint32))
    check()
    new = synth.CSR(indptr[:401] - indptr[0], indices[: int(indptr[400])], -values[: int(indptr[400])])
    g = gpu.insert(_ip(new), _ix(new), new.values).cpu().numpy().astype(np.uint32)
    assert np.array_equal(g, ora.insert(new.indptr, new.indices, new.values))
    check()


# ------------------------------------------------------------ edge cases

def test_empty_and_degenerate_queries():
    w = synth.scaled(synth.WORKLOADS["tiny"], 1200)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs)
    gpu.delete([0, 3])
    ora.delete([0, 3])
    # empty query, all-zero query, single-coordinate query
    ip = np.array([0, 0, 2, 3], np.int64)
    idx = np.array([4, 9, 17], np.int32)
    val = np.array([0.0, 0.0, -1.5], np.float32)
    qs = synth.CSR(ip.astype(np.uint64), idx.astype(np.uint32), val)
    gi, gs = gpu.search(ip, idx, val, k=5, k_prime=50)
    gpu.sync()
    gi = gi.cpu().numpy().astype(np.uint32)
    ref = ora.search(qs.indptr, qs.indices, qs.values, k=5, k_prime=50)
    assert list(gi[0]) == [1, 2, 4, 5, 6]  # all scores 0: smallest live ids
    assert list(gi[1]) == [1, 2, 4, 5, 6]
    assert np.all(gs.cpu().numpy()[:2] == 0.0)
    _check_search(gpu, ora, qs, 5, 50)
    assert list(gi[2]) == list(ref["ids"][2])


def test_fewer_live_than_k_and_empty_index():
    w = synth.scaled(synth.WORKLOADS["tiny"], 6)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs)
    qs = synth.make_queries(w, n_q=3)
    gi, gs = gpu.search(_ip(qs), _ix(qs), qs.values, k=10, k_prime=20)
    gi = gi.cpu().numpy().astype(np.uint32)
    assert np.all(gi[:, 6:] == 0xFFFFFFFF)
    assert np.all(np.isneginf(gs.cpu().numpy()[:, 6:]))
    _check_search(gpu, ora, qs, 10, 20)
    gpu.delete(np.arange(6, dtype=np.int32))
    gi, gs = gpu.search(_ip(qs), _ix(qs), qs.values, k=3, k_prime=3)
    assert np.all(gi.cpu().numpy().astype(np.uint32) == 0xFFFFFFFF)
    empty = sinnamon.Index(w.n, w.m, w.h)
    gi, gs = empty.search(_ip(qs), _ix(qs), qs.values, k=3, k_prime=3)
    assert np.all(gi.cpu().numpy().astype(np.uint32) == 0xFFFFFFFF)


def test_heavy_ties_at_the_boundary():
    """Many documents with identical scores around the k'-th: the select must
    still take exactly k' by (score desc, id asc), as the oracle's Alg. 3."""
    n, m = 64, 64
    rows = [([3], [1.0])] * 3000 + [([3], [2.0])] * 50 + [([5], [1.0])] * 100
    ip = np.zeros(len(rows) + 1, np.uint64)
    ip[1:] = np.cumsum([1] * len(rows))
    idx = np.array([r[0][0] for r in rows], np.uint32)
    val = np.array([r[1][0] for r in rows], np.float32)
    docs = synth.CSR(ip, idx, val)
    w = synth.scaled(synth.WORKLOADS["tiny"], len(rows), n=n, m=m)
    gpu, ora = _pair(w, docs)
    q = synth.CSR(np.array([0, 2], np.uint64), np.array([3, 5], np.uint32),
                  np.array([1.0, 0.5], np.float32))
    ci, cs, cnt = gpu.candidates(_ip(q), _ix(q), q.values, 1000)
    ref = ora.search(q.indptr, q.indices, q.values, k=10, k_prime=1000, candidates=True)
    assert set(ci.cpu().numpy().astype(np.uint32)[0]) == set(ref["cand_ids"][0])
    gi, gs = gpu.search(_ip(q), _ix(q), q.values, k=10, k_prime=1000)
    assert list(gi.cpu().numpy().astype(np.uint32)[0]) == list(ref["ids"][0])


def test_invalid_inputs_are_rejected_without_change():
    w = synth.scaled(synth.WORKLOADS["tiny"], 100)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs)
    before = gpu.stats()
    bad = [(np.array([0, 2], np.int64), np.array([5, 5], np.int32), np.array([1, 1], np.float32)),
           (np.array([0, 2], np.int64), np.array([7, 5], np.int32), np.array([1, 1], np.float32)),
           (np.array([0, 1], np.int64), np.array([w.n], np.int32), np.array([1], np.float32)),
           (np.array([0, 1], np.int64), np.array([1], np.int32), np.array([np.nan], np.float32))]
    for ip, idx, val in bad:
        with pytest.raises(sinnamon.SinnError) as e:
            gpu.insert(ip, idx, val)
        assert e.value.code == sinnamon.SINN_EINVAL
    assert gpu.stats() == before
    with pytest.raises(sinnamon.SinnError) as e:
        gpu.delete([100])
    assert e.value.code == sinnamon.SINN_ENOTFOUND
    with pytest.raises(sinnamon.SinnError) as e:
        gpu.delete([1, 1])
    assert e.value.code == sinnamon.SINN_EINVAL
    assert gpu.stats() == before
    with pytest.raises(sinnamon.SinnError):
        gpu.search(np.array([0, 1], np.int64), np.array([1], np.int32), np.array([1.0], np.float32),
                   k=5, k_prime=4)
    # a malformed query: padded row and a device error at sync
    gi, gs = gpu.search(np.array([0, 2, 3], np.int64), np.array([9, 2, 4], np.int32),
                        np.array([1, 1, 1], np.float32), k=3, k_prime=10)
    with pytest.raises(sinnamon.SinnError) as e:
        gpu.sync()
    assert e.value.code == sinnamon.SINN_EINVAL
    assert np.all(gi.cpu().numpy()[0] == -1)
    gpu.sync()  # error was cleared
    assert np.all(gi.cpu().numpy()[1] >= 0)
    with pytest.raises(sinnamon.SinnError):
        sinnamon.sinn_create(0, 4, 1)
    with pytest.raises(sinnamon.SinnError):
        sinnamon.sinn_create(10, 4, 5)


@pytest.mark.parametrize("nq", [1, 40])
@pytest.mark.parametrize("case", ["l1", "l2", "ties"])
def test_select_levels(case, nq):
    """The k'-th score falls in a bin too large to collect at once, so the
    select narrows it with finer digits (l1, l2) or, for more exact ties than
    the boundary buffer holds, takes the smallest ids in order (ties)."""
    rng = np.random.default_rng(3)
    nd = 100_000
    if case == "l1":    # distinct values sharing their top 12 key bits
        vals = (1.0 + np.arange(nd) * np.finfo(np.float32).eps).astype(np.float32)
    elif case == "l2":  # many exact repeats inside one 24-bit bin
        vals = (1.0 + rng.integers(0, 200, nd) * np.finfo(np.float32).eps).astype(np.float32)
    else:               # all equal
        vals = np.ones(nd, np.float32)
    rng.shuffle(vals)
    ip = np.arange(nd + 1, dtype=np.uint64)
    docs = synth.CSR(ip, np.zeros(nd, np.uint32), vals)
    w = synth.scaled(synth.WORKLOADS["tiny"], nd, n=16, m=16)
    gpu, ora = _pair(w, docs, tile_docs=8192)
    # the same query nq times (a batch of 40 takes the emitted-candidate path
    # and falls back to dense scoring because the boundary bin is huge)
    q = synth.CSR(np.arange(nq + 1, dtype=np.uint64), np.zeros(nq, np.uint32),
                  np.ones(nq, np.float32))
    for kp in (1000, 70_000):
        ci, cs, cnt = gpu.candidates(_ip(q), _ix(q), q.values, kp)
        gpu.sync()
        ref = ora.search(q.indptr[:2], q.indices[:1], q.values[:1], k=10, k_prime=kp,
                         candidates=True)
        gi, gs = gpu.search(_ip(q), _ix(q), q.values, k=10, k_prime=kp)
        ci, gi = ci.cpu().numpy().astype(np.uint32), gi.cpu().numpy().astype(np.uint32)
        for r in range(nq):
            assert int(cnt[r]) == kp
            assert set(ci[r]) == set(ref["cand_ids"][0])
            assert list(gi[r]) == list(ref["ids"][0])


def test_parameters_at_their_maxima():
    """m = 4096 bins, h = 8 mappings, tiles of 16384 ids, a query with exactly
    the default limit of 1024 non-zeros, k = 1024: the search matches the
    oracle; one non-zero more is a malformed query."""
    n = 6000
    w = synth.scaled(synth.WORKLOADS["mixed"], 3000, n=n, m=4096, h=8)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs, tile_docs=16384)
    rng = np.random.default_rng(17)
    rows = []
    for nnz in (1024, 700, 1):
        idx = np.sort(rng.choice(n, nnz, replace=False)).astype(np.uint32)
        rows.append((idx, rng.normal(0, 1, nnz).astype(np.float32)))
    qs = synth.CSR(np.concatenate([[0], np.cumsum([r[0].size for r in rows])]).astype(np.uint64),
                   np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows]))
    _check_search(gpu, ora, qs, 1024, 2048)
    idx = np.sort(rng.choice(n, 1025, replace=False)).astype(np.int32)
    gi, gs = gpu.search(np.array([0, 1025], np.int64), idx, np.ones(1025, np.float32),
                        k=10, k_prime=20)
    with pytest.raises(sinnamon.SinnError) as e:
        gpu.sync()
    assert e.value.code == sinnamon.SINN_EINVAL
    assert np.all(gi.cpu().numpy() == -1)


def test_empty_batches_are_no_ops():
    """Zero documents to insert, zero ids to delete and zero queries to search
    are accepted and change nothing."""
    w = synth.scaled(synth.WORKLOADS["tiny"], 500)
    docs = synth.make_docs(w)
    gpu, ora = _pair(w, docs)
    before = gpu.stats()
    ids = gpu.insert(np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert ids.numel() == 0
    gpu.delete(np.zeros(0, np.int32))
    gi, gs = gpu.search(np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32),
                        k=10, k_prime=20)
    gpu.sync()
    assert gi.shape == (0, 10) and gs.shape == (0, 10)
    assert gpu.stats() == before
