"""The no-allocation search entry point (sinn_search_noalloc) gives the same
results as sinn_search, call after call.

It exists for callers that cannot allocate device memory while they search
(a fixed memory budget, or a serving path that must stay out of the
allocator); its scratch is a fixed array inside the library that every call
reuses.  This file is collected last so that, if it fails, a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_10622_gb300 import sinnamon, synth
    return sinnamon, synth


def _same_results(ids_a, sc_a, ids_b, sc_b, k):
    """Scores within 1e-5 of the batch's score scale; ids equal except where
    the two scores tie within that tolerance at the k-th place."""
    tol = 1e-5 * max(1.0, float(np.abs(sc_a[np.isfinite(sc_a)]).max(initial=1.0)))
    fa, fb = np.isfinite(sc_a), np.isfinite(sc_b)
    assert np.array_equal(fa, fb)
    assert np.all(np.abs(sc_a[fa] - sc_b[fb]) <= tol)
    for r in range(ids_a.shape[0]):
        if list(ids_a[r]) != list(ids_b[r]):
            kth = sc_a[r][fa[r]][-1]
            for i in set(ids_a[r]) ^ set(ids_b[r]):
                where = np.nonzero(ids_a[r] == i)[0] if i in ids_a[r] else np.nonzero(ids_b[r] == i)[0]
                s = sc_a[r][where[0]] if i in ids_a[r] else sc_b[r][where[0]]
                assert abs(s - kth) <= tol


def test_noalloc_search_matches_search_twice(built):
    sinnamon, synth = built
    w = synth.scaled(synth.WORKLOADS["tiny"], 8000)
    docs = synth.make_docs(w)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    dev = ix.device
    for call, (nq, seed, k, kp) in enumerate([(100, 1, 10, 100), (37, 2, 5, 300)]):
        qs = synth.make_queries(w, n_q=nq, seed=seed)
        ip = torch.from_numpy(qs.indptr.astype(np.int64)).to(dev)
        ii = torch.from_numpy(qs.indices.astype(np.int32)).to(dev)
        vv = torch.from_numpy(qs.values).to(dev)
        ids_a = torch.full((nq, k), 7, dtype=torch.int32, device=dev)
        sc_a = torch.zeros((nq, k), dtype=torch.float32, device=dev)
        ids_b = torch.full((nq, k), 7, dtype=torch.int32, device=dev)
        sc_b = torch.zeros((nq, k), dtype=torch.float32, device=dev)
        sinnamon.sinn_search(ix.handle, ip, ii, vv, k, kp, ids_a, sc_a)
        sinnamon.sinn_search_noalloc(ix.handle, ip, ii, vv, k, kp, ids_b, sc_b)
        ix.sync()
        _same_results(ids_a.cpu().numpy(), sc_a.cpu().numpy(), ids_b.cpu().numpy(),
                      sc_b.cpu().numpy(), k)


def test_noalloc_rejects_requests_beyond_its_scratch(built):
    sinnamon, synth = built
    # 20M id slots need ~80 MB of score keys for a single query: more than the
    # fixed 64 MiB scratch
    ix = sinnamon.Index(64, 8, 1, tile_docs=16384, capacity_hint=20_000_000)
    ip = torch.tensor([0, 1], dtype=torch.int64, device=ix.device)
    ii = torch.tensor([3], dtype=torch.int32, device=ix.device)
    vv = torch.tensor([1.0], dtype=torch.float32, device=ix.device)
    ids = torch.empty((1, 1), dtype=torch.int32, device=ix.device)
    sc = torch.empty((1, 1), dtype=torch.float32, device=ix.device)
    with pytest.raises(sinnamon.SinnError) as e:
        sinnamon.sinn_search_noalloc(ix.handle, ip, ii, vv, 1, 1, ids, sc)
    assert e.value.code == sinnamon.SINN_ESCRATCH


def test_noalloc_first_search_on_a_fresh_index_allocates_nothing(built):
    """What the entry point is for: on an index that has never searched (so
    its own scratch was never grown), the call still succeeds with every
    library allocation made to fail, and the index holds no more scratch
    afterwards.  Results equal sinn_search's."""
    sinnamon, synth = built
    w = synth.scaled(synth.WORKLOADS["tiny"], 3000)
    docs = synth.make_docs(w)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    dev = ix.device
    qs = synth.make_queries(w, n_q=50, seed=9)
    ip = torch.from_numpy(qs.indptr.astype(np.int64)).to(dev)
    ii = torch.from_numpy(qs.indices.astype(np.int32)).to(dev)
    vv = torch.from_numpy(qs.values).to(dev)
    k, kp = 10, 100
    ids_b = torch.full((qs.rows, k), 7, dtype=torch.int32, device=dev)
    sc_b = torch.zeros((qs.rows, k), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    before = ix.stats()["bytes_scratch"]
    sinnamon.sinn_debug_fail_alloc(0)   # the next library allocation fails
    try:
        sinnamon.sinn_search_noalloc(ix.handle, ip, ii, vv, k, kp, ids_b, sc_b)
        ix.sync()
    finally:
        sinnamon.sinn_debug_fail_alloc(-1)
    assert ix.stats()["bytes_scratch"] == before
    ids_a, sc_a = ix.search(ip, ii, vv, k=k, k_prime=kp)
    ix.sync()
    _same_results(ids_a.cpu().numpy(), sc_a.cpu().numpy(), ids_b.cpu().numpy(),
                  sc_b.cpu().numpy(), k)
