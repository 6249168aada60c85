"""Failures made on the host, on a GPU that never faults: exhausted memory
injected at each allocation an insert makes (the index must come out
unchanged, then take the same insert once memory is back), at the other
calls that allocate, and a bounded kernel wait that nothing completes (the
host reads an error status and the context stays usable)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402
from tests.test_gpu_parity import _check_search, _ip, _ix, _pair  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield
    sinnamon.sinn_debug_fail_alloc(-1)


def _same_contents(gpu, ora, n, qs):
    st = gpu.stats()
    assert st["live"] == ora.live_count
    for j in range(n):
        assert np.array_equal(gpu.inverted_list(j), ora.inverted_list(j)), j
    _check_search(gpu, ora, qs, 10, 100)


def test_insert_is_all_or_nothing_under_exhausted_memory():
    """The n-th allocation of an insert that grows the id capacity, the
    vector store and several tiles fails, for every n the insert reaches:
    each time SINN_ENOMEM and the same vectors, lists and results as before;
    with memory back, the same insert succeeds and matches the oracle."""
    w = synth.scaled(synth.WORKLOADS["tiny"], 3000, n=400)
    docs = synth.make_docs(w)
    more = synth.make_docs(w, n_docs=5000, seed=91)
    qs = synth.make_queries(w, n_q=12)
    gpu, ora = _pair(w, docs, tile_docs=1024)
    gpu.delete(np.arange(0, 3000, 7, dtype=np.int32))
    ora.delete(np.arange(0, 3000, 7, dtype=np.uint32))
    next_id = gpu.stats()["next_id"]
    failures = 0
    for after in range(64):
        sinnamon.sinn_debug_fail_alloc(after)
        try:
            gpu.insert(_ip(more), _ix(more), more.values)
        except sinnamon.SinnError as e:
            assert e.code == sinnamon.SINN_ENOMEM
            sinnamon.sinn_debug_fail_alloc(-1)
            failures += 1
            assert gpu.stats()["next_id"] == next_id
            _same_contents(gpu, ora, w.n, qs)
            continue
        sinnamon.sinn_debug_fail_alloc(-1)  # every allocation succeeded
        break
    else:
        pytest.fail("the insert never completed")
    assert failures >= 8  # capacity arrays, store, scratch and tile storage
    ids = ora.insert(more.indptr, more.indices, more.values)
    assert gpu.stats()["next_id"] == int(ids.max()) + 1
    _same_contents(gpu, ora, w.n, qs)


def test_other_allocating_calls_report_exhausted_memory_and_recover():
    w = synth.scaled(synth.WORKLOADS["tiny"], 2000, n=400)
    docs = synth.make_docs(w)
    qs = synth.make_queries(w, n_q=8)
    gpu = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024)
    gpu.insert(_ip(docs), _ix(docs), docs.values)
    # a search whose scratch must grow
    sinnamon.sinn_debug_fail_alloc(0)
    with pytest.raises(sinnamon.SinnError) as e:
        gpu.search(_ip(qs), _ix(qs), qs.values, k=10, k_prime=1500)
        gpu.sync()
    assert e.value.code == sinnamon.SINN_ENOMEM
    sinnamon.sinn_debug_fail_alloc(-1)
    ids, _ = gpu.search(_ip(qs), _ix(qs), qs.values, k=10, k_prime=1500)
    gpu.sync()
    ref = oracle.OracleIndex(w.n, w.m, w.h)
    ref.insert(docs.indptr, docs.indices, docs.values)
    want = ref.search(qs.indptr, qs.indices, qs.values, k=10, k_prime=1500)
    assert (ids.cpu().numpy().astype(np.uint32) == want["ids"]).mean() > 0.95
    # index and network creation
    for make in (lambda: sinnamon.Index(w.n, w.m, w.h, tile_docs=1024),
                 lambda: sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=1)):
        sinnamon.sinn_debug_fail_alloc(0)
        with pytest.raises(sinnamon.SinnError) as e:
            make()
        assert e.value.code == sinnamon.SINN_ENOMEM
        sinnamon.sinn_debug_fail_alloc(-1)
        make().close()


def test_a_wait_that_nothing_completes_returns_an_error_status():
    """The bounded mbarrier wait of the tensor-core kernels, run alone: with
    nothing arriving it gives up after its polls and the host reads
    SINN_EDEVICE; with the arrival it completes; the context stays usable."""
    s = torch.cuda.current_stream()
    assert sinnamon.sinn_debug_wait_probe(2000, False, s) == sinnamon.SINN_EDEVICE
    assert sinnamon.sinn_debug_wait_probe(2000, True, s) == sinnamon.SINN_OK
    w = synth.scaled(synth.WORKLOADS["tiny"], 1500)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=6)
    gpu, ora = _pair(w, docs)
    _check_search(gpu, ora, qs, 10, 100)
    mlp = sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=2)
    mlp.forward(torch.zeros((4, sinnamon.KP_FEATURES), device="cuda"))
    mlp.sync()  # no GEMM wait ran out
