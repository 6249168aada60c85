"""The paper's variants on the GPU against the oracle: SINNAMON+ (the Sec.
4.1 note: non-negative data, no lower sketch L), Alg. 6's anytime budget
(the break after a term once the time budget, counted in postings, is
spent) and bfloat16 sketch bins (Sec. 4.1 notes; upper bins rounded up,
lower bins down)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402
from tests import parity  # noqa: E402
from tests.test_gpu_parity import _check_search, _ip, _ix, _pair  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


# ------------------------------------------------------------ SINNAMON+

def test_nonneg_index_keeps_only_u_and_matches_the_oracle():
    w = synth.scaled(synth.WORKLOADS["text"], 9000, n=5000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=40)
    plus, ora = _pair(w, docs, tile_docs=1024, flags=sinnamon.SINN_FLAG_NONNEG)
    full, _ = _pair(w, docs, tile_docs=1024)
    sp, sf = plus.stats(), full.stats()
    assert sp["bytes_sketch"] * 2 == sf["bytes_sketch"]
    ids = np.arange(0, 9000, 97, dtype=np.int32)
    u_p, l_p = plus.sketch_columns(ids)
    u_f, _ = full.sketch_columns(ids)
    assert l_p is None and torch.equal(u_p, u_f)             # U bit for bit
    for i in ids[:20]:
        u_o, _ = ora.sketch_column(int(i))
        assert np.array_equal(u_p[list(ids).index(i)].cpu().numpy().astype(np.float64), u_o)
    _check_search(plus, ora, qs, 10, 300)
    s = plus.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
    live = ora.live_mask()
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        ref, mag = ora.scores(qi, qv, with_magnitude=True)
        parity.check_dense_scores(s[r][: ref.size], ref, mag, live)


def test_nonneg_rejects_negative_inputs():
    w = synth.scaled(synth.WORKLOADS["text"], 2000, n=3000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=6)
    plus, _ = _pair(w, docs, flags=sinnamon.SINN_FLAG_NONNEG)
    before = plus.stats()
    bad = docs.slice(0, 3)
    vals = bad.values.copy()
    vals[1] = -vals[1]
    with pytest.raises(sinnamon.SinnError) as e:
        plus.insert(_ip(bad), _ix(bad), vals)
    assert e.value.code == sinnamon.SINN_EINVAL and plus.stats() == before
    qv = qs.values.copy()
    qv[0] = -abs(qv[0])                                       # row 0 negative
    ids, sc = plus.search(_ip(qs), _ix(qs), qv, k=10, k_prime=100)
    with pytest.raises(sinnamon.SinnError) as e:
        plus.sync()
    assert e.value.code == sinnamon.SINN_EINVAL
    assert (ids[0].cpu().numpy().astype(np.int64) & 0xFFFFFFFF == 0xFFFFFFFF).all()
    assert np.isneginf(sc[0].cpu().numpy()).all()
    assert (ids[1:].cpu().numpy() != -1).all()                # the other rows ran
    with pytest.raises(sinnamon.SinnError):
        sinnamon.Index(10, 4, 1, flags=4)                     # unknown flag


# -------------------------------------------------------------- anytime

@pytest.mark.parametrize("name,n_docs,nq", [("text", 9000, 40), ("mixed", 5000, 33)])
def test_anytime_budget_matches_the_oracle(name, n_docs, nq):
    w = synth.scaled(synth.WORKLOADS[name], n_docs, n=min(synth.WORKLOADS[name].n, 4000))
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=nq)
    gpu, ora = _pair(w, docs, tile_docs=1024)
    # stale postings must not count: delete some documents first
    dele = np.arange(3, n_docs, 11, dtype=np.uint32)
    gpu.delete(dele.astype(np.int32))
    ora.delete(dele)
    lens = np.array([ora.inverted_list(j).size for j in range(w.n)])
    mean_total = np.mean([lens[qs.row(r)[0]].sum() for r in range(qs.rows)])
    live = ora.live_mask()
    for budget in (1, int(mean_total // 4), int(mean_total)):
        gpu.set_budget(budget)
        assert gpu.budget == budget
        s = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
        for r in range(qs.rows):
            qi, qv = qs.row(r)
            ref, mag = ora.scores(qi, qv, with_magnitude=True, budget=budget)
            parity.check_dense_scores(s[r][: ref.size], ref, mag, live)
        _check_search(gpu, ora, qs, 10, 200, budget=budget)
    gpu.set_budget(0)
    full = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
    qi, qv = qs.row(0)
    ref, mag = ora.scores(qi, qv, with_magnitude=True)
    parity.check_dense_scores(full[0][: ref.size], ref, mag, live)


def test_budget_change_records_a_plan_again():
    w = synth.scaled(synth.WORKLOADS["text"], 5000, n=3000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=64)
    gpu, ora = _pair(w, docs, tile_docs=1024)
    q = (torch.from_numpy(_ip(qs)).cuda(), torch.from_numpy(_ix(qs)).cuda(),
         torch.from_numpy(qs.values).cuda())
    plan = sinnamon.Plan(gpu, *q, k=10, k_prime_max=100, scratch_bytes=64 << 20)
    plan.run()
    gpu.set_budget(500)
    ids, sc = (x.cpu().numpy() for x in plan.run())
    assert plan.recordings == 2
    ref = ora.search(qs.indptr, qs.indices, qs.values, k=10, k_prime=100, budget=500)
    exact = [ora.exact_scores(*qs.row(r), with_magnitude=True) for r in range(qs.rows)]
    for r in range(qs.rows):
        e, m = exact[r]
        for i, s_ in zip(ids[r], sc[r]):
            assert parity.score_close(s_, e[i], m[i])
        assert np.mean(ids[r] == ref["ids"][r]) >= 0.8


# ------------------------------------------------------- bfloat16 sketch

def _bf16_pair(w, docs, tile_docs=1024, flags=0):
    gpu = sinnamon.Index(w.n, w.m, w.h, tile_docs=tile_docs,
                         flags=flags | sinnamon.SINN_FLAG_BF16_SKETCH)
    ora = oracle.OracleIndex(w.n, w.m, w.h, sketch_bf16=True)
    g = gpu.insert(_ip(docs), _ix(docs), docs.values).cpu().numpy().astype(np.uint32)
    assert np.array_equal(g, ora.insert(docs.indptr, docs.indices, docs.values))
    return gpu, ora


@pytest.mark.parametrize("name,n_docs,nq", [("mixed", 6000, 40), ("text", 9000, 48)])
def test_bf16_sketch_matches_the_oracle(name, n_docs, nq):
    """Bins bit for bit (the oracle's directed rounding), Alg. 6 scores within
    the fp32 bar of the oracle's FP64 sums of the same rounded bins, and the
    search within the tie band."""
    w = synth.scaled(synth.WORKLOADS[name], n_docs, n=min(synth.WORKLOADS[name].n, 4000))
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=nq)
    gpu, ora = _bf16_pair(w, docs)
    full, _ = _pair(w, docs, tile_docs=1024)
    assert gpu.stats()["bytes_sketch"] * 2 == full.stats()["bytes_sketch"]
    ids = np.arange(0, n_docs, 53, dtype=np.int32)
    u, l = gpu.sketch_columns(ids)
    u, l = u.cpu().numpy(), l.cpu().numpy()
    assert np.all(u.view(np.uint32) & 0xFFFF == 0) and np.all(l.view(np.uint32) & 0xFFFF == 0)
    for r, i in enumerate(ids):
        uo, lo = ora.sketch_column(int(i))
        assert np.array_equal(u[r].astype(np.float64), uo)
        assert np.array_equal(l[r].astype(np.float64), lo)
    s = gpu.scores(_ip(qs), _ix(qs), qs.values).cpu().numpy()
    live = ora.live_mask()
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        ref, mag = ora.scores(qi, qv, with_magnitude=True)
        parity.check_dense_scores(s[r][: ref.size], ref, mag, live)
    _check_search(gpu, ora, qs, 10, 300)


def test_bf16_sketch_streams_and_combines_with_nonneg():
    w = synth.scaled(synth.WORKLOADS["text"], 6000, n=3000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=36)
    gpu, ora = _bf16_pair(w, docs.slice(0, 5000), flags=sinnamon.SINN_FLAG_NONNEG)
    dele = np.arange(7, 5000, 13, dtype=np.uint32)
    gpu.delete(dele.astype(np.int32))
    ora.delete(dele)
    rest = docs.slice(5000, 6000)
    g = gpu.insert(_ip(rest), _ix(rest), rest.values).cpu().numpy().astype(np.uint32)
    assert np.array_equal(g, ora.insert(rest.indptr, rest.indices, rest.values))
    _check_search(gpu, ora, qs, 10, 200)
