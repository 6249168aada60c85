"""Checkpoint and resume (sinn_save / sinn_load): an index that has seen
inserts, deletes (tombstones, free ids), a budget and a tuning comes back
with the same state, and from there behaves exactly as the original: the
same searches bit for bit, the same ids for the next insert, the same lists
and sketch columns, all matching the oracle.  Missing, foreign and truncated
files are refused with SINN_EIO."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_10622_gb300 import sinnamon, synth  # noqa: E402
from tests.test_gpu_parity import _check_search, _ip, _ix, _pair  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _search(ix, qs, k, kp):
    ids, sc = ix.search(_ip(qs), _ix(qs), qs.values, k=k, k_prime=kp)
    ix.sync()
    return ids.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("name,flags", [("mixed", 0), ("text", sinnamon.SINN_FLAG_NONNEG),
                                        ("mixed", sinnamon.SINN_FLAG_BF16_SKETCH)])
def test_saved_index_resumes_exactly(tmp_path, name, flags):
    w = synth.scaled(synth.WORKLOADS[name], 0, n=3000)
    pool = synth.make_docs(w, n_docs=7000, seed=12)
    qs = synth.make_queries(w, n_q=40, seed=13)
    a, ora = _pair(w, pool.slice(0, 5000), tile_docs=1024, flags=flags)
    if flags & sinnamon.SINN_FLAG_BF16_SKETCH:
        ora.close()
        import oracle
        ora = oracle.OracleIndex(w.n, w.m, w.h, seed=0x5151, sketch_bf16=True)
        ora.insert(pool.slice(0, 5000).indptr, pool.slice(0, 5000).indices,
                   pool.slice(0, 5000).values)
    rng = np.random.default_rng(3)
    dele = rng.choice(5000, size=700, replace=False).astype(np.int32)
    a.delete(dele)
    ora.delete(dele.astype(np.uint32))
    a.set_tuning(tiles_per_block=2, bound_every=2)
    path = str(tmp_path / "index.sinn")
    a.save(path)
    b = sinnamon.Index.load(path)
    sa, sb = a.stats(), b.stats()
    for f in ("live", "capacity", "next_id", "postings", "tombstones", "bytes_lists",
              "bytes_sketch", "n", "m", "h", "tile_docs", "flags"):
        assert sa[f] == sb[f], f
    assert a.tuning() == b.tuning()
    for j in range(0, w.n, 11):
        assert np.array_equal(a.inverted_list(j), b.inverted_list(j)), j
    live = np.flatnonzero(ora.live_mask()).astype(np.int32)
    ua, la = a.sketch_columns(live)
    ub, lb = b.sketch_columns(live)
    assert torch.equal(ua, ub) and (la is None or torch.equal(la, lb))
    for k, kp in ((10, 200), (10, 40)):
        ia, sa_ = _search(a, qs, k, kp)
        ib, sb_ = _search(b, qs, k, kp)
        assert np.array_equal(ia, ib) and np.array_equal(sa_, sb_)
    # the next insert takes the same (freed, then fresh) ids on both
    more = pool.slice(5000, 7000)
    ga = a.insert(_ip(more), _ix(more), more.values).cpu().numpy()
    gb = b.insert(_ip(more), _ix(more), more.values).cpu().numpy()
    go = ora.insert(more.indptr, more.indices, more.values)
    assert np.array_equal(ga, gb) and np.array_equal(ga.astype(np.uint32), go)
    if not flags & sinnamon.SINN_FLAG_BF16_SKETCH:
        _check_search(b, ora, qs, 10, 200)
    ia, sa_ = _search(a, qs, 10, 200)
    ib, sb_ = _search(b, qs, 10, 200)
    assert np.array_equal(ia, ib) and np.array_equal(sa_, sb_)
    a.close()
    b.close()


def test_bad_files_are_refused(tmp_path):
    w = synth.scaled(synth.WORKLOADS["tiny"], 1500)
    docs = synth.make_docs(w)
    a, _ = _pair(w, docs)
    good = str(tmp_path / "good.sinn")
    a.save(good)
    data = open(good, "rb").read()
    cases = {"missing": None, "foreign": b"not an index at all" * 10,
             "truncated": data[: len(data) // 2], "empty": b""}
    for name, content in cases.items():
        p = str(tmp_path / f"{name}.sinn")
        if content is not None:
            with open(p, "wb") as f:
                f.write(content)
        with pytest.raises(sinnamon.SinnError) as e:
            sinnamon.Index.load(p)
        assert e.value.code == sinnamon.SINN_EIO, name
    with pytest.raises(sinnamon.SinnError) as e:
        a.save(str(tmp_path / "no_such_dir" / "x.sinn"))
    assert e.value.code == sinnamon.SINN_EIO
    b = sinnamon.Index.load(good)  # the good file still loads
    assert b.stats()["live"] == 1500
    b.close()
    a.close()
    assert os.path.getsize(good) > 0
