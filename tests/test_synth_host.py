"""The seeded input generators (no GPU): the shapes and distributions the
workloads state hold, and the same seed gives the same collection."""
import numpy as np
import pytest

from paper_2301_10622_gb300 import synth


def _rows_ok(ip, idx, counts, n):
    ip = ip.astype(np.int64)
    assert np.array_equal(np.diff(ip), counts)
    for r in range(len(counts)):
        row = idx[ip[r]:ip[r + 1]].astype(np.int64)
        assert np.all(np.diff(row) > 0) and (row.size == 0 or (row[0] >= 0 and row[-1] < n))


def test_alias_table_reproduces_the_weights_exactly():
    w = 1.0 / np.arange(1, 301, dtype=np.float64) ** 1.3
    prob, alias = synth._alias_table(w)
    n = w.size
    p = prob / n
    np.add.at(p, alias, (1.0 - prob) / n)
    assert np.allclose(p, w / w.sum(), rtol=1e-12, atol=1e-15)


def test_uniform_coords_distinct_sorted_and_uniform():
    rng = np.random.default_rng(1)
    n = 200
    counts = rng.integers(1, 60, 3000)
    counts[:50] = 150  # dense rows take the permutation path (2k > n)
    ip, idx = synth.uniform_coords(rng, counts, n)
    _rows_ok(ip, idx, counts, n)
    f = np.bincount(idx, minlength=n)
    e = f.sum() / n
    chi2 = ((f - e) ** 2 / e).sum()          # 199 dof: 99.9% point ~ 268
    assert chi2 < 268, chi2


def test_zipf_single_draws_follow_the_weights():
    rng = np.random.default_rng(2)
    n, rows = 1000, 200_000
    ip, idx = synth.zipf_coords(rng, np.ones(rows, np.int64), n, s=1.0)
    f = np.bincount(idx, minlength=n).astype(np.float64)
    p = 1.0 / np.arange(1, n + 1)
    p /= p.sum()
    # the 20 most popular coordinates one by one, the rest pooled
    obs = np.concatenate([f[:20], [f[20:].sum()]])
    exp = np.concatenate([p[:20], [p[20:].sum()]]) * rows
    chi2 = ((obs - exp) ** 2 / exp).sum()    # 20 dof: 99.9% point ~ 45
    assert chi2 < 45, chi2


def test_zipf_rows_are_distinct_sorted_sets():
    rng = np.random.default_rng(3)
    counts = np.concatenate([rng.integers(1, 200, 500), [900, 1000]])
    ip, idx = synth.zipf_coords(rng, counts, 1000)
    _rows_ok(ip, idx, counts, 1000)
    assert np.all(idx[ip[-2].astype(np.int64):] == np.arange(1000))  # a full row


def test_lognormal_counts_have_the_stated_mean():
    rng = np.random.default_rng(4)
    c = synth.lognormal_counts(rng, 200_000, 120.0, 0.5, 30522)
    assert abs(c.mean() - 120.0) < 0.5 and c.min() >= 1


@pytest.mark.parametrize("name", ["tiny", "text", "mixed"])
def test_workloads_are_seeded_and_shaped(name):
    w = synth.scaled(synth.WORKLOADS[name], 2000, n_queries=300)
    d1, d2 = synth.make_docs(w), synth.make_docs(w)
    q = synth.make_queries(w)
    assert d1.rows == 2000 and q.rows == 300
    assert np.array_equal(d1.indices, d2.indices) and np.array_equal(d1.values, d2.values)
    other = synth.make_docs(w, seed=12345)
    assert not np.array_equal(other.values[:100], d1.values[:100])
    dn = np.diff(d1.indptr.astype(np.int64))
    qn = np.diff(q.indptr.astype(np.int64))
    _rows_ok(d1.indptr, d1.indices, dn, w.n)
    if name == "tiny":
        assert np.all(dn == 32) and np.all(qn == 16)
    if name == "text":
        assert 110 < dn.mean() < 130 and 40 < qn.mean() < 50
        assert np.all(d1.values > 0) and np.all(q.values > 0)
        f = np.bincount(d1.indices, minlength=w.n)
        assert f[0] > 0.9 * d1.rows and f[:10].sum() > f[-10000:].sum()  # popular head
    if name == "mixed":
        assert dn.min() >= 80 and dn.max() <= 160 and np.all(qn == 40)
        assert 0.4 < (d1.values < 0).mean() < 0.6
