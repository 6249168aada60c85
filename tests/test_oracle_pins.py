"""Pins for the CPU oracle: checks against what the paper and mathematics fix,
never against the oracle's own formulas retyped.

Each test names the passage it pins.  These run without a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2301_10622_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _csr(rows):
    ip = np.zeros(len(rows) + 1, np.uint64)
    ip[1:] = np.cumsum([len(r[0]) for r in rows])
    idx = np.concatenate([np.asarray(r[0], np.uint32) for r in rows]) if rows else np.zeros(0, np.uint32)
    val = np.concatenate([np.asarray(r[1], np.float32) for r in rows]) if rows else np.zeros(0, np.float32)
    return ip, idx, val


def _f(x):
    return float(x) if not isinstance(x, str) else float(x.replace("inf", "inf"))


def _random_index(n, m, h, n_docs, nnz, seed, values="normal", table=None):
    rng = np.random.default_rng(seed)
    counts = np.full(n_docs, nnz)
    ip, idx = synth.uniform_coords(rng, counts, n)
    val = (rng.normal(0, 1, idx.size) if values == "normal" else rng.lognormal(0, 0.7, idx.size)).astype(np.float32)
    ix = oracle.OracleIndex(n, m, h, seed=seed, table=table)
    ids = ix.insert(ip, idx, val)
    return ix, synth.CSR(ip, idx, val), ids


def _random_queries(n, n_q, nnz, seed, values="normal"):
    rng = np.random.default_rng(seed)
    ip, idx = synth.uniform_coords(rng, np.full(n_q, nnz), n)
    val = (rng.normal(0, 1, idx.size) if values == "normal" else rng.lognormal(0, 0.7, idx.size)).astype(np.float32)
    return synth.CSR(ip, idx, val)


# ------------------------------------------------------------------ hashing

def test_mix64_published_outputs():
    """SplitMix64 from state 0 (Steele, Lea, Flood 2014) yields 0xE220A8397B1DCDAF,
    0x6E789E6AA1B965F4, 0x06C45D188009454F: its output function applied to
    gamma, 2*gamma, 3*gamma."""
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for t, w in enumerate(want, start=1):
        assert oracle.mix64((t * g) & (2**64 - 1)) == w


@pytest.mark.parametrize("m,h", [(64, 1), (64, 2), (128, 3)])
def test_mappings_uniform_and_independent(m, h):
    """Alg. 5 asks for h independent random mappings [n] -> [m]: bin loads pass a
    chi-square test and two mappings agree on about 1/m of the coordinates."""
    from scipy import stats
    n = 30000
    tab = oracle.OracleIndex(n, m, h).hash_table()
    assert tab.shape == (n, h) and tab.max() < m
    for o in range(h):
        cnt = np.bincount(tab[:, o], minlength=m)
        chi2 = ((cnt - n / m) ** 2 / (n / m)).sum()
        assert stats.chi2.sf(chi2, m - 1) > 1e-4
    for a in range(h):
        for b in range(a + 1, h):
            agree = (tab[:, a] == tab[:, b]).mean()
            assert abs(agree - 1 / m) < 5 * math.sqrt(1 / m / n) + 1e-3
    # another seed gives another mapping
    assert (oracle.OracleIndex(n, m, h, seed=1).hash_table() != tab).mean() > 0.9


# ----------------------------------------------------------- worked example

def _gold():
    with open(os.path.join(GOLD, "worked_example.json")) as f:
        return json.load(f)


def test_worked_example_h1():
    """Hand-computed sketch (Alg. 5), lists, scores (Alg. 6), ranking (Alg. 7)."""
    g = _gold()
    c = g["cases"][0]
    ix = oracle.OracleIndex(g["n"], g["m"], c["h"], table=np.array(c["table"]))
    ids = ix.insert(*_csr([(d["idx"], d["val"]) for d in c["docs"]]))
    assert list(ids) == [0, 1, 2]
    for i in range(3):
        u, l = ix.sketch_column(i)
        assert list(u) == [float(x) for x in c["sketch_u"][i]]
        assert list(l) == [float(x) for x in c["sketch_l"][i]]
    for j, lst in c["lists"].items():
        assert list(ix.inverted_list(int(j))) == lst
    q = c["query"]
    assert list(ix.scores(q["idx"], q["val"])) == c["approx_scores"]
    assert list(ix.exact_scores(q["idx"], q["val"])) == c["exact_scores"]
    qc = _csr([(q["idx"], q["val"])])
    for s in c["search"]:
        r = ix.search(*qc, k=s["k"], k_prime=s["k_prime"])
        assert list(r["ids"][0]) == s["ids"]
        assert list(r["scores"][0]) == s["scores"]


def test_worked_example_h2():
    """h = 2: upper decode is the min over both bins, lower decode the max."""
    g = _gold()
    c = g["cases"][1]
    ix = oracle.OracleIndex(g["n"], g["m"], c["h"], table=np.array(c["table"]))
    ix.insert(*_csr([(d["idx"], d["val"]) for d in c["docs"]]))
    u, l = ix.sketch_column(0)
    assert list(u) == c["sketch_u"][0] and list(l) == c["sketch_l"][0]
    for q in c["queries"]:
        assert list(ix.scores(q["idx"], q["val"])) == q["approx"]
        assert list(ix.exact_scores(q["idx"], q["val"])) == q["exact"]


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("h", [1, 2, 3])
def test_theorem1_upper_bound(h):
    """Thm. 1: with T = infinity the score is an upper bound of <q, x> for every
    document, mixed-sign data included."""
    ix, docs, ids = _random_index(300, 16, h, 400, 24, seed=11 + h)
    qs = _random_queries(300, 20, 12, seed=5)
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        a = ix.scores(qi, qv)
        e = ix.exact_scores(qi, qv)
        assert np.all(a >= e - 1e-12 * (1 + np.abs(e)))
        assert np.any(a > e + 1e-9)  # m << psi: some estimates are loose


def test_injective_mapping_gives_exact_scores():
    """With m = n and an injective mapping no two coordinates share a bin
    (Event A never happens), so every decode is exact and Alg. 6 returns the
    exact inner products; Alg. 7 then returns the exact top-k."""
    n = 200
    perm = np.random.default_rng(3).permutation(n).astype(np.uint32)[:, None]
    ix, docs, ids = _random_index(n, n, 1, 300, 20, seed=21, table=perm)
    qs = _random_queries(n, 15, 10, seed=8)
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        np.testing.assert_allclose(ix.scores(qi, qv), ix.exact_scores(qi, qv), rtol=0, atol=1e-12)
    res = ix.search(qs.indptr, qs.indices, qs.values, k=10, k_prime=10)
    ex = ix.exact_topk(qs.indptr, qs.indices, qs.values, k=10)
    assert np.array_equal(res["ids"], ex["ids"])


@pytest.mark.parametrize("h", [1, 2])
def test_extremes_decoded_exactly(h):
    """The largest value of a vector is always recovered exactly from U (the
    remark after Thm. 2); symmetrically the smallest is recovered from L."""
    ix, docs, ids = _random_index(500, 8, h, 60, 40, seed=31)
    for d in range(docs.rows):
        idx, val = docs.row(d)
        jmax, jmin = int(idx[np.argmax(val)]), int(idx[np.argmin(val)])
        up = ix.scores([jmax], [1.0])[ids[d]]
        lo = ix.scores([jmin], [-1.0])[ids[d]]
        assert up == float(val.max())
        assert lo == -float(val.min())


def test_event_a_characterises_exact_decodes():
    """Proof of Thm. 2: with h = 1 the upper decode of x[i] is exact iff no
    other active coordinate in the same bin holds a larger value (Event A)."""
    ix, docs, ids = _random_index(400, 16, 1, 80, 20, seed=41)
    tab = ix.hash_table()[:, 0]
    for d in range(docs.rows):
        idx, val = docs.row(d)
        for t in range(idx.size):
            dec = ix.scores([int(idx[t])], [1.0])[ids[d]]
            clash = any(tab[idx[s]] == tab[idx[t]] and val[s] > val[t]
                        for s in range(idx.size) if s != t)
            assert (dec == float(val[t])) == (not clash)
            assert dec >= float(val[t])


def test_kprime_covering_all_docs_gives_exact_topk():
    """Alg. 7 with k' >= |X| re-ranks every live document exactly, so its top-k
    is the exact top-k of Eq. 2."""
    ix, docs, ids = _random_index(300, 8, 2, 250, 15, seed=51)
    qs = _random_queries(300, 20, 8, seed=9)
    r = ix.search(qs.indptr, qs.indices, qs.values, k=12, k_prime=250)
    e = ix.exact_topk(qs.indptr, qs.indices, qs.values, k=12)
    assert np.array_equal(r["ids"], e["ids"])
    np.testing.assert_allclose(r["scores"], e["scores"], rtol=0, atol=1e-12)


def test_bruteforce_matches_dense_library_matmul():
    """Eq. 2 by the oracle's sparse brute force equals numpy's dense matrix
    product followed by a lexicographic sort (score desc, id asc)."""
    n = 150
    ix, docs, ids = _random_index(n, 8, 1, 120, 10, seed=61)
    qs = _random_queries(n, 10, 6, seed=10)
    X = np.zeros((docs.rows, n))
    for d in range(docs.rows):
        i, v = docs.row(d)
        X[ids[d], i] = v.astype(np.float64)
    e = ix.exact_topk(qs.indptr, qs.indices, qs.values, k=7)
    for r in range(qs.rows):
        q = np.zeros(n)
        i, v = qs.row(r)
        q[i] = v.astype(np.float64)
        s = X @ q
        order = np.lexsort((np.arange(s.size), -s))[:7]
        assert list(e["ids"][r]) == list(order)
        np.testing.assert_allclose(e["scores"][r], s[order], rtol=1e-12, atol=1e-12)


def test_linscan_equals_bruteforce():
    """Alg. 2 (LinScan) is exact: its top-k equals brute-force MIPS."""
    ix, docs, ids = _random_index(400, 8, 1, 500, 25, seed=71)
    qs = _random_queries(400, 25, 12, seed=12)
    a = ix.linscan_topk(qs.indptr, qs.indices, qs.values, k=10)
    b = ix.exact_topk(qs.indptr, qs.indices, qs.values, k=10)
    assert np.array_equal(a["ids"], b["ids"])
    np.testing.assert_allclose(a["scores"], b["scores"], rtol=1e-12, atol=1e-12)


def test_find_largest_matches_library_sort():
    """Alg. 3 returns the k largest values; with ties broken toward smaller
    index it matches numpy's lexicographic sort."""
    rng = np.random.default_rng(0)
    for trial in range(20):
        v = rng.integers(-5, 5, size=rng.integers(1, 300)).astype(np.float64)
        k = int(rng.integers(1, 40))
        keys, vals = oracle.find_largest(v, k)
        order = np.lexsort((np.arange(v.size), -v))[:k]
        assert list(keys) == list(order)
        assert list(vals) == list(v[order])


# ------------------------------------------------------------ statistics

def _table_mc(m, h, dist, rng, n=24000, docs=1500):
    p = 120 / n
    ix = oracle.OracleIndex(n, m, h, seed=0x5151 + 10 * m + h)
    act = rng.random((docs, n)) < p
    rows = [np.nonzero(a)[0] for a in act]
    ip = np.zeros(docs + 1, np.uint64)
    ip[1:] = np.cumsum([r.size for r in rows])
    idx = np.concatenate(rows).astype(np.uint32)
    if dist == "uniform":
        v = rng.uniform(-1, 1, idx.size)
    elif dist == "gauss01":
        v = rng.normal(0, 0.1, idx.size)
    else:  # Gaussian(0,1) truncated to [-1, 1]
        v = rng.normal(0, 1, 3 * idx.size)
        v = v[np.abs(v) <= 1][: idx.size]
    v = v.astype(np.float32)
    ids = ix.insert(ip, idx, v)
    tab = ix.hash_table()
    err = []
    for d in range(docs):
        u, _ = ix.sketch_column(int(ids[d]))
        a, b = int(ip[d]), int(ip[d + 1])
        err.append(u[tab[idx[a:b]]].min(axis=1) - v[a:b].astype(np.float64))
    e = np.concatenate(err)
    return (e > 0).mean(), e.mean()


@pytest.mark.slow
def test_tables_1_and_2_by_monte_carlo():
    """Monte Carlo of the oracle's sketch under the paper's probabilistic model
    (each of n coordinates active with p, n*p = 120) reproduces Table 1
    (P[error]) and Table 2 (E[error]) to the printed two decimals (+-0.015)."""
    with open(os.path.join(GOLD, "sketch_error_tables.json")) as f:
        g = json.load(f)
    rng = np.random.default_rng(2024)
    for dist, t2key in (("uniform", "uniform"), ("gauss01", "gauss01"),
                        ("gauss1t", "gauss1_truncated")):
        t1 = g["table1_prob_error"]["uniform" if dist == "uniform" else "gauss01"]
        t2 = g["table2_expected_error"][t2key]
        for a, m in enumerate(g["m"]):
            for b, h in enumerate(g["h"]):
                pe, ee = _table_mc(m, h, dist, rng)
                assert abs(pe - t1[a][b]) <= 0.015, (dist, m, h, pe)
                assert abs(ee - t2[a][b]) <= 0.015, (dist, m, h, ee)


def test_error_probability_closed_form_tiny_workload():
    """Tiny workload (n=1000, psi=32 distinct uniform coordinates, m=64, h=1):
    with continuous values a coordinate's upper decode is exact iff it is the
    largest of its bin-mates, so P[err] = 1 - E[1/(1+T)] with T hypergeometric
    given the bin sizes; with equal bins this is 1 - (m/psi)(1-(1-1/m)^psi) =
    0.2083 (the finite-sample form of Thm. 2's error probability)."""
    from scipy import stats
    n, m, psi = 1000, 64, 32
    w = synth.WORKLOADS["tiny"]
    docs = synth.make_docs(w, n_docs=6000)
    ix = oracle.OracleIndex(n, m, 1)
    ids = ix.insert(docs.indptr, docs.indices, docs.values)
    tab = ix.hash_table()[:, 0]
    err = []
    for d in range(docs.rows):
        u, _ = ix.sketch_column(int(ids[d]))
        i, v = docs.row(d)
        err.append(u[tab[i]] > v.astype(np.float64))
    mc = np.concatenate(err).mean()
    sizes = np.bincount(tab, minlength=m)
    t = np.arange(psi)
    expect = 0.0
    for s in sizes:
        if s == 0:
            continue
        pmf = stats.hypergeom.pmf(t, n - 1, s - 1, psi - 1)
        expect += (s / n) * (1 - (pmf / (1 + t)).sum())
    assert abs(mc - expect) < 0.005
    assert abs(expect - (1 - (m / psi) * (1 - (1 - 1 / m) ** psi))) < 0.01
    assert abs(1 - (m / psi) * (1 - (1 - 1 / m) ** psi) - 0.2083) < 1e-4


# ----------------------------------------------------------- streaming

def test_delete_reuse_and_stale_columns():
    """Sec. 4.3: deletion removes the id from every list, leaves its sketch
    column in place, and frees the id for the next insert (smallest first);
    a reused id carries none of the old vector's postings."""
    ix, docs, ids = _random_index(200, 8, 2, 50, 12, seed=81)
    before_u, before_l = ix.sketch_column(7)
    ix.delete([7, 3, 30])
    assert not ix.is_live(7) and ix.live_count == 47
    u, l = ix.sketch_column(7)
    assert np.array_equal(u, before_u) and np.array_equal(l, before_l)
    for j in range(200):
        lst = ix.inverted_list(j)
        assert not set(lst) & {3, 7, 30}
        assert list(lst) == sorted(lst)
    # the next inserts take 3, 7, 30 in that order, then fresh ids
    new = _random_queries(200, 5, 9, seed=99)  # any vectors will do
    got = ix.insert(new.indptr, new.indices, new.values)
    assert list(got) == [3, 7, 30, 50, 51]
    i, v = new.row(1)
    u, l = ix.sketch_column(7)
    for j in range(200):
        assert (7 in set(ix.inverted_list(j))) == (j in set(i.tolist()))
    # and a fresh build of the surviving vectors gives the same scores
    fresh = oracle.OracleIndex(200, 8, 2, seed=81)
    live = ix.live_ids()
    rows = [ix.doc(int(t)) for t in live]
    fresh.insert(*_csr([(r[0], r[1].astype(np.float32)) for r in rows]))
    qs = _random_queries(200, 8, 10, seed=5)
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        np.testing.assert_array_equal(ix.scores(qi, qv)[live], fresh.scores(qi, qv))


def test_deleted_ids_never_returned():
    ix, docs, ids = _random_index(100, 8, 1, 40, 10, seed=91)
    gone = [0, 5, 6, 39]
    ix.delete(gone)
    qs = _random_queries(100, 10, 5, seed=3)
    r = ix.search(qs.indptr, qs.indices, qs.values, k=36, k_prime=40, candidates=True)
    assert not set(r["ids"].ravel()) & set(gone)
    assert np.all(r["count"] == 36)
    assert not set(r["cand_ids"].ravel()) & set(gone)


def test_empty_query_returns_lowest_ids():
    """An empty query scores every live document 0 (Alg. 6 visits nothing);
    FindLargest over equal scores keeps the smallest ids."""
    ix, docs, ids = _random_index(100, 8, 1, 30, 10, seed=5)
    ix.delete([0, 2])
    ip = np.zeros(2, np.uint64)
    r = ix.search(ip, np.zeros(0, np.uint32), np.zeros(0, np.float32), k=3, k_prime=5)
    assert list(r["ids"][0]) == [1, 3, 4]
    assert list(r["scores"][0]) == [0.0, 0.0, 0.0]


def test_fewer_live_docs_than_k_pads():
    ix, docs, ids = _random_index(50, 8, 1, 4, 5, seed=5)
    qs = _random_queries(50, 1, 5, seed=1)
    r = ix.search(qs.indptr, qs.indices, qs.values, k=6, k_prime=6)
    assert r["count"][0] == 4
    assert list(r["ids"][0][4:]) == [0xFFFFFFFF] * 2
    assert np.all(np.isneginf(r["scores"][0][4:]))


def test_zero_entries_are_not_indexed():
    """nz(x) holds the coordinates with x[j] != 0 (Alg. 5)."""
    ix = oracle.OracleIndex(10, 4, 1, table=np.arange(10) % 4)
    ix.insert(*_csr([([1, 2, 5], [1.0, 0.0, -0.0])]))
    assert list(ix.inverted_list(1)) == [0]
    assert list(ix.inverted_list(2)) == [] and list(ix.inverted_list(5)) == []
    u, l = ix.sketch_column(0)
    assert list(u) == [-np.inf, 1.0, -np.inf, -np.inf]


def test_invalid_inputs_leave_index_unchanged():
    ix = oracle.OracleIndex(10, 4, 1)
    ix.insert(*_csr([([1, 2], [1.0, 2.0])]))
    bad = [([3, 3], [1.0, 1.0]), ([4, 2], [1.0, 1.0]), ([10], [1.0]), ([1], [np.nan]),
           ([1], [np.inf])]
    for b in bad:
        with pytest.raises(oracle.OracleError) as e:
            ix.insert(*_csr([([0], [1.0]), b]))
        assert e.value.code == oracle.EINVAL
    assert ix.live_count == 1 and ix.n_slots == 1
    with pytest.raises(oracle.OracleError) as e:
        ix.delete([1])
    assert e.value.code == oracle.ENOTFOUND
    ix.insert(*_csr([([3], [1.0])]))
    with pytest.raises(oracle.OracleError) as e:
        ix.delete([0, 0])
    assert e.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError):
        ix.search(*_csr([([1], [1.0])]), k=2, k_prime=1)
    assert ix.live_count == 2


# ----------------------------------------------------------------- anytime

def test_worked_example_anytime_budget():
    """Alg. 6's break "if time budget T exhausted", with T counted in postings:
    hand-worked partial scores after each term of the worked example."""
    g = _gold()
    c = g["cases"][0]
    ix = oracle.OracleIndex(g["n"], g["m"], c["h"], table=np.array(c["table"]))
    ix.insert(*_csr([(d["idx"], d["val"]) for d in c["docs"]]))
    q = c["query"]
    for case in c["anytime"]["cases"]:
        assert list(ix.scores(q["idx"], q["val"], budget=case["budget"])) == case["scores"]
    qc = _csr([(q["idx"], q["val"])])
    for s in c["anytime"]["search"]:
        r = ix.search(*qc, k=s["k"], k_prime=s["k_prime"], budget=s["budget"])
        assert list(r["ids"][0]) == s["ids"] and list(r["scores"][0]) == s["scores"]


@pytest.mark.parametrize("h", [1, 2])
def test_anytime_scores_bound_the_processed_coordinates(h):
    """With a budget the scores are upper bounds of the inner product over the
    coordinates processed (Sec. 4.2's remark on the anytime variant), and the
    processed coordinates are a prefix of Alg. 6's order chosen by the
    budget; budget 0 is T = infinity."""
    ix, docs, ids = _random_index(300, 16, h, 400, 24, seed=21 + h)
    qs = _random_queries(300, 20, 12, seed=7)
    lens = np.array([ix.inverted_list(j).size for j in range(300)])
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        keep = qv != 0
        qi, qv = qi[keep], qv[keep]
        order = np.lexsort((qi, -np.abs(qv.astype(np.float64))))
        cum = np.cumsum(lens[qi[order]])
        for budget in (1, int(cum[len(cum) // 2]), int(cum[-1]) + 1):
            t = min(int(np.searchsorted(cum, budget)) + 1, len(cum))
            sel = np.sort(order[:t])  # coordinates ascending, as CSR wants
            a = ix.scores(qi, qv, budget=budget)
            a_prefix = ix.scores(qi[sel], qv[sel])       # same terms, T = infinity
            np.testing.assert_array_equal(a, a_prefix)
            e = ix.exact_scores(qi[sel], qv[sel])
            assert np.all(a >= e - 1e-12 * (1 + np.abs(e)))
        np.testing.assert_array_equal(ix.scores(qi, qv, budget=0), ix.scores(qi, qv))


# -------------------------------------------------------- bfloat16 sketch

def test_bf16_sketch_hand_values():
    """bfloat16 bins (Sec. 4.1 notes), U rounded up and L rounded down:
    1 + 2^-20 lies between the bfloat16 neighbours 1 and 1 + 2^-7."""
    x = np.float32(1.0 + 2.0 ** -20)
    tab = np.array([[0], [0], [1]], np.uint32)                  # n = 3, m = 2
    ix = oracle.OracleIndex(3, 2, 1, table=tab, sketch_bf16=True)
    ix.insert(*_csr([([0, 2], [x, 3.0]), ([0, 1], [-x, 0.5]), ([2], [-0.1])]))
    u, l = ix.sketch_column(0)
    assert list(u) == [1.0078125, 3.0] and list(l) == [1.0, 3.0]
    u, l = ix.sketch_column(1)                                  # bin 0: {-x, 0.5}
    assert list(u) == [0.5, -np.inf] and list(l) == [-1.0078125, np.inf]
    u, l = ix.sketch_column(2)                                  # -0.1 in bin 1
    f = np.float32(-0.1).view(np.uint32)
    lo = np.uint32((f & 0xFFFF0000) + 0x10000).view(np.float32)  # away from zero
    hi = np.uint32(f & 0xFFFF0000).view(np.float32)               # toward zero
    assert u[1] == hi and l[1] == lo and lo < -0.1 < hi
    # scores read the rounded bins: q = (1, 0, 1) on doc 0 -> u_0 + u_1
    assert ix.scores([0, 2], [1.0, 1.0])[0] == 1.0078125 + 3.0


@pytest.mark.parametrize("h", [1, 2])
def test_bf16_sketch_is_the_directed_rounding_and_keeps_theorem1(h):
    """Each bin is the fp32 bin rounded to bfloat16 in its direction: a
    bfloat16 value on the right side with no bfloat16 value in between; and
    the scores stay upper bounds of the inner products."""
    full, docs, ids = _random_index(300, 16, h, 200, 24, seed=31 + h)
    bf = oracle.OracleIndex(300, 16, h, seed=31 + h, sketch_bf16=True)
    bf.insert(docs.indptr, docs.indices, docs.values)
    for i in range(0, 200, 7):
        for a, b, up in zip(full.sketch_column(i), bf.sketch_column(i), (True, False)):
            fin = np.isfinite(a)
            assert np.array_equal(a[~fin], b[~fin])
            a32, b32 = a[fin].astype(np.float32), b[fin].astype(np.float32)
            assert np.all(b32.view(np.uint32) & 0xFFFF == 0)        # representable
            assert np.all(b32 >= a32) if up else np.all(b32 <= a32)
            # the next bfloat16 toward a is past a
            bits = b32.view(np.uint32).astype(np.int64)
            step = np.where((b32 > 0) == up, -0x10000, 0x10000)
            nb = (bits + step).astype(np.uint32).view(np.float32)
            moved = b32 != a32
            assert np.all((nb[moved] < a32[moved]) if up else (nb[moved] > a32[moved]))
    qs = _random_queries(300, 20, 12, seed=8)
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        a, e = bf.scores(qi, qv), bf.exact_scores(qi, qv)
        assert np.all(a >= e - 1e-12 * (1 + np.abs(e)))
