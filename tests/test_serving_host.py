"""Host-side parts of the serving loop (no GPU): the request stream, the
live-id list that delete requests pick from, and the CSR row gathering that
feeds inserts and query batches."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2301_10622_gb300 import serving, synth  # noqa: E402


def test_poisson_stream_rates_order_and_seed():
    rates = {"insert": 2000.0, "delete": 300.0, "query": 1200.0}
    a = serving.poisson_stream(2.0, rates, 500, 40, seed=9)
    b = serving.poisson_stream(2.0, rates, 500, 40, seed=9)
    assert [(r.t, r.kind, r.row, r.u) for r in a] == [(r.t, r.kind, r.row, r.u) for r in b]
    t = np.array([r.t for r in a])
    assert np.all(np.diff(t) >= 0) and t.min() >= 0 and t.max() <= 2.0
    for kind, rate in rates.items():
        n = sum(r.kind == kind for r in a)
        # Poisson count: mean rate*T, sd sqrt(rate*T); 5 sd
        assert abs(n - rate * 2.0) <= 5 * np.sqrt(rate * 2.0), (kind, n)
    ins = [r.row for r in a if r.kind == "insert"]
    assert ins == [i % 500 for i in range(len(ins))]          # the pool in order
    q = np.array([r.row for r in a if r.kind == "query"])
    assert q.min() >= 0 and q.max() < 40
    u = np.array([r.u for r in a if r.kind == "delete"])
    assert np.all((u >= 0) & (u < 1))
    # exponential gaps within one kind (a Poisson process): mean 1/rate
    tq = np.array([r.t for r in a if r.kind == "query"])
    assert abs(np.diff(tq).mean() * 1200.0 - 1.0) < 0.15


def test_live_list_picks_uniformly_and_deterministically():
    live = serving.LiveList(range(10))
    assert live.take(0.0) == 0 and len(live) == 9
    assert live.take(0.999) == 8            # last entry (9 moved into slot 0)
    live.add([100, 101])
    assert sorted(live.a) == [1, 2, 3, 4, 5, 6, 7, 9, 100, 101]
    rng = np.random.default_rng(0)
    counts = np.zeros(50)
    for _ in range(20000):
        ll = serving.LiveList(range(50))
        counts[ll.take(float(rng.random()))] += 1
    # chi-square against uniform over 50 ids (49 dof; 99.9% point ~ 86)
    chi2 = ((counts - 400.0) ** 2 / 400.0).sum()
    assert chi2 < 86, chi2
    a, b = serving.LiveList(range(30)), serving.LiveList(range(30))
    us = rng.random(30)
    assert [a.take(x) for x in us] == [b.take(x) for x in us]
    assert len(a) == 0


def test_csr_rows_gathers_the_rows():
    w = synth.scaled(synth.WORKLOADS["text"], 300, n=500)
    docs = synth.make_docs(w)
    rows = [5, 0, 299, 5, 17]
    ip, idx, val = serving.csr_rows(docs, rows)
    want = docs.take(rows)
    assert np.array_equal(ip, want.indptr.astype(np.int64))
    assert np.array_equal(idx, want.indices.astype(np.int32))
    assert np.array_equal(val, want.values)
    ip0, idx0, val0 = serving.csr_rows(docs, [])
    assert ip0.tolist() == [0] and idx0.size == 0 and val0.size == 0
