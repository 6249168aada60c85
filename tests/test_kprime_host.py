"""The k' labels' arithmetic (no GPU): from a batch of candidate lists and
exact top-k lists, kprime.labels_from gives the approximate rank of the
keep-th found exact id and certifies the top-k exactly when Thm. 1 allows it
(every live id a candidate, or the k-th exact score at or above the last
candidate's approximate score).  Checked against a plain loop on random
batches with ties, missing ids, padding and garbage beyond each count.
The margin calibration's order (negative margins first, the least margin
whose held-out recall reaches the target) against a stand-in index."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2301_10622_gb300 import kprime  # noqa: E402


def _brute(cid, cs, cnt, ids, sc, cap, k, keep):
    kp, cert = [], []
    for r in range(cid.shape[0]):
        n = int(cnt[r])
        cand = sorted(zip(cs[r][:n].tolist(), cid[r][:n].tolist()), key=lambda t: (-t[0], t[1]))
        rank_of = {i: p + 1 for p, (_, i) in enumerate(cand)}
        ranks = sorted(rank_of.get(int(i), cap + 1) if i >= 0 else cap + 1 for i in ids[r])
        tau = cand[-1][0] if n else 0.0
        ok = n < cap or float(sc[r][k - 1]) >= tau
        cert.append(ok)
        kp.append(min(ranks[keep - 1], cap) if ok else cap)
    return np.array(kp), np.array(cert)


@pytest.mark.parametrize("seed", range(6))
def test_labels_equal_the_plain_definition(seed):
    rng = np.random.default_rng(seed)
    nq, cap, k, keep = 24, 40, 10, 9
    cid = np.full((nq, cap), 7777, np.int32)          # garbage beyond each count
    cs = rng.standard_normal((nq, cap)).astype(np.float32) * 100
    cnt = rng.integers(0, cap + 1, nq).astype(np.int32)
    cnt[:4] = cap                                      # some full lists
    ids = np.full((nq, k), -1, np.int32)
    sc = np.full((nq, k), -np.inf, np.float32)
    for r in range(nq):
        n = int(cnt[r])
        pool = rng.choice(1000, size=n + 15, replace=False)
        cid[r, :n] = pool[:n]
        cs[r, :n] = np.round(rng.standard_normal(n), 1)   # ties on the score
        # the exact top-k: mostly candidates, some outside, some padding
        m = min(k, int(rng.integers(0, k + 1)))
        picks = [int(x) for x in rng.choice(pool, size=m, replace=False)]
        ids[r, :m] = picks
        sc[r, :m] = np.sort(rng.standard_normal(m) + rng.choice([-1.0, 2.0]))[::-1]
    want_kp, want_cert = _brute(cid, cs, cnt, ids, sc, cap, k, keep)
    kp, cert = kprime.labels_from(torch.from_numpy(cid), torch.from_numpy(cs),
                                  torch.from_numpy(cnt), torch.from_numpy(ids),
                                  torch.from_numpy(sc), cap, k, keep)
    assert np.array_equal(cert.numpy(), want_cert)
    assert np.array_equal(kp.numpy(), want_kp)


def test_labels_by_hand():
    """Candidates 5 (0.9), 3 (0.9), 8 (0.5), 1 (0.2): ranks 3->1, 5->2, 8->3,
    1->4 (equal scores by id).  Exact top-2 {8, 3} with keep = 2: k' = 3.
    With the list full (4 candidates of cap 4), the 2nd exact score 0.3 is at
    or above the last candidate's 0.2, so the top-2 is certified; at 0.1 it
    is not, and k' falls back to the cap.  With room left (cap 6) every live
    id is a candidate, so it is certified whatever the scores."""
    cid = torch.tensor([[5, 3, 8, 1]], dtype=torch.int32)
    cs = torch.tensor([[0.9, 0.9, 0.5, 0.2]])
    cnt = torch.tensor([4], dtype=torch.int32)
    ids = torch.tensor([[8, 3]], dtype=torch.int32)
    kp, cert = kprime.labels_from(cid, cs, cnt, ids, torch.tensor([[0.7, 0.3]]), 4, 2, 2)
    assert kp.tolist() == [3] and cert.tolist() == [True]
    kp, cert = kprime.labels_from(cid, cs, cnt, ids, torch.tensor([[0.7, 0.1]]), 4, 2, 2)
    assert kp.tolist() == [4] and cert.tolist() == [False]
    cid6 = torch.tensor([[5, 3, 8, 1, 0, 0]], dtype=torch.int32)
    cs6 = torch.tensor([[0.9, 0.9, 0.5, 0.2, 9.0, 9.0]])  # garbage beyond the count
    kp, cert = kprime.labels_from(cid6, cs6, cnt, ids, torch.tensor([[0.7, 0.1]]), 6, 2, 2)
    assert kp.tolist() == [3] and cert.tolist() == [True]


class _FakeNet:
    """A network stand-in: keeps the policy kprime.calibrate_margin sets."""

    def __init__(self):
        self.pol = {"shifts": [0, 1], "posting_cost": 0.001, "margin": 0.0}
        self.set_calls = []

    def policy(self):
        return dict(self.pol)

    def set_policy(self, shifts, posting_cost, margin):
        self.pol = {"shifts": list(shifts), "posting_cost": posting_cost, "margin": margin}
        self.set_calls.append(margin)


class _FakeIndex:
    """Answers a learned search with the exact top 10 for the first
    round(recall(margin) * rows) queries and misses them all for the rest."""

    def __init__(self, exact, recall_of):
        self.exact, self.recall_of, self.net = exact, recall_of, None

    def search_learned(self, net, ip, ii, v, k, kp_min, kp_max):
        self.net = net
        rows = self.exact.shape[0]
        good = int(round(self.recall_of(net.pol["margin"]) * rows))
        ids = np.where(np.arange(rows)[:, None] < good, self.exact, self.exact + 1000)
        return torch.from_numpy(ids), None, None

    def sync(self):
        pass


class _Q:
    def __init__(self, rows):
        self.indptr = np.arange(rows + 1, dtype=np.int64)
        self.indices = np.zeros(rows, np.int32)
        self.values = np.ones(rows, np.float32)


def test_calibration_takes_the_least_margin_reaching_the_target():
    rows = 200
    exact = np.arange(rows * 10, dtype=np.int64).reshape(rows, 10)
    # recall rises with the margin: 0.80 at -2, +0.05 per 1/4 of log2 k'
    rec = lambda mg: min(1.0, 0.80 + 0.2 * (mg + 2.0))  # noqa: E731
    net, curve = _FakeNet(), []
    ix = _FakeIndex(exact, rec)
    mg, r = kprime.calibrate_margin(ix, net, _Q(rows), exact, target=0.92, curve=curve)
    assert mg == -1.25 and r == pytest.approx(0.95)
    assert net.pol["margin"] == -1.25                    # left set on the policy
    assert net.pol["shifts"] == [0, 1] and net.pol["posting_cost"] == 0.001
    assert [m for m, _ in curve] == [-2.0, -1.5, -1.25]  # increasing, stops at the first
    assert curve[0][1] == pytest.approx(0.80) and curve[1][1] == pytest.approx(0.90)


def test_calibration_ends_at_the_largest_margin_when_the_target_is_out_of_reach():
    rows = 50
    exact = np.arange(rows * 10, dtype=np.int64).reshape(rows, 10)
    net, curve = _FakeNet(), []
    mg, r = kprime.calibrate_margin(_FakeIndex(exact, lambda mg: 0.5), net, _Q(rows), exact,
                                    target=0.92, margins=(1.0, -1.0, 0.0), curve=curve)
    assert mg == 1.0 and r == pytest.approx(0.5)
    assert [m for m, _ in curve] == [-1.0, 0.0, 1.0]
