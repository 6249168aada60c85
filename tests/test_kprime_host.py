"""The k' labels' arithmetic (no GPU): from a batch of candidate lists and
exact top-k lists, kprime.labels_from gives the approximate rank of the
keep-th found exact id and certifies the top-k exactly when Thm. 1 allows it
(every live id a candidate, or the k-th exact score at or above the last
candidate's approximate score).  Checked against a plain loop on random
batches with ties, missing ids, padding and garbage beyond each count."""
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
