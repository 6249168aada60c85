"""The parity checkers themselves (no GPU): each accepts a correct result,
accepts a reordering inside the stated tie band, and rejects each planted
mistake a kernel could make (a score off by more than 1e-5 of its
magnitude, a wrong id outside the band, a missing or duplicated id, an
unsorted or badly padded output, a vacant slot with a finite score)."""
import numpy as np
import pytest

from tests import parity


def _scores(n=40, seed=0):
    rng = np.random.default_rng(seed)
    ref = rng.standard_normal(n) * 10.0
    mag = np.abs(ref) + rng.random(n) * 5.0 + 1.0
    return ref, mag


def test_score_close_is_the_relative_band():
    mag = np.array([100.0, 100.0, 100.0])
    ref = np.array([1.0, 1.0, 1.0])
    got = parity.score_close(np.array([1.0 + 0.9e-3, 1.0 - 0.9e-3, 1.0 + 1.1e-3]), ref, mag)
    assert got.tolist() == [True, True, False]
    # a zero magnitude (empty sum) allows no difference beyond the floor
    assert parity.score_close(0.0, 0.0, 0.0) and not parity.score_close(1e-20, 0.0, 0.0)


def test_dense_scores_accept_and_reject():
    ref, mag = _scores()
    live = np.ones(ref.size, bool)
    live[[3, 17]] = False
    gpu = ref.astype(np.float32).astype(np.float64)
    gpu[~live] = -np.inf
    parity.check_dense_scores(gpu, ref, mag, live)
    off = gpu.copy()
    off[5] += 2.0 * parity.REL * mag[5]                # outside the band
    with pytest.raises(AssertionError):
        parity.check_dense_scores(off, ref, mag, live)
    vacant = gpu.copy()
    vacant[3] = 0.0                                    # a vacant slot scored
    with pytest.raises(AssertionError):
        parity.check_dense_scores(vacant, ref, mag, live)


def _top(ref, kq):
    return np.array(sorted(range(ref.size), key=lambda i: (-ref[i], i))[:kq])


def test_candidate_set_tie_band():
    ref, mag = _scores(seed=1)
    kq = 10
    ora = _top(ref, kq)
    assert parity.check_candidate_set(ora[::-1], ora, ref, mag, kq) == 0  # order is free
    # the (kq+1)-th id moved into the band of the boundary: a swap is allowed
    nxt = _top(ref, kq + 1)[-1]
    tied = ref.copy()
    tied[nxt] = ref[ora[-1]] - 0.5 * parity.REL * mag[ora[-1]]
    swapped = np.concatenate([ora[:-1], [nxt]])
    assert parity.check_candidate_set(swapped, ora, tied, mag, kq) == 2
    # the same swap with the scores apart is a wrong candidate set
    with pytest.raises(AssertionError):
        parity.check_candidate_set(swapped, ora, ref, mag, kq)
    # a duplicated id leaves kq - 1 distinct candidates
    dup = ora.copy()
    dup[0] = dup[1]
    with pytest.raises(AssertionError):
        parity.check_candidate_set(dup, ora, ref, mag, kq)


def _padded(ids, scores, width):
    out_i = np.full(width, 0xFFFFFFFF, np.uint32)
    out_s = np.full(width, -np.inf, np.float32)
    out_i[:len(ids)] = ids
    out_s[:len(scores)] = scores
    return out_i, out_s


def test_topk_accepts_the_exact_answer_and_rejects_mistakes():
    exact, mag = _scores(seed=2)
    cand = _top(exact, 20)
    k = 10
    best = cand[:k]
    ids, sc = _padded(best, exact[best].astype(np.float32), 12)
    parity.check_topk(ids, sc, cand, exact, mag, k)

    wrong = best.copy()
    wrong[-1] = cand[k + 3]                            # a worse candidate, outside the band
    i2, s2 = _padded(wrong, exact[wrong].astype(np.float32), 12)
    order = np.argsort(-s2[:k], kind="stable")
    i2[:k], s2[:k] = i2[:k][order], s2[:k][order]
    with pytest.raises(AssertionError):
        parity.check_topk(i2, s2, cand, exact, mag, k)

    bad_score = sc.copy()
    bad_score[4] += np.float32(3.0 * parity.REL * mag[best[4]])
    with pytest.raises(AssertionError):
        parity.check_topk(ids, bad_score, cand, exact, mag, k)

    unsorted_i, unsorted_s = ids.copy(), sc.copy()
    unsorted_i[[0, 1]], unsorted_s[[0, 1]] = unsorted_i[[1, 0]], unsorted_s[[1, 0]]
    with pytest.raises(AssertionError):
        parity.check_topk(unsorted_i, unsorted_s, cand, exact, mag, k)

    bad_pad = ids.copy()
    bad_pad[k] = 7                                     # padding must be the all-ones id
    with pytest.raises(AssertionError):
        parity.check_topk(bad_pad, sc, cand, exact, mag, k)


def test_topk_swap_inside_the_band_is_accepted():
    exact, mag = _scores(seed=3)
    cand = _top(exact, 20)
    k = 10
    tied = exact.copy()
    tied[cand[k]] = exact[cand[k - 1]] - 0.5 * parity.REL * mag[cand[k - 1]]
    got = np.concatenate([cand[:k - 1], [cand[k]]])
    ids, sc = _padded(got, tied[got].astype(np.float32), k)
    parity.check_topk(ids, sc, cand, tied, mag, k)


def test_topk_with_fewer_candidates_than_k():
    exact, mag = _scores(seed=4)
    cand = _top(exact, 4)
    ids, sc = _padded(cand, exact[cand].astype(np.float32), 10)
    parity.check_topk(ids, sc, cand, exact, mag, 10)
