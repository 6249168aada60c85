"""Helpers that compare the CUDA path with the CPU oracle (test code only).

Tolerances follow the stated bar: an fp32 score s_gpu of a sum whose terms
have absolute values summing to M must satisfy |s_gpu - s_fp64| <= 1e-5 * M
(the accumulated rounding of fp32 is far below that: about psi * 2^-24 * M).
Where fp32 rounding may reorder two ids, the comparison accepts the swap only
when the ids' fp64 scores lie within that band of the boundary.
"""
from __future__ import annotations

import numpy as np

REL = 1e-5
TINY = 1e-30


def score_close(s_gpu, s_ref, mag):
    s_gpu = np.asarray(s_gpu, np.float64)
    return np.abs(s_gpu - s_ref) <= REL * np.maximum(mag, TINY) + 1e-35


def check_dense_scores(gpu, ref, mag, live):
    """gpu: fp32 scores over slots; ref/mag: oracle fp64 over slots."""
    g = np.asarray(gpu, np.float64)[: ref.size]
    assert np.all(np.isneginf(g[~live])), "non-live slots must score -inf"
    ok = score_close(g[live], ref[live], mag[live])
    bad = np.nonzero(~ok)[0]
    assert ok.all(), f"{bad.size} scores off, e.g. slot {np.nonzero(live)[0][bad[:5]]}"


def check_candidate_set(gpu_ids, ora_ids, ref_scores, mag, kq):
    """Candidate sets (Alg. 7) equal except inside the tie band around
    the k'-th approximate score."""
    g = set(int(x) for x in np.asarray(gpu_ids)[:kq])
    o = set(int(x) for x in np.asarray(ora_ids)[:kq])
    assert len(g) == kq, f"expected {kq} distinct candidates, got {len(g)}"
    if g == o:
        return 0
    # boundary score: k'-th best oracle score
    order = sorted(o, key=lambda i: (-ref_scores[i], i))
    b = order[-1]
    tau, mb = ref_scores[b], mag[b]
    for i in g ^ o:
        band = 2 * REL * max(mag[i], mb, TINY)
        assert abs(ref_scores[i] - tau) <= band, (
            f"id {i} differs outside the tie band: {ref_scores[i]} vs boundary {tau}")
    return len(g ^ o)


def check_topk(gpu_ids, gpu_scores, cand_ids, exact, exact_mag, k):
    """Top-k after re-rank: the GPU's k ids must be the best k of its own
    candidate set by fp64 exact score (ids may swap only within the band), and
    each returned score must be the exact score within tolerance."""
    cand = [int(c) for c in cand_ids]
    r = min(k, len(cand))
    best = sorted(cand, key=lambda i: (-exact[i], i))[:r]
    gi = [int(x) for x in np.asarray(gpu_ids)[:r]]
    gs = np.asarray(gpu_scores, np.float64)[:r]
    assert len(set(gi)) == r
    for i, s in zip(gi, gs):
        assert score_close(s, exact[i], exact_mag[i]), (i, s, exact[i])
    if gi != best:
        tau = exact[best[-1]]
        mb = exact_mag[best[-1]]
        for i in set(gi) ^ set(best):
            assert abs(exact[i] - tau) <= 2 * REL * max(exact_mag[i], mb, TINY), (i, exact[i], tau)
        # within the returned list, order must follow the fp32 scores
    assert np.all(np.diff(gs) <= 0), "scores must be non-increasing"
    pad_ids = np.asarray(gpu_ids)[r:]
    assert np.all(pad_ids.astype(np.int64) & 0xFFFFFFFF == 0xFFFFFFFF)
    assert np.all(np.isneginf(np.asarray(gpu_scores)[r:]))


