"""Reference of the learned budget-level choice (test infrastructure only).

Alg. 6 may stop scoring once a time budget is spent (its anytime break), and
Alg. 7 can make up for a short budget with a deeper re-rank.  The library's
policy picks, per query, one of a few budget levels and a k' from a
network's predictions; this module restates that choice from its definition
so the CUDA kernel can be checked against it:

  level l keeps ceil(P_q / 2^shift[l]) postings of the query's P_q (the whole
  query when shift[l] = 0, budget 0 = no break); it needs
  k'_l = max(ceil(2^v), kp_min) with v = clamp(y_l + margin, 0, 31), and is
  feasible when ceil(2^v) <= kp_max; among feasible levels the least
  posting_cost * postings + k'_l wins, ties going to the earlier level; with
  none feasible, level 0 at kp_max.

The integer decisions (ceil, the comparisons) are taken in the precision the
kernel takes them in: v and 2^v in float32, the cost as the float32 rounding
of the exact posting_cost * float32(postings) + k'_l (the kernel's fused
multiply-add).
"""
from __future__ import annotations

import numpy as np


def level_budget(P: int, shift: int) -> int:
    """ceil(P / 2^shift) as an integer; the whole query (budget 0) at shift 0."""
    if shift == 0:
        return 0
    return (int(P) + (1 << shift) - 1) >> shift


def level_postings(P: int, shift: int) -> int:
    return int(P) if shift == 0 else level_budget(P, shift)


def choose(y, P, shifts, posting_cost: float, margin: float, kp_min: int, kp_max: int):
    """y: [n_q, L] network outputs (float32), P: [n_q] postings per query.
    Returns (k' int64[n_q], budget int64[n_q], level int64[n_q], cost
    float32[n_q, L] with +inf for infeasible levels)."""
    y = np.asarray(y, np.float32)
    nq, L = y.shape
    assert L == len(shifts)
    kp = np.zeros(nq, np.int64)
    bud = np.zeros(nq, np.int64)
    lev = np.zeros(nq, np.int64)
    costs = np.full((nq, L), np.inf, np.float32)
    pc = np.float32(posting_cost)
    for q in range(nq):
        best, best_cost, best_kp = -1, None, kp_max
        for l, sh in enumerate(shifts):
            v = np.float32(y[q, l]) + np.float32(margin)
            v = np.float32(min(max(v, np.float32(0.0)), np.float32(31.0)))
            need = np.ceil(np.exp2(v, dtype=np.float32))
            if need > np.float32(kp_max):
                continue
            k_l = max(int(need), kp_min)
            b = np.float32(level_postings(int(P[q]), sh))
            c = np.float32(float(pc) * float(b) + float(k_l))
            costs[q, l] = c
            if best < 0 or c < best_cost:
                best, best_cost, best_kp = l, c, k_l
        sh = shifts[best] if best >= 0 else 0
        kp[q] = best_kp
        bud[q] = level_budget(int(P[q]), sh)
        lev[q] = max(best, 0)
    return kp, bud, lev, costs
