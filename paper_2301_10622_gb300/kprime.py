"""Learned per-query k': labels, training and evaluation.

The paper suggests choosing Alg. 7's re-ranking depth k' per query from the
expected sketching error (end of Sec. 5.3; an open question in Sec. 7).  Here
a small network (``sinnamon.MLP``, hand-written CUDA) predicts, from cheap
query features (``sinn_kp_features``), log2 of the smallest k' that still
recovers at least 9 of the exact top 10.

Labels come from the method itself, on the GPU:
  1. ``sinn_candidates(q, K)`` gives the K ids of best approximate score and
     ``sinn_search(q, k=10, k'=K)`` their exact top 10 (Alg. 7).
  2. Thm. 1: an id outside the K candidates has exact score <= approximate
     score <= the K-th approximate score tau_K.  So when the 10th exact score
     found is >= tau_K, those 10 ids are the exact top 10 of the collection.
  3. Each of them has an approximate rank (its place among the candidates by
     score desc, id asc).  k' = 9th smallest rank is the least depth with
     recall@10 >= 0.9.  Uncertified queries get the cap K.
Budget levels (Alg. 6's anytime break, learned together with k'): scoring
can stop once ceil(P_q / 2^s) of the query's P_q postings are visited, and
the re-rank then needs a larger k' to keep 9 of the exact top 10.  For each
level s the label is that least k' under the budgeted scores (step 3 with
``sinn_candidates_kpb``); the network reads the query's features and -s and
predicts log2 of it, and the library's policy takes, per query, the level of
least predicted cost (``sinn_mlp_set_policy``).

Only argument marshalling and bookkeeping (sorting candidates, array
arithmetic) happen here in PyTorch; scores, selection and training run in
the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import sinnamon


def _batches(csr, size):
    for a in range(0, csr.rows, size):
        yield a, csr.slice(a, min(csr.rows, a + size))


def labels(ix: "sinnamon.Index", queries, k: int = 10, cap: int = 20000, keep: int = 9,
           batch: int = 512):
    """Minimal k' per query with recall@k >= keep/k, from the method's own
    scores.  Returns (kprime int64[n], certified bool[n], exact top-k ids)."""
    assert keep <= k
    out_kp = np.zeros(queries.rows, np.int64)
    out_ok = np.zeros(queries.rows, bool)
    out_ids = np.zeros((queries.rows, k), np.int64)
    for a, qs in _batches(queries, batch):
        ids, sc = ix.search(qs.indptr.astype(np.int64), qs.indices.astype(np.int32), qs.values,
                            k=k, k_prime=cap)
        cid, cs, cnt = ix.candidates(qs.indptr.astype(np.int64), qs.indices.astype(np.int32),
                                     qs.values, cap)
        ix.sync()
        nq = qs.rows
        kp, cert = labels_from(cid, cs, cnt, ids, sc, cap, k, keep)
        out_kp[a:a + nq] = kp.cpu().numpy()
        out_ok[a:a + nq] = cert.cpu().numpy()
        out_ids[a:a + nq] = ids.to(torch.int64).cpu().numpy()
    return out_kp, out_ok, out_ids


def labels_from(cid, cs, cnt, ids, sc, cap: int, k: int = 10, keep: int = 9):
    """Steps 2-3 above for a batch: from each query's cnt candidates (ids cid,
    approximate scores cs, rows of length cap) and its exact top-k (ids, sc,
    best first), the least k' with recall >= keep/k and whether the top-k is
    certified exact.  Returns (k' int64[nq], certified bool[nq])."""
    valid = torch.arange(cap, device=cid.device)[None, :] < cnt[:, None].to(torch.int64)
    # tau_K: the smallest approximate score among the candidates
    tau = torch.where(valid, cs, torch.full_like(cs, float("inf"))).min(dim=1).values
    tau = torch.where(cnt > 0, tau, torch.zeros_like(tau))
    rank = exact_ranks(cid, cs, cnt, ids, cap)
    kth = torch.sort(rank, dim=1).values[:, keep - 1]
    tenth = sc[:, k - 1]
    full = cnt.to(torch.int64) < cap                         # every live id is a candidate
    cert = full | (tenth >= tau)
    kp = torch.where(cert, kth.clamp(max=cap), torch.full_like(kth, cap))
    return kp, cert


DEFAULT_SHIFTS = (0, 1, 2, 3, 4, 5)


def exact_ranks(cid, cs, cnt, ids, cap: int):
    """1-based approximate ranks (score desc, id asc) among each query's cnt
    candidates (ids cid, scores cs, rows of length cap) of the given ids
    [nq, k]; cap + 1 where an id is not a candidate."""
    nq = cid.shape[0]
    dev = cid.device
    valid = torch.arange(cap, device=dev)[None, :] < cnt[:, None].to(torch.int64)
    big = 1 << 40
    cid64 = torch.where(valid, cid.to(torch.int64), torch.full_like(cid, 0, dtype=torch.int64) + big)
    cs = torch.where(valid, cs, torch.full_like(cs, -float("inf")))
    o1 = torch.argsort(cid64, dim=1, stable=True)
    s1 = torch.gather(cs, 1, o1)
    o2 = torch.argsort(-s1, dim=1, stable=True)
    order = torch.gather(o1, 1, o2)                      # rank r -> slot
    rank_of_slot = torch.empty_like(order)
    rank_of_slot.scatter_(1, order, torch.arange(1, cap + 1, device=dev).expand(nq, cap))
    sid, sperm = torch.sort(cid64, dim=1)
    ids64 = ids.to(torch.int64)
    pos = torch.searchsorted(sid, ids64).clamp(max=cap - 1)
    found = (torch.gather(sid, 1, pos) == ids64) & (ids64 >= 0)
    rank = torch.gather(rank_of_slot, 1, torch.gather(sperm, 1, pos))
    return torch.where(found, rank, torch.full_like(rank, cap + 1))


def level_labels(ix: "sinnamon.Index", queries, exact_ids, certified, shifts=DEFAULT_SHIFTS,
                 k: int = 10, cap: int = 20000, keep: int = 9, batch: int = 512):
    """Per budget level (scoring stops at ceil(P_q / 2^s) postings), the
    least k' keeping `keep` of the exact top k (the certified ids from
    ``labels``); cap where that is beyond cap candidates or the top k is not
    certified.  Returns int64[n, L]."""
    n = queries.rows
    out = np.full((n, len(shifts)), cap, np.int64)
    for a, qs in _batches(queries, batch):
        ip, ii = qs.indptr.astype(np.int64), qs.indices.astype(np.int32)
        P = ix.query_postings(ip, ii, qs.values)
        ex = torch.from_numpy(exact_ids[a:a + qs.rows]).to(P.device)
        for li, sh in enumerate(shifts):
            bud = torch.zeros_like(P) if sh == 0 else (P + (1 << sh) - 1) >> sh
            cid, cs, cnt = ix.candidates_kpb(ip, ii, qs.values, cap, bud)
            rank = exact_ranks(cid, cs, cnt, ex, cap)
            kth = torch.sort(rank, dim=1).values[:, keep - 1].clamp(max=cap)
            out[a:a + qs.rows, li] = kth.cpu().numpy()
    out[~np.asarray(certified, bool)] = cap
    return out


def level_rows(F: torch.Tensor, shifts) -> torch.Tensor:
    """Network inputs [n * L, 20]: each query's features followed by -s."""
    n, L = F.shape[0], len(shifts)
    lv = -torch.tensor(shifts, dtype=torch.float32, device=F.device)
    X = torch.cat([F.repeat_interleave(L, dim=0), lv.repeat(n)[:, None]], dim=1)
    return X.contiguous()


def train_levels(ix, queries, kp_levels, shifts=DEFAULT_SHIFTS, k: int = 10, tau: float = 0.9,
                 epochs: int = 30, batch: int = 8192, lr: float = 2e-3, seed: int = 7,
                 hidden: int = 256, log=None) -> "sinnamon.MLP":
    """Fit log2 of each level's k' (pinball loss at tau) from the query's
    features and the level; the network is returned without a policy."""
    F = features(ix, queries)
    X = level_rows(F, shifts)
    t = torch.from_numpy(np.log2(np.maximum(kp_levels, k).astype(np.float32)).reshape(-1)).to(X.device)
    return _fit(X, t, tau, epochs, batch, lr, seed, hidden, log)


def _fit(X, t, tau, epochs, batch, lr, seed, hidden, log):
    mean = X.mean(dim=0).cpu().numpy()
    std = X.std(dim=0).clamp(min=1e-6).cpu().numpy()
    mlp = sinnamon.MLP(X.shape[1], hidden, seed=seed, device=X.device)
    mlp.set_normalizer(mean, std)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot = torch.zeros((), device=X.device)
        for a in range(0, n, batch):
            idx = perm[a:a + batch]
            xb, tb = X[idx].contiguous(), t[idx].contiguous()
            loss = mlp.train_step(xb, tb, tau, lr * (0.5 * (1 + math.cos(math.pi * ep / epochs))))
            tot += loss[0] * idx.numel()
        if log:
            log(f"epoch {ep}: pinball loss {float(tot) / n:.4f}")
    mlp.sync()  # raises if a tensor-core GEMM's bounded wait ran out
    return mlp


def measure_costs(ix, queries, k: int = 10, k_prime: int = 1000, reps: int = 3):
    """posting_cost for the policy: the measured time of scoring one posting
    over the time of selecting and re-ranking one candidate, from the
    library's phase timing of a fixed-k' search of `queries`."""
    ip, ii = queries.indptr.astype(np.int64), queries.indices.astype(np.int32)
    P = float(ix.query_postings(ip, ii, queries.values).sum().item())
    ix.search(ip, ii, queries.values, k=k, k_prime=k_prime)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        sinnamon.sinn_timing_start(ix.handle)
        ix.search(ip, ii, queries.values, k=k, k_prime=k_prime)
        torch.cuda.synchronize()
        tm = sinnamon.sinn_timing_stop(ix.handle)["ms"]
        per_post = tm["score"] / max(P, 1.0)
        per_cand = (tm["select"] + tm["rerank"]) / (queries.rows * k_prime)
        c = per_post / max(per_cand, 1e-12)
        best = c if best is None else min(best, c)
    return best


def recall(ids, exact_ids, k: int = 10) -> float:
    ids = ids.cpu().numpy().astype(np.int64) if isinstance(ids, torch.Tensor) else ids
    return float(np.mean([len(set(ids[r][:k]) & set(exact_ids[r][:k])) / k
                          for r in range(ids.shape[0])]))


CAL_MARGINS = (-2.0, -1.5, -1.25, -1.0, -0.875, -0.75, -0.625, -0.5, -0.375, -0.25, -0.125,
               0.0, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0)


def calibrate_margin(ix, mlp, queries, exact_ids, k: int = 10, kp_min: int = 10,
                     kp_max: int = 4096, target: float = 0.92, margins=CAL_MARGINS,
                     curve=None):
    """The least margin (added to every predicted log2 k') at which the
    learned search keeps mean recall@k >= target on held-out queries whose
    exact top k the method certified; sets it on the network's policy.
    Margins are tried in increasing order, negative ones first: the pinball
    fit at tau = 0.9 puts most queries above their label already, so the
    mean recall at margin 0 can sit well above the target.  `curve`, if a
    list, receives each (margin, recall) tried.  Returns (margin, recall)."""
    pol = mlp.policy()
    ip, ii = queries.indptr.astype(np.int64), queries.indices.astype(np.int32)
    got = None
    for mg in sorted(margins):
        mlp.set_policy(pol["shifts"], pol["posting_cost"], mg)
        ids, _, _ = ix.search_learned(mlp, ip, ii, queries.values, k, kp_min, kp_max)
        ix.sync()
        r = recall(ids, exact_ids, k)
        got = (mg, r)
        if curve is not None:
            curve.append((float(mg), float(r)))
        if r >= target:
            break
    return got


def features(ix, queries, batch: int = 8192) -> torch.Tensor:
    parts = []
    for _, qs in _batches(queries, batch):
        parts.append(ix.kp_features(qs.indptr.astype(np.int64), qs.indices.astype(np.int32),
                                    qs.values))
    return torch.cat(parts)


def train(ix, queries, kp_labels, k: int = 10, tau: float = 0.9, epochs: int = 30,
          batch: int = 2048, lr: float = 2e-3, seed: int = 7, hidden: int = 256,
          log=None) -> "sinnamon.MLP":
    """Fit log2(k') with the pinball loss at quantile tau (most queries get a
    k' at or above their label)."""
    X = features(ix, queries)
    t = torch.from_numpy(np.log2(np.maximum(kp_labels, k).astype(np.float32))).to(X.device)
    return _fit(X, t, tau, epochs, batch, lr, seed, hidden, log)


def evaluate(ix, mlp, queries, exact_ids, k: int = 10, kp_min: int = 10, kp_max: int = 20000,
             fixed: int = 1000):
    """recall@k and mean k' of the learned search vs. a fixed k'."""
    ip = queries.indptr.astype(np.int64)
    ii = queries.indices.astype(np.int32)
    ids_l, _, kp = ix.search_learned(mlp, ip, ii, queries.values, k, kp_min, kp_max)
    ids_f, _ = ix.search(ip, ii, queries.values, k=k, k_prime=fixed)
    ix.sync()

    def recall(ids):
        ids = ids.cpu().numpy().astype(np.int64)
        return float(np.mean([len(set(ids[r]) & set(exact_ids[r])) / k
                              for r in range(ids.shape[0])]))

    return {"recall_learned": recall(ids_l), "recall_fixed": recall(ids_f),
            "mean_kprime_learned": float(kp.float().mean().item()), "fixed_kprime": fixed,
            "p90_kprime_learned": float(kp.float().quantile(0.9).item())}
