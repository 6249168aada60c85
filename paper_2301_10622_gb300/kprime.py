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
    nq = cid.shape[0]
    # candidates in approximate-rank order: score desc, id asc
    cid64 = cid.to(torch.int64)
    valid = torch.arange(cap, device=cid.device)[None, :] < cnt[:, None].to(torch.int64)
    cs = torch.where(valid, cs, torch.full_like(cs, -float("inf")))
    cid64 = torch.where(valid, cid64, torch.full_like(cid64, 1 << 40))
    o1 = torch.argsort(cid64, dim=1, stable=True)
    s1 = torch.gather(cs, 1, o1)
    o2 = torch.argsort(-s1, dim=1, stable=True)
    order = torch.gather(o1, 1, o2)
    ranked_ids = torch.gather(cid64, 1, order)               # rank r -> id
    tau = torch.where(cnt > 0, torch.gather(s1, 1, o2)[torch.arange(nq, device=cs.device),
                                                       (cnt - 1).clamp(min=0).to(torch.int64)],
                      torch.zeros(nq, device=cs.device))
    # rank of each exact top-k id among the candidates (1-based)
    ids64 = ids.to(torch.int64)
    match = ranked_ids[:, None, :] == ids64[:, :, None]      # nq x k x cap
    has = match.any(dim=2)
    rank = match.to(torch.int8).argmax(dim=2).to(torch.int64) + 1
    rank = torch.where(has & (ids64 >= 0), rank, torch.full_like(rank, cap + 1))
    kth = torch.sort(rank, dim=1).values[:, keep - 1]
    tenth = sc[:, k - 1]
    full = cnt.to(torch.int64) < cap                         # every live id is a candidate
    cert = full | (tenth >= tau)
    kp = torch.where(cert, kth.clamp(max=cap), torch.full_like(kth, cap))
    return kp, cert


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
    mean = X.mean(dim=0).cpu().numpy()
    std = X.std(dim=0).clamp(min=1e-6).cpu().numpy()
    mlp = sinnamon.MLP(sinnamon.KP_FEATURES, hidden, seed=seed, device=X.device)
    mlp.set_normalizer(mean, std)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot = 0.0
        for a in range(0, n, batch):
            idx = perm[a:a + batch]
            xb, tb = X[idx].contiguous(), t[idx].contiguous()
            loss = mlp.train_step(xb, tb, tau, lr * (0.5 * (1 + math.cos(math.pi * ep / epochs))))
            tot += float(loss.item()) * idx.numel()
        if log:
            log(f"epoch {ep}: pinball loss {tot / n:.4f}")
    mlp.sync()  # raises if a tensor-core GEMM's bounded wait ran out
    return mlp


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
