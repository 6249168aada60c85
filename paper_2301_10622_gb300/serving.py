"""Continuous-batching serving loop over one GPU index.

Requests (insert a vector, delete a live vector, search a query) arrive over
time.  The loop keeps the index on the device and:
  * admits waiting queries into a free search context (a "slot": its own
    scratch memory and stream) as soon as one frees up, as one batch of at
    most ``max_batch`` queries, the most that fit the slot's scratch; the
    batch size follows the load;
  * runs several slots' searches at once on different streams (a search
    only reads the index);
  * applies inserts and deletes at epoch boundaries: once the oldest
    pending mutation has waited ``mutation_delay`` seconds, it admits every
    waiting query (all arrived before the boundary), waits for the searches
    in flight (a mutation changes the index in place), then applies every
    pending mutation -- the epoch's deletes, then its inserts.
Consistency (snapshot rule): requests get sequence numbers in the order the
loop applies or admits them; a query sees exactly the mutations with smaller
sequence numbers.  Those all arrived before it, and the newer ones it misses
arrived at most one epoch (about ``mutation_delay`` plus the drain) before
it.  The loop returns its log in sequence order so that ``replay`` can
reproduce any query alone.

The host does scheduling and argument marshalling only; inserts, deletes and
searches are the library's calls (sinn_insert, sinn_delete, sinn_search_ctx,
sinn_search_learned_ctx).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import sinnamon


@dataclass
class Request:
    t: float          # arrival time, seconds from the start of serving
    kind: str         # "insert" | "delete" | "query"
    row: int = -1     # insert: row of the document pool; query: row of the query pool
    u: float = 0.0    # delete: removes the floor(u * live)-th entry of the live list


def poisson_stream(duration: float, rates: dict, n_docs_pool: int, n_q_pool: int,
                   seed: int = 4000):
    """Merged Poisson arrivals of the kinds in ``rates`` (per second) over
    ``duration`` seconds; inserts walk the document pool in order, queries
    draw pool rows uniformly, deletes carry a uniform draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for kind in ("insert", "delete", "query"):
        rate = rates.get(kind, 0.0)
        if rate <= 0:
            continue
        n = int(rng.poisson(rate * duration))
        ts = np.sort(rng.uniform(0.0, duration, n))
        if kind == "insert":
            rows = np.arange(n) % n_docs_pool
            reqs += [Request(float(t), kind, int(r)) for t, r in zip(ts, rows)]
        elif kind == "query":
            rows = rng.integers(0, n_q_pool, n)
            reqs += [Request(float(t), kind, int(r)) for t, r in zip(ts, rows)]
        else:
            us = rng.random(n)
            reqs += [Request(float(t), kind, -1, float(u)) for t, u in zip(ts, us)]
    reqs.sort(key=lambda r: r.t)
    return reqs


class LiveList:
    """Live ids in a swap-remove array: uniform picks in O(1), deterministic
    for a given order of operations."""

    def __init__(self, ids=()):
        self.a = [int(i) for i in ids]

    def __len__(self):
        return len(self.a)

    def add(self, ids):
        self.a.extend(int(i) for i in ids)

    def take(self, u: float) -> int:
        j = min(int(u * len(self.a)), len(self.a) - 1)
        d = self.a[j]
        self.a[j] = self.a[-1]
        self.a.pop()
        return d


def csr_rows(pool, rows):
    """Rows of a CSR pool as (indptr int64, indices int32, values float32)."""
    rows = np.asarray(rows, np.int64)
    ip = pool.indptr.astype(np.int64)
    lens = ip[rows + 1] - ip[rows]
    out_ip = np.zeros(rows.size + 1, np.int64)
    np.cumsum(lens, out=out_ip[1:])
    total = int(out_ip[-1])
    if total:
        gather = np.repeat(ip[rows] - out_ip[:-1], lens) + np.arange(total)
    else:
        gather = np.zeros(0, np.int64)
    return out_ip, pool.indices[gather].astype(np.int32), \
        np.ascontiguousarray(pool.values[gather], np.float32)


class _Slot:
    """One search context with its stream, staging and output buffers."""

    def __init__(self, index, scratch_bytes, max_batch, max_nnz, k, mlp):
        dev = index.device
        self.ctx = sinnamon.Context(index, scratch_bytes, mlp=mlp, max_queries=max_batch)
        self.stream = torch.cuda.Stream(device=dev)
        pin = dict(pin_memory=True)
        self.h_ip = torch.empty(max_batch + 1, dtype=torch.int64, **pin)
        self.h_ix = torch.empty(max(max_nnz, 1), dtype=torch.int32, **pin)
        self.h_v = torch.empty(max(max_nnz, 1), dtype=torch.float32, **pin)
        self.d_ip = torch.empty(self.h_ip.shape, dtype=torch.int64, device=dev)
        self.d_ix = torch.empty(self.h_ix.shape, dtype=torch.int32, device=dev)
        self.d_v = torch.empty(self.h_v.shape, dtype=torch.float32, device=dev)
        self.ids = torch.empty((max_batch, k), dtype=torch.int32, device=dev)
        self.sc = torch.empty((max_batch, k), dtype=torch.float32, device=dev)
        self.kp = torch.empty(max_batch, dtype=torch.int32, device=dev)
        self.h_ids = torch.empty((max_batch, k), dtype=torch.int32, **pin)
        self.h_sc = torch.empty((max_batch, k), dtype=torch.float32, **pin)
        self.h_kp = torch.empty(max_batch, dtype=torch.int32, **pin)
        self.done = torch.cuda.Event()
        self.batch = None  # request indices in flight


class Server:
    """Serves a request stream against ``index`` (see the module docstring).

    queries / docs_pool: CSR pools that query and insert requests point into.
    live_ids: ids live in ``index`` at the start (delete requests pick among
    the live ids).  slots: number of concurrent search contexts; slot_bytes:
    scratch of each.  k_prime: fixed re-ranking depth when ``mlp`` is None;
    with ``mlp`` each query's k' comes from the network, clamped to
    [k, kp_max].
    """

    def __init__(self, index, queries, docs_pool, live_ids, slots: int = 4,
                 slot_bytes: int = 1 << 30, max_batch: int = 512, k: int = 10,
                 k_prime: int = 1000, mlp=None, kp_max: int = 4096,
                 mutation_delay: float = 0.005):
        self.ix, self.queries, self.pool = index, queries, docs_pool
        self.k, self.k_prime, self.mlp, self.kp_max = k, k_prime, mlp, kp_max
        self.mutation_delay = mutation_delay
        self.live = LiveList(live_ids)
        q_lens = np.diff(queries.indptr.astype(np.int64))
        probe = sinnamon.Context(index, 1 << 20)
        per_q = probe.query_bytes(kp_max if mlp is not None else k_prime)
        probe.close()
        # admission by scratch memory: a slot takes as many queries as fit
        self.max_batch = int(max(1, min(max_batch, slot_bytes // max(per_q, 1))))
        max_nnz = int(np.sort(q_lens)[::-1][:self.max_batch].sum())
        if mlp is not None:
            # make the network's bf16 weights current before the slots share it
            mlp.forward(torch.zeros((1, sinnamon.KP_FEATURES), device=index.device))
        self.slots = [_Slot(index, slot_bytes, self.max_batch, max_nnz, k, mlp)
                      for _ in range(slots)]
        self.mutated = torch.cuda.Event()
        self.mutated.record(torch.cuda.current_stream(index.device))
        self.t_delete = self.t_insert = 0.0
        torch.cuda.synchronize(index.device)

    # ------------------------------------------------------------ mutations
    def _apply(self, reqs, pending, log):
        """Apply one epoch's mutations: first its deletes (each picks among
        the ids live when the epoch opened), then its inserts, which reuse
        the freed ids first -- one library call each."""
        t0 = time.perf_counter()
        dels = [r for r in pending if reqs[r].kind == "delete"]
        ins = [r for r in pending if reqs[r].kind == "insert"]
        if dels:
            ids = [self.live.take(reqs[r].u) for r in dels if len(self.live)]
            if ids:
                self.ix.delete(np.asarray(ids, np.int32))
            log.append(("delete", dels, None, np.asarray(ids, np.int64)))
        t1 = time.perf_counter()
        if ins:
            rows = [reqs[r].row for r in ins]
            ip, idx, val = csr_rows(self.pool, rows)
            ids = self.ix.insert(ip, idx, val).cpu().numpy().astype(np.int64)
            self.live.add(ids)
            log.append(("insert", ins, rows, ids))
        self.mutated.record(torch.cuda.current_stream(self.ix.device))
        t2 = time.perf_counter()
        self.t_delete += t1 - t0
        self.t_insert += t2 - t1

    # ------------------------------------------------------------ searches
    def _launch(self, s, batch, reqs, log):
        rows = [reqs[q].row for q in batch]
        ip, idx, val = csr_rows(self.queries, rows)
        n, nz = len(batch), idx.size
        s.h_ip.numpy()[:n + 1] = ip
        s.h_ix.numpy()[:nz] = idx
        s.h_v.numpy()[:nz] = val
        with torch.cuda.stream(s.stream):
            s.stream.wait_event(self.mutated)
            s.d_ip[:n + 1].copy_(s.h_ip[:n + 1], non_blocking=True)
            s.d_ix[:nz].copy_(s.h_ix[:nz], non_blocking=True)
            s.d_v[:nz].copy_(s.h_v[:nz], non_blocking=True)
            if self.mlp is None:
                s.ctx.search(s.d_ip[:n + 1], s.d_ix, s.d_v, self.k, self.k_prime, s.ids[:n],
                             s.sc[:n], stream=s.stream)
                s.kp[:n].fill_(self.k_prime)
            else:
                s.ctx.search_learned(s.d_ip[:n + 1], s.d_ix, s.d_v, self.k, self.k, self.kp_max,
                                     s.ids[:n], s.sc[:n], s.kp[:n], stream=s.stream)
            s.h_ids[:n].copy_(s.ids[:n], non_blocking=True)
            s.h_sc[:n].copy_(s.sc[:n], non_blocking=True)
            s.h_kp[:n].copy_(s.kp[:n], non_blocking=True)
            s.done.record(s.stream)
        s.batch = list(batch)
        log.append(("query", list(batch), rows, None))

    def _reap(self, s, results, done_t, t0):
        n = len(s.batch)
        ids = s.h_ids[:n].numpy().copy()
        sc = s.h_sc[:n].numpy().copy()
        kp = s.h_kp[:n].numpy().copy()
        t = time.perf_counter() - t0
        for r, q in enumerate(s.batch):
            results[q] = (ids[r], sc[r], int(kp[r]))
            done_t[q] = t
        s.batch = None

    def _poll(self, results, done_t, t0, block=False):
        for s in self.slots:
            if s.batch is not None and (block or s.done.query()):
                if block:
                    s.done.synchronize()
                self._reap(s, results, done_t, t0)

    def serve(self, reqs, max_wall: float | None = None):
        """Serve ``reqs`` (sorted by arrival) in real time.

        Stops taking new arrivals once ``max_wall`` seconds have passed (an
        overloaded server would otherwise fall behind without end); the
        requests not taken are counted as dropped.  Returns (stats, results,
        log): results maps a query's request index to (ids, scores, k'); log
        lists ("insert"|"delete"|"query", request indices, pool rows, ids)
        in sequence order."""
        n = len(reqs)
        results, done_t = {}, np.full(n, np.nan)
        log, wq, wm = [], [], []
        nxt, batches, inflight_max, epochs, t_drain = 0, 0, 0, 0, 0.0
        self.t_delete = self.t_insert = 0.0
        t0 = time.perf_counter()

        def admit(queue):
            nonlocal batches, inflight_max
            for s in self.slots:
                if queue and s.batch is None:
                    b, queue = queue[:self.max_batch], queue[self.max_batch:]
                    self._launch(s, b, reqs, log)
                    batches += 1
            inflight_max = max(inflight_max, sum(s.batch is not None for s in self.slots))
            return queue

        while nxt < n or wq or wm or any(s.batch is not None for s in self.slots):
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                nxt = n
            while nxt < n and reqs[nxt].t <= now:
                (wq if reqs[nxt].kind == "query" else wm).append(nxt)
                nxt += 1
            self._poll(results, done_t, t0)
            if wm and (now - reqs[wm[0]].t >= self.mutation_delay or nxt >= n):
                # epoch boundary: every waiting query arrived before it and
                # runs on the old snapshot; then the searches drain and the
                # pending mutations apply
                while wq:
                    wq = admit(wq)
                    if wq:
                        self._poll(results, done_t, t0, block=True)
                td = time.perf_counter()
                self._poll(results, done_t, t0, block=True)
                t_drain += time.perf_counter() - td
                self._apply(reqs, wm, log)
                done_t[wm] = time.perf_counter() - t0
                wm = []
                epochs += 1
                continue
            wq = admit(wq)
            if not wq and not wm and nxt < n and all(s.batch is None for s in self.slots):
                wait = reqs[nxt].t - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        wall = time.perf_counter() - t0
        kinds = np.array([r.kind for r in reqs])
        arrive = np.array([r.t for r in reqs])
        lat = (done_t - arrive) * 1000.0
        served = ~np.isnan(lat)
        ql = lat[(kinds == "query") & served]
        ml = lat[(kinds != "query") & served]

        def pct(a, p):
            return float(np.percentile(a, p)) if a.size else None

        stats = {"requests": n, "queries": int(ql.size), "mutations": int(ml.size),
                 "dropped": int(n - served.sum()), "wall_s": wall,
                 "queries_per_s": ql.size / wall, "mutations_per_s": ml.size / wall,
                 "p50_ms": pct(ql, 50), "p99_ms": pct(ql, 99),
                 "mutation_p50_ms": pct(ml, 50), "mutation_p99_ms": pct(ml, 99),
                 "query_batches": batches, "mean_batch": ql.size / max(batches, 1),
                 "epochs": epochs, "epoch_drain_s": t_drain, "epoch_delete_s": self.t_delete,
                 "epoch_insert_s": self.t_insert, "max_batch": self.max_batch,
                 "max_inflight": inflight_max, "slots": len(self.slots)}
        return stats, results, log


def replay(index, queries, docs_pool, log, k: int, k_prime: int = 1000, mlp=None,
           kp_max: int = 4096, pick=None, approx=False):
    """Apply a served log to another index holding the same starting
    documents and answer the chosen queries (request indices in ``pick``;
    all when None) one at a time at their place in the sequence.  Returns
    {request index: (ids, scores, k')}, plus each query's Alg. 6 scores over
    all ids at that point when ``approx``."""
    out, scores = {}, {}
    for kind, reqs_i, rows, ids in log:
        if kind == "insert":
            ip, idx, val = csr_rows(docs_pool, rows)
            got = index.insert(ip, idx, val).cpu().numpy().astype(np.int64)
            if not np.array_equal(got, ids):
                raise AssertionError("replayed insert assigned other ids")
        elif kind == "delete":
            if ids.size:
                index.delete(ids.astype(np.int32))
        else:
            for q, row in zip(reqs_i, rows):
                if pick is not None and q not in pick:
                    continue
                ip, idx, val = csr_rows(queries, [row])
                if mlp is None:
                    r_ids, r_sc = index.search(ip, idx, val, k=k, k_prime=k_prime)
                    kp = k_prime
                else:
                    r_ids, r_sc, r_kp = index.search_learned(mlp, ip, idx, val, k, k, kp_max)
                    kp = int(r_kp.cpu().numpy()[0])
                out[q] = (r_ids.cpu().numpy()[0], r_sc.cpu().numpy()[0], kp)
                if approx:
                    scores[q] = index.scores(ip, idx, val).cpu().numpy()[0]
    return (out, scores) if approx else out
