"""Continuous-batching serving loop over one GPU index.

Requests (insert a vector, delete a live vector, search a query) arrive over
time.  The loop keeps the index on the device and:
  * admits waiting queries into a free search context (a "slot": its own
    scratch memory and stream) as soon as one frees up, as one batch of at
    most ``max_batch`` queries, the most that fit the slot's scratch; the
    batch size follows the load;
  * runs several slots' searches at once on different streams (a search
    only reads the index);
  * applies inserts and deletes in epochs: once the oldest pending mutation
    has waited ``mutation_delay`` seconds, every pending mutation is applied
    at the next sequence number (the epoch's deletes, then its inserts) while
    the searches in flight keep running -- no drain.
Consistency (snapshot rule): a query is searched at the sequence number of
the last epoch applied before it arrived, so it counts exactly the mutations
applied before its arrival, however long it waits for a slot or runs beside
later epochs (the library's snapshot searches: born <= s < died).  Deleted
ids keep their postings until no queued or running query is older than the
delete (``sinn_reclaim``), and a tile rebuilt by an epoch is rebuilt again
only once the searches older than that epoch are done (an insert returns
SINN_EBUSY before that; the loop then waits for the oldest searches only).
The loop returns its log in order, reclaims included, so that ``replay``
can reproduce every id and answer any query alone.

The host does scheduling and argument marshalling only; inserts, deletes and
searches are the library's calls (sinn_insert_at, sinn_delete_at,
sinn_reclaim, sinn_search_ctx, sinn_search_learned_ctx at a context's
snapshot).
"""
from __future__ import annotations

import gc
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
        self.snap = None   # their snapshot


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
        # mutations run on a stream of their own, ordered before later
        # searches by an event and beside the ones in flight
        self.mstream = torch.cuda.Stream(device=index.device)
        self.mutated = torch.cuda.Event()
        self.mutated.record(torch.cuda.current_stream(index.device))
        self.t_delete = self.t_insert = self.t_wait = 0.0
        self.seq = 0            # the last epoch applied (the starting documents: 0)
        self.reclaimed = 0      # the reclaim horizon handed to the library
        self.busy_waits = 0
        torch.cuda.synchronize(index.device)

    # ------------------------------------------------------------ mutations
    def _reclaim(self, log, horizon):
        if horizon > self.reclaimed:
            with torch.cuda.stream(self.mstream):
                self.ix.reclaim(horizon, stream=self.mstream)
            self.reclaimed = horizon
            log.append(("reclaim", [], None, None, horizon))

    def _apply(self, reqs, pending, log, horizon_fn, wait_oldest):
        """Apply one epoch's mutations at the next sequence number: first its
        deletes (each picks among the ids live when the epoch opened), then
        its inserts, which reuse reclaimed ids first -- one library call
        each.  An insert that would rebuild a tile some older search may
        still read (SINN_EBUSY) waits for the oldest searches and retries."""
        t0 = time.perf_counter()
        self._reclaim(log, horizon_fn())
        self.seq += 1
        e = self.seq
        dels = [r for r in pending if reqs[r].kind == "delete"]
        ins = [r for r in pending if reqs[r].kind == "insert"]
        if dels:
            ids = [self.live.take(reqs[r].u) for r in dels if len(self.live)]
            if ids:
                with torch.cuda.stream(self.mstream):
                    self.ix.delete_at(np.asarray(ids, np.int32), e, stream=self.mstream)
            log.append(("delete", dels, None, np.asarray(ids, np.int64), e))
        t1 = time.perf_counter()
        if ins:
            rows = [reqs[r].row for r in ins]
            ip, idx, val = csr_rows(self.pool, rows)
            while True:
                try:
                    with torch.cuda.stream(self.mstream):
                        got = self.ix.insert_at(ip, idx, val, e, stream=self.mstream)
                        ids = got.cpu().numpy().astype(np.int64)
                    break
                except sinnamon.SinnError as err:
                    if err.code != sinnamon.SINN_EBUSY:
                        raise
                    self.busy_waits += 1
                    tw = time.perf_counter()
                    wait_oldest()
                    self.t_wait += time.perf_counter() - tw
                    self._reclaim(log, horizon_fn())
            self.live.add(ids)
            log.append(("insert", ins, rows, ids, e))
        self.mutated.record(self.mstream)
        t2 = time.perf_counter()
        self.t_delete += t1 - t0
        self.t_insert += t2 - t1

    # ------------------------------------------------------------ searches
    def _launch(self, s, batch, reqs, log, snap):
        rows = [reqs[q].row for q in batch]
        ip, idx, val = csr_rows(self.queries, rows)
        n, nz = len(batch), idx.size
        s.h_ip.numpy()[:n + 1] = ip
        s.h_ix.numpy()[:nz] = idx
        s.h_v.numpy()[:nz] = val
        s.ctx.set_snapshot(snap)  # the epochs applied before these queries arrived
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
        s.snap = snap
        log.append(("query", list(batch), rows, None, snap))

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
        s.snap = None

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
        lists ("insert"|"delete"|"query"|"reclaim", request indices, pool
        rows, ids, sequence number) in the order the loop made the calls (a
        query's number is its snapshot, a reclaim's its horizon)."""
        # the interpreter's cyclic collector is paused while serving: a full
        # collection over the requests, results and log objects stalls the
        # loop for tens of milliseconds, which every queued query would wait
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._serve(reqs, max_wall)
        finally:
            if gc_was:
                gc.enable()

    def _serve(self, reqs, max_wall):
        n = len(reqs)
        results, done_t = {}, np.full(n, np.nan)
        log, wm = [], []
        wq = []  # waiting queries: (request index, snapshot)
        nxt, batches, inflight_max, epochs, overlapped = 0, 0, 0, 0, 0
        epoch_max = 0.0  # the longest epoch, host time
        self.launch_max = 0.0  # the longest batch launch, host time
        self.t_delete = self.t_insert = self.t_wait = 0.0
        self.busy_waits = 0
        t0 = time.perf_counter()

        def admit(queue):
            # a batch holds queries of one snapshot (arrival order keeps them
            # contiguous)
            nonlocal batches, inflight_max
            for s in self.slots:
                if queue and s.batch is None:
                    snap = queue[0][1]
                    j = 0
                    while j < len(queue) and j < self.max_batch and queue[j][1] == snap:
                        j += 1
                    tl = time.perf_counter()
                    self._launch(s, [q for q, _ in queue[:j]], reqs, log, snap)
                    self.launch_max = max(self.launch_max, time.perf_counter() - tl)
                    queue = queue[j:]
                    batches += 1
            inflight_max = max(inflight_max, sum(s.batch is not None for s in self.slots))
            return queue

        def horizon():
            # no search at a smaller number is queued or running, and every
            # later arrival gets at least the current number
            snaps = [s.snap for s in self.slots if s.batch is not None] + [p for _, p in wq]
            return min(snaps + [self.seq])

        def wait_oldest():
            nonlocal wq
            busy = [s for s in self.slots if s.batch is not None]
            if busy:
                s = min(busy, key=lambda x: x.snap)
                s.done.synchronize()
                self._reap(s, results, done_t, t0)
            wq = admit(wq)

        while nxt < n or wq or wm or any(s.batch is not None for s in self.slots):
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                nxt = n
            while nxt < n and reqs[nxt].t <= now:
                if reqs[nxt].kind == "query":
                    wq.append((nxt, self.seq))
                else:
                    wm.append(nxt)
                nxt += 1
            self._poll(results, done_t, t0)
            wq = admit(wq)
            if wm and (now - reqs[wm[0]].t >= self.mutation_delay or nxt >= n):
                # an epoch: applied at the next number while searches run
                overlapped += any(s.batch is not None for s in self.slots)
                te = time.perf_counter()
                self._apply(reqs, wm, log, horizon, wait_oldest)
                epoch_max = max(epoch_max, time.perf_counter() - te)
                done_t[wm] = time.perf_counter() - t0
                wm = []
                epochs += 1
                continue
            if not wq and not wm and nxt < n and all(s.batch is None for s in self.slots):
                wait = reqs[nxt].t - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        self._reclaim(log, horizon())  # nothing is in flight any more
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
                 "epochs": epochs, "epochs_overlapped": overlapped,
                 "epoch_max_ms": 1000.0 * epoch_max, "launch_max_ms": 1000.0 * self.launch_max,
                 "epoch_busy_wait_s": self.t_wait,
                 "busy_waits": self.busy_waits, "epoch_delete_s": self.t_delete,
                 "epoch_insert_s": self.t_insert, "max_batch": self.max_batch,
                 "max_inflight": inflight_max, "slots": len(self.slots)}
        return stats, results, log


def replay(index, queries, docs_pool, log, k: int, k_prime: int = 1000, mlp=None,
           kp_max: int = 4096, pick=None, approx=False, k_primes=None):
    """Apply a served log to another index holding the same starting
    documents -- the same library calls in the same order, so every id comes
    out the same -- and answer each chosen query (request indices in
    ``pick``; all when None) alone, by a plain search (no snapshot) at the
    point where exactly the epochs up to its snapshot have been applied.
    k' per query: ``k_primes[q]`` when given, else the network's (``mlp``)
    or ``k_prime``.  Returns {request index: (ids, scores, k')}, plus each
    query's Alg. 6 scores over all ids at that point when ``approx``."""
    out, scores = {}, {}
    by_snap = {}
    for kind, reqs_i, rows, ids, seq in log:
        if kind == "query":
            by_snap.setdefault(seq, []).append((reqs_i, rows))
    done = set()

    def answer_upto(e):
        for snap in sorted(x for x in by_snap if x <= e and x not in done):
            done.add(snap)
            for reqs_i, rows in by_snap[snap]:
                for q, row in zip(reqs_i, rows):
                    if pick is not None and q not in pick:
                        continue
                    ip, idx, val = csr_rows(queries, [row])
                    if k_primes is not None or mlp is None:
                        kp = k_prime if k_primes is None else int(k_primes[q])
                        r_ids, r_sc = index.search(ip, idx, val, k=k, k_prime=kp)
                    else:
                        r_ids, r_sc, r_kp = index.search_learned(mlp, ip, idx, val, k, k, kp_max)
                        kp = int(r_kp.cpu().numpy()[0])
                    out[q] = (r_ids.cpu().numpy()[0], r_sc.cpu().numpy()[0], kp)
                    if approx:
                        scores[q] = index.scores(ip, idx, val).cpu().numpy()[0]

    applied = 0  # the last epoch applied
    for kind, reqs_i, rows, ids, seq in log:
        if kind in ("insert", "delete") and seq > applied:
            answer_upto(applied)  # an epoch starts: the earlier snapshots are complete
            applied = seq
        if kind == "insert":
            ip, idx, val = csr_rows(docs_pool, rows)
            got = index.insert_at(ip, idx, val, seq).cpu().numpy().astype(np.int64)
            if not np.array_equal(got, ids):
                raise AssertionError("replayed insert assigned other ids")
        elif kind == "delete":
            if ids.size:
                index.delete_at(ids.astype(np.int32), seq)
        elif kind == "reclaim":
            index.reclaim(seq)
    answer_upto(applied)
    return (out, scores) if approx else out
