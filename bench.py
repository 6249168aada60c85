#!/usr/bin/env python
"""Benchmark: streaming SINNAMON on the text-like workload (one JSON line).

One step = one pass of the whole path over one batch of synthetic input:
delete D live vectors (Sec. 4.3), insert D new ones (Alg. 5; they reuse the
freed ids), then search a batch of Q queries (Alg. 6 + Alg. 7) with each
query's Alg. 6 budget and k' chosen by the learned network (trained before
timing on the method's own labels; --fixed-kprime uses the whole query and
k' = 1000 instead).  The metric is queries/s (Q per step); recall@10 against
the FP64 exact top-10 is measured on the same index and reported beside it,
as are the plain baseline (one query per call, fixed k'), the batched
fixed-k' search and the mixed-sign workload's line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank holds its own replica of the index and searches its
own query batch (replicas only: the method's path does not shard), so value =
all ranks' queries / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at recall@10>=0.9 (batched search with learned per-query k' and Alg. 6 budget)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


_T_START = time.time()


def log(*a):
    print(f"[{time.time() - _T_START:7.1f}s]", *a, file=sys.stderr, flush=True)


def job_throughput(elapsed_s: float, units: float, device=None):
    """Whole-job throughput of replicas: every rank's units over the slowest
    rank's time (MAX over ranks; one process without a process group).
    Returns (units/s, slowest elapsed seconds)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if world > 1:
        t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
        dist.barrier()
    return world * units / elapsed_s, elapsed_s


# ----------------------------------------------------------------- inputs

def _synth_key():
    """First 12 hex digits of synth.py's sha256: a change to the generator
    (or its seeds) makes new cache files instead of reusing stale inputs."""
    import hashlib
    src = os.path.join(ROOT, "paper_2301_10622_gb300", "synth.py")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]


def cached(name, fn):
    """With SINN_BENCH_CACHE=1, generated inputs are cached in /tmp under
    their name (which carries the size and seed) and the generator's hash,
    and regenerated when absent; otherwise every run generates them (on a
    fresh machine writing the cache costs more than it saves)."""
    if os.environ.get("SINN_BENCH_CACHE", "0") != "1":
        return fn()
    path = f"/tmp/sinn_bench_{name}_{_synth_key()}.npz"
    if os.path.exists(path):
        z = np.load(path)
        from paper_2301_10622_gb300.synth import CSR
        return CSR(z["indptr"], z["indices"], z["values"])
    c = fn()
    tmp = path + f".{os.getpid()}.npz"
    np.savez(tmp, indptr=c.indptr, indices=c.indices, values=c.values)
    os.replace(tmp, path)
    return c


def make_inputs(args, rank, workload=None, n_docs=0):
    from paper_2301_10622_gb300 import synth
    w = synth.WORKLOADS[workload or args.workload]
    nd = n_docs or args.docs or w.n_docs
    t0 = time.time()
    docs = cached(f"{w.name}_docs_{nd}_s{synth._seed(w, 1000)}",
                  lambda: synth.make_docs(w, n_docs=nd))
    pool_n = args.churn * (args.steps + args.warmup + 8)
    pool = cached(f"{w.name}_pool_{pool_n}_s5000",
                  lambda: synth.make_docs(w, n_docs=pool_n, seed=5000))
    nq = args.queries or w.n_queries
    qseed = synth._seed(w, 2000) + 100 * rank
    qs = cached(f"{w.name}_q_{nq}_s{qseed}", lambda: synth.make_queries(w, n_q=nq, seed=qseed))
    log(f"inputs ready in {time.time() - t0:.1f}s: docs={docs.rows} nnz={docs.nnz} "
        f"queries={qs.rows} pool={pool.rows}")
    return w, docs, pool, qs


def list_lengths(w, docs):
    nz = docs.values != 0
    return np.bincount(docs.indices[nz], minlength=w.n).astype(np.int64)


def scored_postings(qs, lens, budgets=None):
    """Postings Alg. 6 visits per query: every term's list, or with budgets[q]
    > 0 the terms in Alg. 6 order (|q_j| descending, ties j ascending) up to
    the first at which the running sum reaches the budget."""
    out = np.zeros(qs.rows, np.int64)
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        keep = qv != 0
        qi, qv = qi[keep], qv[keep]
        ln = lens[qi]
        b = 0 if budgets is None else int(budgets[r])
        if b == 0:
            out[r] = int(ln.sum())
            continue
        order = np.lexsort((qi, -np.abs(qv)))
        cum = np.cumsum(ln[order])
        t = int(np.searchsorted(cum, b))          # first term with cum >= b
        out[r] = int(cum[min(t, cum.size - 1)]) if cum.size else 0
    return out


def algorithmic_bytes(w, postings):
    """Bytes the scoring kernel must move per query (the unshared
    algorithmic count): for each posting of the lists it scores, a 4-byte id
    and h 4-byte sketch reads (only the sign's plane is read)."""
    return postings.astype(np.float64) * (4 + 4 * w.h)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- oracle side

def oracle_index(w, docs):
    import oracle
    ora = oracle.OracleIndex(w.n, w.m, w.h)
    t0 = time.time()
    ora.insert(docs.indptr, docs.indices, docs.values)
    log(f"oracle index built in {time.time() - t0:.1f}s")
    return ora


def cpu_baseline(ora, w, qs, target_s, k, kp):
    """The oracle (Alg. 6 + Alg. 7, FP64) on bounded samples of the queries:
    all host cores (the reported value) and one thread beside it."""
    cores = os.cpu_count() or 1
    one = qs.slice(0, 1)
    t0 = time.time()
    ora.search(one.indptr, one.indices, one.values, k=k, k_prime=kp, threads=1)
    t1 = max(time.time() - t0, 1e-4)
    s = int(min(qs.rows, max(cores, target_s * cores / t1 * 0.8)))
    sample = qs.slice(0, s)
    t0 = time.time()
    ora.search(sample.indptr, sample.indices, sample.values, k=k, k_prime=kp, threads=cores)
    dt = time.time() - t0
    s1 = int(min(qs.rows, max(1, 0.5 * target_s / t1)))
    t0 = time.time()
    ora.search(qs.indptr[:s1 + 1], qs.indices, qs.values, k=k, k_prime=kp, threads=1)
    dt1 = time.time() - t0
    return {"value": s / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"first {s} of {qs.rows} queries over the full index "
                      f"(k={k}, k'={kp}), FP64 Alg. 6+7, {dt:.1f}s on {cores} threads",
            "single_thread": {"value": s1 / dt1, "unit": "queries/s", "cores": 1,
                              "sample": f"first {s1} queries, {dt1:.1f}s on 1 thread"}}


TRUTH_DEPTH = 64  # exact results kept per query for the recall's tie check


def exact_truth(ora, qs_sample, threads):
    """The FP64 exact top TRUTH_DEPTH of each query (the oracle's LinScan)."""
    return ora.linscan_topk(qs_sample.indptr, qs_sample.indices, qs_sample.values,
                            k=TRUTH_DEPTH, threads=threads)


def recall_at_10(ora, qs_sample, gpu_ids, threads, ex=None):
    """recall@10 of the GPU's top-10 against the FP64 exact top-10 (``ex``:
    exact_truth of these queries, computed here when None); a returned id
    whose exact score ties the exact 10th score counts as a hit.  A missed
    id's exact score comes from the exact list, or, when that list is all
    tied with the 10th, from the oracle's dense exact scores."""
    if ex is None:
        ex = exact_truth(ora, qs_sample, threads)
    hits = 0
    for r in range(qs_sample.rows):
        truth = set(int(x) for x in ex["ids"][r][:10])
        known = {int(i): float(v) for i, v in zip(ex["ids"][r], ex["scores"][r])}
        qi, qv = qs_sample.row(r)
        tenth = ex["scores"][r][9]
        tol = 1e-9 * max(1.0, abs(tenth))
        deep = ex["scores"][r][-1] >= tenth - tol  # the exact list ends inside the tie
        got = [int(x) & 0xFFFFFFFF for x in gpu_ids[r][:10]]
        exact = None
        for g in got:
            if g in truth:
                hits += 1
            elif g in known:
                hits += known[g] >= tenth - tol
            elif deep:
                if exact is None:
                    exact = ora.exact_scores(qi, qv)
                hits += g < exact.size and exact[g] >= tenth - tol
    return hits / (10 * qs_sample.rows)


# --------------------------------------------------------------- reference

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2301_10622_gb300 import synth  # noqa: F401
    import oracle
    oracle.build()
    w, docs, pool, qs = make_inputs(args, 0)
    ora = oracle_index(w, docs)
    cores = os.cpu_count() or 1
    one = qs.slice(0, 1)
    t0 = time.time()
    ora.search(one.indptr, one.indices, one.values, k=w.k, k_prime=w.k_prime, threads=1)
    t1 = max(time.time() - t0, 1e-4)
    per_step_s = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    s = int(min(qs.rows, max(cores, per_step_s * cores / t1 * 0.8)))
    churn = max(1, min(args.churn, 20))
    rng = np.random.default_rng(11)
    times = []
    pos = 0
    n_live = docs.rows
    for step in range(args.warmup + args.steps):
        t0 = time.time()
        dele = rng.choice(n_live, size=churn, replace=False).astype(np.uint32)
        ora.delete(dele)
        part = pool.slice(pos, pos + churn)
        pos += churn
        ora.insert(part.indptr, part.indices, part.values)
        sample = qs.slice((step * s) % max(1, qs.rows - s), (step * s) % max(1, qs.rows - s) + s)
        ora.search(sample.indptr, sample.indices, sample.values, k=w.k, k_prime=w.k_prime,
                   threads=cores)
        dt = time.time() - t0
        if step >= args.warmup:
            times.append(dt)
    ms = 1000 * float(np.mean(times))
    value = s / (ms / 1000)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(args, w, docs, qs, None),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: delete {churn} + insert {churn} vectors, then "
                                   f"{s} of {qs.rows} queries (k={w.k}, k'={w.k_prime}), FP64"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def source_code_hash(path):
    """First 16 hex digits of the sha256 of a C/CUDA source with its comments,
    trailing blanks and empty lines removed: edits to comments keep it."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def profile_figures(name, src_file="search.cu"):
    """Figures of a committed ncu summary (profiles/<name>.md) as a dict of
    its `key: value` lines, or None when the summary is missing or the
    kernel source changed since its counters were taken."""
    prof = os.path.join(ROOT, "profiles", name + ".md")
    src = os.path.join(ROOT, "paper_2301_10622_gb300", "csrc", src_file)
    try:
        text = open(prof).read()
    except OSError:
        return None
    fig = {}
    for ln in text.splitlines():
        ln = ln.strip()
        if ":" in ln and " " not in ln.split(":")[0]:
            key, val = ln.split(":", 1)
            try:
                fig[key] = float(val.split()[0])
            except (ValueError, IndexError):
                fig[key] = val.strip()
    want = fig.get("source_code_sha256_16")
    if want is None or source_code_hash(src) != str(want).split()[0]:
        return None
    return fig


def dram_figures(fig, launch_ms, peak, units_per_launch, docs):
    """DRAM bytes per launch from a profile's counters, scaled to this run's
    units per launch; the DRAM fraction of peak over the live launch time;
    the L1 / L2 throughput fractions and the global-load sectors per
    request (the gathers' coalescing) the profile read.  None entries
    when the profile does not match this kernel or this index size, and no
    traffic when this run's launches hold more than 10% more or fewer units
    than the profiled ones (a launch streams the index about once, so its
    traffic is not proportional to its queries)."""
    out = {"traffic": None, "dram_frac": None, "l1_frac": None, "l2_frac": None,
           "sectors_per_request": None}
    if not fig or fig.get("docs_in_index") != docs:
        return out
    per, q = fig.get("traffic_bytes_per_launch"), fig.get("queries_per_launch")
    if per and q and launch_ms and abs(units_per_launch - q) <= 0.1 * q:
        t = per * units_per_launch / q
        out["traffic"] = t
        out["dram_frac"] = t / (launch_ms / 1000.0) / 1e9 / peak
    out["l1_frac"] = fig.get("l1_throughput_frac")
    out["l2_frac"] = fig.get("l2_throughput_frac")
    out["sectors_per_request"] = fig.get("sectors_per_request")
    return out


WORKLOAD_TEXT = {
    "text": ("text-like streaming: n={n}, {docs} docs with Zipf(1) coordinates, nnz/doc "
             "lognormal(mean 120, sigma 0.5), values lognormal(0,0.7); {nq} queries/step nnz "
             "lognormal(mean 45)"),
    "mixed": ("mixed-sign streaming: n={n}, {docs} docs with uniform coordinates, nnz/doc "
              "uniform 80-160, values N(0,1); {nq} queries/step of 40 nnz, values N(0,1)"),
    "tiny": ("tiny: n={n}, {docs} docs of 32 uniform coordinates, values N(0,1); {nq} "
             "queries/step of 16 nnz"),
}


def config_dict(args, w, docs, qs, tile_docs, index_gb=0.0):
    desc = WORKLOAD_TEXT[w.name].format(n=w.n, docs=docs.rows, nq=qs.rows)
    return {"workload": (f"{desc}; m={w.m}, h={w.h}, k={w.k}, k'={w.k_prime}; churn "
                         f"{args.churn} deletes + {args.churn} inserts per step"),
            "docs": docs.rows, "queries_per_step": qs.rows, "churn_per_step": args.churn,
            "n": w.n, "m": w.m, "h": w.h, "k": w.k, "k_prime": w.k_prime,
            "tile_docs": tile_docs,
            "l2": (f"inputs larger than L2: the index's lists and sketch "
                   f"({index_gb:.2f} GB) are read by every step" if index_gb else
                   "inputs larger than L2: the whole index is read by every step")}


# ------------------------------------------------------------------- ours

def build_index(sinnamon, w, docs, dev, T, scratch_gb, flags=0):
    ix = sinnamon.Index(w.n, w.m, w.h, device=dev, tile_docs=T, capacity_hint=docs.rows,
                        scratch_bytes=scratch_gb << 30, flags=flags)
    for a in range(0, docs.rows, 200_000):
        part = docs.slice(a, min(docs.rows, a + 200_000))
        ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    return ix


def train_policy(args, w, ix, k, kp):
    """The learned Alg. 6 budget with k' (trained before timing, on labels
    the method generates): per budget level P_q / 2^s the least k' keeping 9
    of the exact top 10; a network over (features, -s); the per-posting cost
    measured; the margin calibrated on held-out queries for recall >= 0.92."""
    from paper_2301_10622_gb300 import kprime, synth
    t0 = time.time()
    tq = cached(f"{w.name}_train_{args.train_queries}_s3000",
                lambda: synth.make_queries(w, n_q=args.train_queries, seed=3000))
    cq = cached(f"{w.name}_cal_{args.cal_queries}_s3002",
                lambda: synth.make_queries(w, n_q=args.cal_queries, seed=3002))
    shifts = tuple(int(x) for x in args.shifts.split(","))
    _, cert, ex = kprime.labels(ix, tq, k=k, cap=args.kp_cap)
    lv = kprime.level_labels(ix, tq, ex, cert, shifts, k=k, cap=args.kp_cap)
    t_lab = time.time() - t0
    mlp = kprime.train_levels(ix, tq, lv, shifts, k=k, epochs=args.epochs)
    t_fit = time.time() - t0 - t_lab
    pc = kprime.measure_costs(ix, cq, k=k, k_prime=kp)
    mlp.set_policy(shifts, pc, 0.0)
    _, _, ex_c = kprime.labels(ix, cq, k=k, cap=args.kp_cap)
    curve = []
    margin, cal_rec = kprime.calibrate_margin(ix, mlp, cq, ex_c, k=k, kp_min=k,
                                              kp_max=args.kp_max, target=args.cal_recall,
                                              curve=curve)
    info = {"train_queries": tq.rows, "label_cap": args.kp_cap, "search_cap": args.kp_max,
            "certified_labels": float(np.mean(cert)), "levels_shifts": list(shifts),
            "label_median_per_level": [float(np.median(lv[:, i])) for i in range(len(shifts))],
            "label_feasible_per_level": [float(np.mean(lv[:, i] <= args.kp_max))
                                         for i in range(len(shifts))],
            "posting_cost": pc, "margin": margin, "calibration_queries": cq.rows,
            "calibration_recall": cal_rec, "calibration_curve": curve,
            "label_seconds": t_lab, "fit_seconds": t_fit,
            "train_seconds": time.time() - t0}
    log(f"budget + k' network trained: {info}")
    return mlp, info


def timed_best(fn, reps=3):
    """Best CUDA-event time (ms) of fn() on the current stream, after one warm-up."""
    import torch
    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def plain_search(sinnamon, h, qs, g_qix, g_qv, k, kp, dev, npl, alg_full):
    """One query per call (the plain per-query arm): queries/s, latency
    percentiles and the scorer-bytes rate of a lone query."""
    import torch
    npl = min(npl, qs.rows)
    one_ids = torch.empty((1, k), dtype=torch.int32, device=dev)
    one_sc = torch.empty((1, k), dtype=torch.float32, device=dev)
    offs = qs.indptr.astype(np.int64)
    qip1 = [torch.tensor([0, offs[r + 1] - offs[r]], dtype=torch.int64, device=dev)
            for r in range(npl)]
    for r in range(min(3, npl)):
        a = int(offs[r])
        sinnamon.sinn_search(h, qip1[r], g_qix[a:], g_qv[a:], k, kp, one_ids, one_sc)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(npl)]
    torch.cuda.nvtx.range_push("bench plain searches")
    t0 = time.perf_counter()
    for r in range(npl):
        a = int(offs[r])
        evs[r][0].record()
        sinnamon.sinn_search(h, qip1[r], g_qix[a:], g_qv[a:], k, kp, one_ids, one_sc)
        evs[r][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    plain_s = time.perf_counter() - t0
    lat = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    bytes_q = float(np.mean(alg_full[:npl]))
    return {"qps": npl / plain_s, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "queries": npl, "k_prime": kp,
            "alg_bytes_per_query": bytes_q,
            "effective_gbs_at_mean_latency": bytes_q / (float(lat.mean()) / 1000.0) / 1e9}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_10622_gb300 import sinnamon

    w, docs, pool, qs = make_inputs(args, rank)
    k, kp = w.k, w.k_prime
    T = args.tile_docs
    tile_choice = None
    if T == 0:
        # the tile size chosen by measurement (untimed): indexes of the
        # collection at each candidate, launch-autotuned, timed on a sample
        from paper_2301_10622_gb300 import autotune
        t0 = time.time()
        sq = qs.slice(0, min(qs.rows, 2000))
        T, res = autotune.choose_tile_docs(w.n, w.m, w.h, docs, sq, k, kp, device=dev,
                                           scratch_bytes=args.scratch_gb << 30, log=log)
        tile_choice = {str(t): round(r["ms"], 3) for t, r in res.items()}
        log(f"tile size {T} chosen in {time.time() - t0:.1f}s: {tile_choice}")
    t0 = time.time()
    ix = build_index(sinnamon, w, docs, dev, T, args.scratch_gb)
    torch.cuda.synchronize()
    st = ix.stats()
    log(f"gpu index built in {time.time() - t0:.1f}s: {st}")
    lens = list_lengths(w, docs)

    # launch tuning chosen by the autotuner on the step's batch of queries (a
    # smaller sample misjudges how many queries a launch should take)
    tuning = None
    if not args.no_autotune:
        t0 = time.time()
        sq = qs.slice(0, min(qs.rows, args.autotune_queries or qs.rows))
        tuning = ix.autotune(sq.indptr.astype(np.int64), sq.indices.astype(np.int32), sq.values,
                             k, kp, reps=2)
        log(f"autotuned in {time.time() - t0:.1f}s: {tuning}")
    if args.tuning:  # fields set by hand, after (or instead of) the autotuner
        ix.set_tuning(**{kv.split("=")[0]: int(kv.split("=")[1])
                         for kv in args.tuning.split(",")})
    tuning = ix.tuning()

    mlp, kp_info = None, None
    if not args.fixed_kprime:
        mlp, kp_info = train_policy(args, w, ix, k, kp)

    # device-resident step inputs
    g_qip = torch.from_numpy(qs.indptr.astype(np.int64)).to(dev)
    g_qix = torch.from_numpy(qs.indices.astype(np.int32)).to(dev)
    g_qv = torch.from_numpy(qs.values).to(dev)
    out_ids = torch.empty((qs.rows, k), dtype=torch.int32, device=dev)
    out_sc = torch.empty((qs.rows, k), dtype=torch.float32, device=dev)
    nsteps = args.warmup + args.steps
    n_e2e = args.e2e_steps
    rng = np.random.default_rng(7 + rank)
    nparts = nsteps + n_e2e + 2
    dels = [torch.from_numpy(rng.choice(docs.rows, size=args.churn, replace=False)
                             .astype(np.int32)).to(dev) for _ in range(nparts)]
    parts = []
    for s_ in range(nparts):
        p = pool.slice((s_ * args.churn) % max(1, pool.rows - args.churn),
                       (s_ * args.churn) % max(1, pool.rows - args.churn) + args.churn)
        parts.append((torch.from_numpy(p.indptr.astype(np.int64)).to(dev),
                      torch.from_numpy(p.indices.astype(np.int32)).to(dev),
                      torch.from_numpy(p.values).to(dev), p))
    new_ids = torch.empty(args.churn, dtype=torch.int32, device=dev)
    out_kp = torch.empty(qs.rows, dtype=torch.int32, device=dev)
    h = ix.handle
    executed = []

    def search(qip, qix, qv, oids, osc):
        if mlp is None:
            sinnamon.sinn_search(h, qip, qix, qv, k, kp, oids, osc)
        else:
            sinnamon.sinn_search_learned(h, mlp.handle, qip, qix, qv, k, k, args.kp_max, oids,
                                         osc, out_kp)

    # the step's search as one recorded CUDA graph, replayed every step
    plan = None
    if not args.no_graph:
        plan = (sinnamon.Plan(ix, g_qip, g_qix, g_qv, k, kp, scratch_bytes=args.scratch_gb << 30)
                if mlp is None else
                sinnamon.Plan(ix, g_qip, g_qix, g_qv, k, args.kp_max, mlp=mlp, k_prime_min=k,
                              scratch_bytes=args.scratch_gb << 30))
        out_ids, out_sc = plan.out_ids, plan.out_scores
        if mlp is not None:
            out_kp = plan.out_kprime

    def step(si):
        executed.append(si)
        sinnamon.sinn_delete(h, dels[si])
        ip, ii, vv, _ = parts[si]
        sinnamon.sinn_insert(h, ip, ii, vv, new_ids)
        if plan is not None:
            plan.run()
        else:
            search(g_qip, g_qix, g_qv, out_ids, out_sc)

    for si in range(args.warmup):
        step(si)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    with clocks:
        sinnamon.sinn_timing_start(h)
        torch.cuda.nvtx.range_push("bench timed steps")  # a profiler can select these launches
        ev0.record()
        for si in range(args.warmup, nsteps):
            step(si)
        ev1.record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        tm = sinnamon.sinn_timing_stop(h)
    ix.sync()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    value, elapsed = job_throughput(elapsed, qs.rows * args.steps, dev)
    ms_step = 1000 * elapsed / args.steps

    # roofline of the scoring kernel (live CUDA-event durations from the
    # library): the bytes Alg. 6 must move for the postings each query
    # actually scored (its learned budget), 4-byte ids + h 4-byte bins each
    budgets = None
    if mlp is not None:
        _, bud = ix.kp_choose(mlp, g_qip, g_qix, g_qv, k, args.kp_max)
        budgets = bud.cpu().numpy()
    P_full = scored_postings(qs, lens)
    P_scored = scored_postings(qs, lens, budgets)
    alg_q = algorithmic_bytes(w, P_scored)
    score_ms = tm["ms"]["score"]
    launches = max(1, tm["spans"]["score"])
    achieved = float(alg_q.sum()) * args.steps / (score_ms / 1000.0) / 1e9 if score_ms else None
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    dr = dram_figures(profile_figures(f"k_score_emit_{w.name}"), score_ms / launches, peak,
                      qs.rows * args.steps / launches, docs.rows)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "frac_kind": ("effective: algorithmic bytes (4 + 4h per scored posting) over the "
                          "scoring time; queries resident together share each tile's lists and "
                          "sketch rows through L2, so it can exceed 1"),
            "traffic": dr["traffic"], "dram_frac": dr["dram_frac"], "l1_frac": dr["l1_frac"],
            "l2_frac": dr["l2_frac"], "sectors_per_request": dr["sectors_per_request"],
            "kernel": "k_score_emit", "launches": launches,
            "avg_launch_ms": score_ms / launches,
            "peak_source": "measured" if peaks else "fallback",
            "alg_bytes_per_query": float(alg_q.mean()),
            "postings_scored_per_query": float(P_scored.mean()),
            "postings_per_query_unbudgeted": float(P_full.mean())}

    # ---- untimed extras on rank 0: e2e, plain per-query, recall, CPU baseline
    extras = {}
    if rank == 0:
        # e2e: the same step through the host-buffer C ABI search, copies of
        # the step's inputs and results inside the timed region
        pin_q = (torch.from_numpy(qs.indptr.astype(np.int64)).pin_memory(),
                 torch.from_numpy(qs.indices.view(np.int32)).pin_memory(),
                 torch.from_numpy(qs.values).pin_memory())
        ids_pin = torch.empty((qs.rows, k), dtype=torch.int32).pin_memory()
        sc_pin = torch.empty((qs.rows, k), dtype=torch.float32).pin_memory()
        kp_pin = torch.empty(qs.rows, dtype=torch.int32).pin_memory()
        hid_pin = torch.empty(args.churn, dtype=torch.int32).pin_memory()
        pin_m = []
        for si in range(n_e2e):
            _, _, _, p = parts[si + nsteps]
            pin_m.append((torch.from_numpy(p.indptr.astype(np.int64)).pin_memory(),
                          torch.from_numpy(p.indices.astype(np.int32)).pin_memory(),
                          torch.from_numpy(p.values).pin_memory(),
                          torch.from_numpy(dels[si + nsteps].cpu().numpy()).pin_memory()))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for si in range(n_e2e):
            pip, pii, pvv, pdl = pin_m[si]
            executed.append(si + nsteps)
            sinnamon.sinn_delete(h, pdl.to(dev, non_blocking=True))
            sinnamon.sinn_insert(h, pip.to(dev, non_blocking=True),
                                 pii.to(dev, non_blocking=True), pvv.to(dev, non_blocking=True),
                                 new_ids)
            hid_pin.copy_(new_ids, non_blocking=True)
            if mlp is None:
                sinnamon.sinn_search_host(h, *pin_q, k, kp, ids_pin, sc_pin)
            else:
                sinnamon.sinn_search_learned_host(h, mlp.handle, *pin_q, k, k, args.kp_max,
                                                  ids_pin, sc_pin, kp_pin)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / max(1, n_e2e)
        p0 = parts[nsteps][3]
        h2d = int(qs.indptr.nbytes + qs.indices.nbytes + qs.values.nbytes + p0.indptr.nbytes
                  + p0.indices.nbytes + p0.values.nbytes + args.churn * 4)
        d2h = int(qs.rows * k * 8 + args.churn * 4 + (qs.rows * 4 if mlp is not None else 0))
        extras["e2e"] = {"value": qs.rows / e2e_s, "unit": "queries/s", "steps": n_e2e,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "call": "sinn_search_learned_host" if mlp is not None
                         else "sinn_search_host"}

        # plain per-query search: one query per call, fixed k'
        alg_full = algorithmic_bytes(w, P_full)
        extras["plain"] = plain_search(sinnamon, h, qs, g_qix, g_qv, k, kp, dev,
                                       args.plain_queries, alg_full)
        extras["plain"]["frac_of_peak_effective"] = (
            extras["plain"]["effective_gbs_at_mean_latency"] / peak)

        # batched latency (learned, as timed) and the batched fixed-k' search
        ms_b = timed_best(lambda: plan.run() if plan is not None
                          else search(g_qip, g_qix, g_qv, out_ids, out_sc))
        extras["batched"] = {"qps": value / world, "batch_ms": ms_b,
                             "plan_recordings": plan.recordings if plan is not None else None}
        fx_ids = torch.empty((qs.rows, k), dtype=torch.int32, device=dev)
        fx_sc = torch.empty((qs.rows, k), dtype=torch.float32, device=dev)
        ms_f = timed_best(lambda: sinnamon.sinn_search(h, g_qip, g_qix, g_qv, k, kp, fx_ids,
                                                       fx_sc))
        extras["batched_fixed_kprime"] = {"qps": qs.rows / (ms_f / 1000.0), "batch_ms": ms_f,
                                          "k_prime": kp}
        if plan is not None:
            plan.run()   # the learned results on the index as it stands now
        torch.cuda.synchronize()
        if mlp is not None:
            kps = out_kp.float()
            bfrac = np.where(budgets > 0, P_scored / np.maximum(P_full, 1), 1.0)
            extras["learned_kprime"] = dict(
                kp_info, mean=float(kps.mean().item()), p50=float(kps.median().item()),
                p90=float(kps.quantile(0.9).item()), max=float(kps.max().item()),
                mean_scored_fraction=float(bfrac.mean()),
                queries_with_budget=float(np.mean(budgets > 0)),
                speedup_vs_fixed_kprime=extras["batched_fixed_kprime"]["batch_ms"] / ms_b)
        ora = None
        if not args.skip_oracle:
            import oracle
            oracle.build()
            # the GPU index after churn: rebuild the same collection on the oracle
            live_docs = reconstruct(docs, parts, dels, executed)
            ora = oracle_index(w, live_docs)
            nr = min(args.recall_queries, qs.rows)
            samp = qs.slice(0, nr)
            cores = os.cpu_count() or 1
            truth = exact_truth(ora, samp, cores)
            extras["recall_at_10"] = recall_at_10(ora, samp, out_ids.cpu().numpy()[:nr],
                                                  cores, truth)
            extras["recall_at_10_fixed_kprime"] = recall_at_10(
                ora, samp, fx_ids.cpu().numpy()[:nr], cores, truth)
            extras["recall_queries"] = nr
            extras["cpu_baseline"] = cpu_baseline(ora, w, qs, args.cpu_seconds, k, kp)
        if not args.skip_variants:
            extras.update(run_variants(args, w, live_docs if ora is not None else docs, ix,
                                       (g_qip, g_qix, g_qv), qs, k, kp, float(P_full.mean()),
                                       ora, T, truth if ora is not None else None))
        if args.serve_seconds > 0:
            extras["serving"] = run_serving(args, w, ix, qs, docs.rows, mlp, k, kp)
        if ora is not None:
            ora.close()
        if not args.skip_mixed:
            extras["mixed"] = run_mixed(args, dev)
    if world > 1:
        dist.barrier()
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(config_dict(args, w, docs, qs, T,
                                   (st["bytes_lists"] + st["bytes_sketch"]) / 1e9),
                       tuning=tuning,
                       tile_choice_ms=tile_choice,
                       search=("learned per-query Alg. 6 budget and k' (sinn_search_learned "
                               "with a budget-level policy)" if mlp is not None
                               else f"fixed k'={kp}"),
                       search_launch=("one recorded CUDA graph per step (sinn_plan)"
                                      if plan is not None else "direct launches")),
        "roofline": roof,
        "cpu_baseline": extras.get("cpu_baseline"),
        "e2e": extras.get("e2e"),
        "gpu_launches": tm["launches"],
        "clocks": clocks.summary(),
        "recall_at_10": extras.get("recall_at_10"),
        "recall_queries": extras.get("recall_queries"),
        "recall_at_10_fixed_kprime": extras.get("recall_at_10_fixed_kprime"),
        "plain": extras.get("plain"),
        "batched": extras.get("batched"),
        "batched_fixed_kprime": extras.get("batched_fixed_kprime"),
        "learned_kprime": extras.get("learned_kprime"),
        "serving": extras.get("serving"),
        "anytime": extras.get("anytime"),
        "sinnamon_plus": extras.get("sinnamon_plus"),
        "bf16_sketch": extras.get("bf16_sketch"),
        "phases_ms_per_step": {p: v / args.steps for p, v in tm["ms"].items()},
        "index": st,
        "extra": {"mixed": extras.get("mixed"), "plain": extras.get("plain")},
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_mixed(args, dev):
    """The mixed-sign workload (8.8M documents, uniform coordinates, N(0,1)
    values, m = 64, h = 2: both sketch planes read) as an extra line: its
    batched fixed-k' search of 10,000 queries, one-query searches, the
    scorer's roofline, the insert and delete phases of churn steps, and
    recall@10 against the FP64 oracle on a sample."""
    import torch
    from paper_2301_10622_gb300 import sinnamon
    w, docs, pool, qs = make_inputs(args, 0, workload="mixed", n_docs=args.mixed_docs)
    k, kp = w.k, w.k_prime
    ora_job = ex = None
    if not args.skip_oracle:
        # the checker's index builds on one host thread (the C call releases
        # the interpreter lock) while the device part runs
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        oracle.build()
        ex = ThreadPoolExecutor(1)
        ora_job = ex.submit(oracle_index, w, docs)
    t0 = time.time()
    ix = build_index(sinnamon, w, docs, dev, 4096, args.scratch_gb)
    torch.cuda.synchronize()
    t_build = time.time() - t0
    sq = qs.slice(0, min(qs.rows, args.autotune_queries or qs.rows))
    tuning = ix.autotune(sq.indptr.astype(np.int64), sq.indices.astype(np.int32), sq.values,
                         k, kp, reps=1)
    g = (torch.from_numpy(qs.indptr.astype(np.int64)).to(dev),
         torch.from_numpy(qs.indices.astype(np.int32)).to(dev), torch.from_numpy(qs.values).to(dev))
    ids = torch.empty((qs.rows, k), dtype=torch.int32, device=dev)
    sc = torch.empty((qs.rows, k), dtype=torch.float32, device=dev)
    torch.cuda.nvtx.range_push("bench mixed search")  # a profiler can select these launches
    ms = timed_best(lambda: sinnamon.sinn_search(ix.handle, *g, k, kp, ids, sc))
    torch.cuda.nvtx.range_pop()
    sinnamon.sinn_timing_start(ix.handle)
    sinnamon.sinn_search(ix.handle, *g, k, kp, ids, sc)
    torch.cuda.synchronize()
    tm = sinnamon.sinn_timing_stop(ix.handle)
    lens = list_lengths(w, docs)
    P = scored_postings(qs, lens)
    alg = algorithmic_bytes(w, P)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    s_ms = tm["ms"]["score"]
    launches = max(1, tm["spans"]["score"])
    achieved = float(alg.sum()) / (s_ms / 1000.0) / 1e9
    floor = P.astype(np.float64) * (4 + 32 * w.h)   # a 32-byte sector per bin gather
    fl_gbs = float(floor.sum()) / (s_ms / 1000.0) / 1e9
    dr = dram_figures(profile_figures("k_score_emit_mixed"), s_ms / launches, peak,
                      qs.rows / launches, docs.rows)
    out = {"workload": (f"mixed-sign: n={w.n}, {docs.rows} docs, uniform coordinates, nnz/doc "
                        f"uniform 80-160, N(0,1) values; {qs.rows} queries of 40 nnz; "
                        f"m={w.m}, h={w.h}, k={k}, k'={kp}"),
           "qps": qs.rows / (ms / 1000.0), "batch_ms": ms,
           "phases_ms": tm["ms"], "tuning": tuning, "index_build_s": t_build,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "frac_kind": "effective (4 + 4h bytes per "
                        "scored posting over the scoring time)",
                        "sector_floor_gbs": fl_gbs, "sector_floor_frac": fl_gbs / peak,
                        "traffic": dr["traffic"], "dram_frac": dr["dram_frac"],
                        "l1_frac": dr["l1_frac"], "l2_frac": dr["l2_frac"],
                        "sectors_per_request": dr["sectors_per_request"],
                        "kernel": "k_score_emit", "launches": launches,
                        "avg_launch_ms": s_ms / launches,
                        "alg_bytes_per_query": float(alg.mean()),
                        "postings_per_query": float(P.mean())}}
    out["plain"] = plain_search(sinnamon, ix.handle, qs, g[1], g[2], k, kp, dev,
                                min(100, args.plain_queries), alg)
    # streaming churn: steps of `churn` deletes of random live ids and as many
    # inserts (which take the freed ids), timed by phase
    rng = np.random.default_rng(77)
    churn = []
    for si in range(4):
        d = torch.from_numpy(rng.choice(docs.rows, args.churn, replace=False).astype(np.int32))
        part = pool.slice(si * args.churn, (si + 1) * args.churn)
        sinnamon.sinn_timing_start(ix.handle)
        ix.delete(d.to(dev))
        ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
        torch.cuda.synchronize()
        churn.append(sinnamon.sinn_timing_stop(ix.handle)["ms"])
    out["churn"] = {"per_step": args.churn, "steps": len(churn) - 1,
                    "insert_ms": float(np.median([c["insert"] for c in churn[1:]])),
                    "delete_ms": float(np.median([c["delete"] for c in churn[1:]]))}
    if ora_job is not None:
        ora = ora_job.result()
        ex.shutdown()
        nr = min(args.mixed_recall_queries, qs.rows)
        out["recall_at_10"] = recall_at_10(ora, qs.slice(0, nr), ids.cpu().numpy()[:nr],
                                           os.cpu_count() or 1)
        out["recall_queries"] = nr
        ora.close()
    ix.close()
    log(f"mixed: {out}")
    return out


def run_variants(args, w, docs, ix, q, qs, k, kp, mean_postings, ora, tile_docs, truth):
    """The paper's variants, untimed extras: Alg. 6 with an anytime budget
    (half and a quarter of the mean postings per query) on the bench's
    index, and SINNAMON+ (U only) and bfloat16-bin indexes of the same
    collection (``docs``, in id order); each searched with fixed k' as one
    batch, recall against the exact top-10 ``truth`` of the first queries."""
    import torch
    from paper_2301_10622_gb300 import sinnamon
    out = {}

    def timed(index, reps=3):
        """queries/s of the best of `reps` searches after one warm-up"""
        ids = torch.empty((qs.rows, k), dtype=torch.int32, device=q[0].device)
        sc = torch.empty((qs.rows, k), dtype=torch.float32, device=q[0].device)
        sinnamon.sinn_search(index.handle, *q, k, kp, ids, sc)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sinnamon.sinn_search(index.handle, *q, k, kp, ids, sc)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return qs.rows / (best / 1000.0), ids

    nr = min(args.recall_queries, qs.rows)
    runs = []
    for frac in (0.5, 0.25):
        budget = int(mean_postings * frac)
        ix.set_budget(budget)
        qps, ids = timed(ix)
        rec = (recall_at_10(ora, qs.slice(0, nr), ids.cpu().numpy()[:nr], os.cpu_count() or 1,
                            truth) if ora is not None else None)
        runs.append({"budget_postings": budget, "fraction_of_mean_postings": frac,
                     "qps": qps, "k_prime": kp, "recall_at_10": rec})
    ix.set_budget(0)
    out["anytime"] = runs
    plus = sinnamon.Index(w.n, w.m, w.h, device=q[0].device, tile_docs=tile_docs,
                          capacity_hint=docs.rows, scratch_bytes=args.scratch_gb << 30,
                          flags=sinnamon.SINN_FLAG_NONNEG)
    for a in range(0, docs.rows, 200_000):
        part = docs.slice(a, min(docs.rows, a + 200_000))
        plus.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    qps, _ = timed(plus)
    out["sinnamon_plus"] = {"qps": qps, "k_prime": kp, "docs": docs.rows,
                            "bytes_sketch": plus.stats()["bytes_sketch"],
                            "bytes_sketch_full": ix.stats()["bytes_sketch"]}
    plus.close()
    # bfloat16 bins (upper rounded up, lower down)
    bf = sinnamon.Index(w.n, w.m, w.h, device=q[0].device, tile_docs=tile_docs,
                        capacity_hint=docs.rows, scratch_bytes=args.scratch_gb << 30,
                        flags=sinnamon.SINN_FLAG_BF16_SKETCH)
    for a in range(0, docs.rows, 200_000):
        part = docs.slice(a, min(docs.rows, a + 200_000))
        bf.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
    qps, ids = timed(bf)
    rec = None
    if ora is not None:  # the same collection and ids as the bench's index
        rec = recall_at_10(ora, qs.slice(0, nr), ids.cpu().numpy()[:nr], os.cpu_count() or 1,
                           truth)
    out["bf16_sketch"] = {"qps": qps, "k_prime": kp, "docs": docs.rows, "recall_at_10": rec,
                          "bytes_sketch": bf.stats()["bytes_sketch"]}
    bf.close()
    log(f"variants: {out}")
    return out


def run_serving(args, w, ix, qs, n_live, mlp, k, kp):
    """Continuous-batching serving on the bench's index after the timed steps:
    Poisson arrivals of inserts, deletes and queries (rates per second) for
    a fixed wall time; every id below n_live is live at this point (each
    step re-inserted as many vectors as it deleted, into the freed ids)."""
    from paper_2301_10622_gb300 import serving, synth
    r_ins, r_del, r_q = (float(x) for x in args.serve_rates.split(","))
    n_pool = int(r_ins * args.serve_seconds * 1.1) + 64
    spool = cached(f"{w.name}_serve_{n_pool}", lambda: synth.make_docs(w, n_docs=n_pool,
                                                                       seed=5001))
    reqs = serving.poisson_stream(args.serve_seconds, {"insert": r_ins, "delete": r_del,
                                                       "query": r_q}, spool.rows, qs.rows)
    # room for the stream's inserts up front: growing the id capacity or the
    # vector store mid-stream would pause the device
    n_ins = sum(r.kind == "insert" for r in reqs)
    ix.reserve(n_ins + 4096, int(spool.nnz / max(spool.rows, 1) * n_ins * 1.2) + (1 << 16))
    srv = serving.Server(ix, qs, spool, np.arange(n_live), slots=args.serve_slots,
                         slot_bytes=int(args.serve_slot_gb * (1 << 30)), k=k, k_prime=kp,
                         mlp=mlp, kp_max=args.kp_max, mutation_delay=args.serve_delay)
    stats, results, _ = srv.serve(reqs, max_wall=3 * args.serve_seconds + 5)
    stats.update({"rates_per_s": {"insert": r_ins, "delete": r_del, "query": r_q},
                  "seconds": args.serve_seconds, "start_docs": n_live,
                  "learned_kprime": mlp is not None, "mutation_delay_s": args.serve_delay,
                  "mean_kprime": float(np.mean([v[2] for v in results.values()]))
                  if results else None})
    log(f"serving: {stats}")
    return stats


def reconstruct(docs, parts, dels, executed):
    """The collection after the executed steps, in id order.  Every step deleted
    a set of ids and re-inserted as many vectors, which took exactly the freed
    ids in ascending order (smallest free id first)."""
    from paper_2301_10622_gb300.synth import CSR
    src = np.full(docs.rows, -1, np.int64)   # -1: original collection
    srow = np.arange(docs.rows, dtype=np.int64)
    for si in executed:
        d = np.sort(dels[si].cpu().numpy().astype(np.int64))
        src[d] = si
        srow[d] = np.arange(d.size)
    lens = np.diff(docs.indptr.astype(np.int64))[srow] * (src < 0)
    for si in np.unique(src[src >= 0]):
        sel = src == si
        lens[sel] = np.diff(parts[si][3].indptr.astype(np.int64))[srow[sel]]
    ip = np.zeros(docs.rows + 1, np.uint64)
    ip[1:] = np.cumsum(lens)
    idx = np.zeros(int(ip[-1]), np.uint32)
    val = np.zeros(int(ip[-1]), np.float32)
    orig = np.nonzero(src < 0)[0]
    # original rows: vectorised gather
    o_ip = docs.indptr.astype(np.int64)
    starts, cnt = o_ip[srow[orig]], lens[orig]
    gather = np.repeat(starts - np.cumsum(np.concatenate(([0], cnt[:-1]))), cnt) + np.arange(cnt.sum())
    dst = np.repeat(ip[orig].astype(np.int64) - np.cumsum(np.concatenate(([0], cnt[:-1]))), cnt) + np.arange(cnt.sum())
    idx[dst] = docs.indices[gather]
    val[dst] = docs.values[gather]
    for i in np.nonzero(src >= 0)[0]:
        s_ = parts[src[i]][3]
        a_, b_ = int(s_.indptr[srow[i]]), int(s_.indptr[srow[i] + 1])
        idx[int(ip[i]):int(ip[i + 1])] = s_.indices[a_:b_]
        val[int(ip[i]):int(ip[i + 1])] = s_.values[a_:b_]
    return CSR(ip, idx, val)


def arg_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="text")
    ap.add_argument("--docs", type=int, default=0)
    ap.add_argument("--queries", type=int, default=0)
    ap.add_argument("--churn", type=int, default=1000)
    ap.add_argument("--tile-docs", type=int, default=0,
                    help="ids per tile; 0 = chosen by measurement")
    ap.add_argument("--scratch-gb", type=int, default=64,
                    help="search scratch per index; more holds more queries per launch")
    ap.add_argument("--plain-queries", type=int, default=300)
    ap.add_argument("--recall-queries", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-oracle", action="store_true")
    ap.add_argument("--fixed-kprime", action="store_true")
    ap.add_argument("--train-queries", type=int, default=200000)
    ap.add_argument("--cal-queries", type=int, default=2000)
    ap.add_argument("--cal-recall", type=float, default=0.92)
    ap.add_argument("--shifts", default="0,1,2,3,4,5",
                    help="budget levels P_q / 2^s of the learned policy")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--mixed-docs", type=int, default=0)
    ap.add_argument("--mixed-recall-queries", type=int, default=500)
    ap.add_argument("--kp-cap", type=int, default=20000)
    ap.add_argument("--kp-max", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--no-graph", action="store_true", help="launch the search directly")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune-queries", type=int, default=0,
                    help="queries the launch autotuner times; 0 = the whole batch")
    ap.add_argument("--tuning", default="",
                    help="launch tuning fields to set, e.g. array_walk=1,tiles_per_block=2")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rates", default="20000,2000,5000",
                    help="inserts,deletes,queries per second")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-slot-gb", type=float, default=1.0)
    ap.add_argument("--serve-delay", type=float, default=0.005)
    return ap


def main():
    args = arg_parser().parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
