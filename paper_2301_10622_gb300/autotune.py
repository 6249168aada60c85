"""Choice of the index's tile size by measurement.

The run-time launch parameters are tuned inside the library
(`sinn_autotune`); the tile size T is fixed when an index is created, so it
is chosen here: an index of a sample of the collection is built at each
candidate T, its launch parameters are autotuned on a sample of the
queries, and the batched search is timed with CUDA events.  Every step runs
in the library's kernels; this module only builds, times and compares.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import sinnamon


def tuning_key(device_name: str, n: int, m: int, h: int, tile_docs: int, docs: int, k: int,
               k_prime: int, flags: int = 0) -> str:
    """The shape a tuning was chosen for: the GPU, the index parameters, its
    size rounded to a power of two, and the search's k and k'."""
    docs_p2 = 1 << max(0, int(docs) - 1).bit_length()
    return (f"{device_name}|n={n}|m={m}|h={h}|T={tile_docs}|flags={flags}|docs~{docs_p2}"
            f"|k={k}|kp={k_prime}")


def cached_tuning(path: str, key: str, tune):
    """The tuning stored under `key` in the JSON file at `path`; if there is
    none, `tune()` chooses one, which is stored (the file is rewritten whole,
    through a temporary file) and returned."""
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    if key in table:
        return dict(table[key]), True
    t = dict(tune())
    table[key] = t
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return t, False


def autotune_cached(ix, queries, k: int, k_prime: int, path: str, reps: int = 2, log=None):
    """Index.autotune on `queries` (CSR), or the tuning cached in `path` for
    this GPU and index shape, which is then set on the index."""
    st = ix.stats()
    key = tuning_key(torch.cuda.get_device_name(ix.device), st["n"], st["m"], st["h"],
                     st["tile_docs"], st["live"], k, k_prime, ix.flags)
    t, hit = cached_tuning(path, key, lambda: ix.autotune(
        queries.indptr.astype(np.int64), queries.indices.astype(np.int32), queries.values,
        k=k, k_prime=k_prime, reps=reps))
    if hit:
        ix.set_tuning(**t)
    if log:
        log(f"tuning {'from cache' if hit else 'measured'} ({key}): {t}")
    return t


def choose_tile_docs(n: int, m: int, h: int, docs, queries, k: int, k_prime: int,
                     candidates=(2048, 4096, 8192), reps: int = 3, device=None,
                     scratch_bytes: int = 4 << 30, log=None):
    """Returns (best T, {T: {"ms": search ms, "tuning": dict}}) for the
    search of `queries` (CSR) over an index of `docs` (CSR)."""
    dev = torch.device(device or "cuda")
    q = (torch.from_numpy(queries.indptr.astype(np.int64)).to(dev),
         torch.from_numpy(queries.indices.astype(np.int32)).to(dev),
         torch.from_numpy(queries.values).to(dev))
    ids = torch.empty((queries.rows, k), dtype=torch.int32, device=dev)
    sc = torch.empty((queries.rows, k), dtype=torch.float32, device=dev)
    results = {}
    for T in candidates:
        ix = sinnamon.Index(n, m, h, device=dev, tile_docs=T, capacity_hint=docs.rows,
                            scratch_bytes=scratch_bytes)
        for a in range(0, docs.rows, 200_000):
            part = docs.slice(a, min(docs.rows, a + 200_000))
            ix.insert(part.indptr.astype(np.int64), part.indices.astype(np.int32), part.values)
        tuning = ix.autotune(*q, k=k, k_prime=k_prime, reps=1)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sinnamon.sinn_search(ix.handle, *q, k, k_prime, ids, sc)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        results[T] = {"ms": best, "tuning": tuning}
        if log:
            log(f"tile {T}: {best:.2f} ms for {queries.rows} queries, tuning {tuning}")
        ix.close()
    return min(results, key=lambda t: results[t]["ms"]), results
