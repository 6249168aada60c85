"""Choice of the index's tile size by measurement.

The run-time launch parameters are tuned inside the library
(`sinn_autotune`); the tile size T is fixed when an index is created, so it
is chosen here: an index of a sample of the collection is built at each
candidate T, its launch parameters are autotuned on a sample of the
queries, and the batched search is timed with CUDA events.  Every step runs
in the library's kernels; this module only builds, times and compares.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sinnamon


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
