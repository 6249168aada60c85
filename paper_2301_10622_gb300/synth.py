"""Seeded synthetic inputs for SINNAMON workloads.

This module only draws random sparse vectors; it holds none of the method's
arithmetic.  Both the CUDA path and the CPU oracle consume what it returns.

Every collection is returned as CSR: ``indptr`` (uint64, rows+1), ``indices``
(uint32, strictly increasing within a row) and ``values`` (float32).

Distribution readings (the workload descriptions give only the family names):
  * a lognormal count with mean mu and spread sigma: the distribution's mean
    is mu, so the log-space location is ln(mu) - sigma^2/2; draws are rounded
    to the nearest integer and clamped to [1, n].  When sigma is not given it
    is 0.5.
  * lognormal values with parameters (0, s): log-space location 0, scale s.
  * Zipf(s) coordinates: coordinate c (0-based) has weight 1/(c+1)^s; a vector's
    coordinates are drawn one after another without replacement (each draw is
    proportional to the weights of the coordinates not yet taken).
  * uniform coordinates: a uniformly random subset of the given size.
The random generator is numpy's PCG64 seeded with the given seed.  A
collection of more than ``BLOCK_ROWS`` rows is drawn in blocks of that many
rows, block b from its own PCG64 stream (the seed's SeedSequence, child b), on
several threads; the rows do not depend on the number of threads.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BLOCK_ROWS = 1 << 18


@dataclass
class CSR:
    indptr: np.ndarray
    indices: np.ndarray
    values: np.ndarray

    @property
    def rows(self) -> int:
        return int(self.indptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row(self, r: int):
        a, b = int(self.indptr[r]), int(self.indptr[r + 1])
        return self.indices[a:b], self.values[a:b]

    def take(self, rows) -> "CSR":
        rows = np.asarray(rows, dtype=np.int64)
        lens = (self.indptr[rows + 1] - self.indptr[rows]).astype(np.int64)
        ip = np.zeros(rows.size + 1, np.uint64)
        np.cumsum(lens, out=ip[1:])
        idx = np.concatenate([self.indices[int(self.indptr[r]):int(self.indptr[r + 1])]
                              for r in rows]) if rows.size else np.zeros(0, np.uint32)
        val = np.concatenate([self.values[int(self.indptr[r]):int(self.indptr[r + 1])]
                              for r in rows]) if rows.size else np.zeros(0, np.float32)
        return CSR(ip, idx.astype(np.uint32), val.astype(np.float32))

    def slice(self, a: int, b: int) -> "CSR":
        o0, o1 = int(self.indptr[a]), int(self.indptr[b])
        return CSR((self.indptr[a:b + 1] - self.indptr[a]).astype(np.uint64),
                   self.indices[o0:o1], self.values[o0:o1])


def lognormal_counts(rng, size: int, mean: float, sigma: float, n: int) -> np.ndarray:
    mu = np.log(mean) - 0.5 * sigma * sigma
    c = np.rint(rng.lognormal(mu, sigma, size)).astype(np.int64)
    return np.clip(c, 1, n)


def _indptr(counts):
    ip = np.zeros(len(counts) + 1, np.uint64)
    np.cumsum(np.asarray(counts, dtype=np.int64), out=ip[1:])
    return ip


def uniform_coords(rng, counts: np.ndarray, n: int):
    """Per row, a uniformly random set of counts[r] distinct coordinates of [n],
    sorted ascending.  Returns (indptr, indices)."""
    counts = np.asarray(counts, dtype=np.int64)
    ip = _indptr(counts)
    idx = np.zeros(int(ip[-1]), np.uint32)
    for k in np.unique(counts):
        rows = np.nonzero(counts == k)[0]
        for a in range(0, rows.size, 1 << 16):
            blk = rows[a:a + (1 << 16)]
            if 2 * k > n:  # dense rows: permutation prefix
                d = np.argsort(rng.random((blk.size, n)), axis=1)[:, :k]
                d.sort(axis=1)
            else:
                d = rng.integers(0, n, size=(blk.size, k))
                while True:
                    d.sort(axis=1)
                    dup = np.zeros(d.shape, bool)
                    dup[:, 1:] = d[:, 1:] == d[:, :-1]
                    nd = int(dup.sum())
                    if nd == 0:
                        break
                    d[dup] = rng.integers(0, n, size=nd)
            pos = ip[blk].astype(np.int64)[:, None] + np.arange(k)[None, :]
            idx[pos] = d
    return ip, idx


def _alias_table(w: np.ndarray):
    """Vose's alias tables for drawing index i with probability w[i]/sum(w)."""
    n = w.size
    p = w * (n / w.sum())
    prob = np.zeros(n)
    alias = np.zeros(n, np.int64)
    small = [i for i in range(n) if p[i] < 1.0]
    large = [i for i in range(n) if p[i] >= 1.0]
    while small and large:
        s_, l_ = small.pop(), large.pop()
        prob[s_] = p[s_]
        alias[s_] = l_
        p[l_] = p[l_] + p[s_] - 1.0
        (small if p[l_] < 1.0 else large).append(l_)
    for i in small + large:
        prob[i] = 1.0
        alias[i] = i
    return prob, alias


def zipf_coords(rng, counts: np.ndarray, n: int, s: float = 1.0):
    """Per row, counts[r] distinct coordinates drawn one at a time without
    replacement with weight 1/(c+1)^s, returned sorted ascending.  Drawing with
    replacement and skipping values already taken is the same process."""
    counts = np.asarray(counts, dtype=np.int64)
    ip = _indptr(counts)
    idx = np.zeros(int(ip[-1]), np.uint32)
    prob, alias = _alias_table(1.0 / np.power(np.arange(1, n + 1, dtype=np.float64), s))
    order = np.argsort(counts, kind="stable")
    chunk = 1 << 13
    for a in range(0, order.size, chunk):
        todo = order[a:a + chunk]
        draws = int(1.5 * counts[todo].max()) + 32
        while todo.size:
            col = rng.integers(0, n, size=(todo.size, draws))
            d = np.where(rng.random((todo.size, draws)) < prob[col], col, alias[col])
            # first occurrence of each value along the row, in draw order
            srt = np.argsort(d, axis=1, kind="stable")
            ds = np.take_along_axis(d, srt, axis=1)
            first_sorted = np.ones(ds.shape, bool)
            first_sorted[:, 1:] = ds[:, 1:] != ds[:, :-1]
            first = np.zeros(d.shape, bool)
            np.put_along_axis(first, srt, first_sorted, axis=1)
            rank = np.cumsum(first, axis=1)
            need = counts[todo]
            ok = rank[:, -1] >= need
            keep = first & (rank <= need[:, None]) & ok[:, None]
            r_loc, c_loc = np.nonzero(keep)          # row-major: rows ascending
            key = r_loc.astype(np.int64) * n + d[r_loc, c_loc]
            key.sort()
            rows_ok = todo[ok]
            lens = need[ok]
            starts = ip[rows_ok].astype(np.int64)
            offs = np.repeat(starts - np.concatenate(([0], np.cumsum(lens)[:-1])), lens)
            idx[np.arange(key.size) + offs] = (key % n).astype(np.uint32)
            todo = todo[~ok]
            draws *= 2
    return ip, idx


def normal_values(rng, nnz: int, sigma: float = 1.0) -> np.ndarray:
    return rng.normal(0.0, sigma, nnz).astype(np.float32)


def lognormal_values(rng, nnz: int, sigma: float = 0.7) -> np.ndarray:
    return rng.lognormal(0.0, sigma, nnz).astype(np.float32)


# ---------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    n: int
    n_docs: int
    n_queries: int
    m: int
    h: int
    k: int
    k_prime: int
    doc_coords: str          # "uniform" | "zipf"
    doc_nnz: tuple           # ("fixed", v) | ("lognormal", mean, sigma) | ("uniform", lo, hi)
    doc_values: str          # "normal" | "lognormal"
    q_nnz: tuple
    q_values: str
    q_coords: str = ""
    extra: dict = field(default_factory=dict)

    def describe(self) -> str:
        return (f"{self.name}: n={self.n}, docs={self.n_docs}, queries={self.n_queries}, "
                f"m={self.m}, h={self.h}, k={self.k}, k'={self.k_prime}")


WORKLOADS = {
    # tiny plain SINNAMON check
    "tiny": Workload("tiny", n=1000, n_docs=10_000, n_queries=100, m=64, h=1, k=10,
                     k_prime=100, doc_coords="uniform", doc_nnz=("fixed", 32),
                     doc_values="normal", q_nnz=("fixed", 16), q_values="normal",
                     q_coords="uniform"),
    # text-like (SPLADE-shaped) collection: BERT WordPiece vocabulary size
    "text": Workload("text", n=30_522, n_docs=1_000_000, n_queries=10_000, m=128, h=1, k=10,
                     k_prime=1000, doc_coords="zipf", doc_nnz=("lognormal", 120.0, 0.5),
                     doc_values="lognormal", q_nnz=("lognormal", 45.0, 0.5),
                     q_values="lognormal", q_coords="zipf"),
    # mixed-sign real-valued stress collection
    "mixed": Workload("mixed", n=30_000, n_docs=8_800_000, n_queries=10_000, m=64, h=2, k=10,
                      k_prime=2000, doc_coords="uniform", doc_nnz=("uniform", 80, 160),
                      doc_values="normal", q_nnz=("fixed", 40), q_values="normal",
                      q_coords="uniform"),
}


def _counts(rng, spec, rows, n):
    if spec[0] == "fixed":
        return np.full(rows, min(int(spec[1]), n), np.int64)
    if spec[0] == "lognormal":
        return lognormal_counts(rng, rows, spec[1], spec[2], n)
    if spec[0] == "uniform":
        return np.minimum(rng.integers(int(spec[1]), int(spec[2]) + 1, rows), n)
    raise ValueError(spec)


def _fill(rng, counts, n, coords, values):
    if coords == "zipf":
        ip, idx = zipf_coords(rng, counts, n)
    else:
        ip, idx = uniform_coords(rng, counts, n)
    nnz = int(ip[-1])
    val = normal_values(rng, nnz) if values == "normal" else lognormal_values(rng, nnz)
    return ip, idx, val


def _vectors(seed, rows, n, coords, nnz_spec, values):
    if rows <= BLOCK_ROWS:
        rng = np.random.Generator(np.random.PCG64(seed))
        ip, idx, val = _fill(rng, _counts(rng, nnz_spec, rows, n), n, coords, values)
        return CSR(ip, idx, val)
    nb = (rows + BLOCK_ROWS - 1) // BLOCK_ROWS
    rngs = [np.random.Generator(np.random.PCG64(c))
            for c in np.random.SeedSequence(seed).spawn(nb)]
    counts = [_counts(rngs[b], nnz_spec, min(BLOCK_ROWS, rows - b * BLOCK_ROWS), n)
              for b in range(nb)]
    ip = _indptr(np.concatenate(counts))
    idx = np.empty(int(ip[-1]), np.uint32)
    val = np.empty(int(ip[-1]), np.float32)

    def block(b):
        _, bi, bv = _fill(rngs[b], counts[b], n, coords, values)
        o = int(ip[b * BLOCK_ROWS])
        idx[o:o + bi.size] = bi
        val[o:o + bv.size] = bv

    with ThreadPoolExecutor(max(1, min(nb, os.cpu_count() or 1))) as ex:
        list(ex.map(block, range(nb)))
    return CSR(ip, idx, val)


def make_docs(w: Workload, n_docs: int | None = None, seed: int | None = None) -> CSR:
    """Documents of workload w (seed default: 1000 + workload number)."""
    rows = w.n_docs if n_docs is None else n_docs
    return _vectors(_seed(w, 1000) if seed is None else seed, rows, w.n, w.doc_coords,
                    w.doc_nnz, w.doc_values)


def make_queries(w: Workload, n_q: int | None = None, seed: int | None = None) -> CSR:
    """Queries of workload w (seed default: 2000 + workload number)."""
    rows = w.n_queries if n_q is None else n_q
    return _vectors(_seed(w, 2000) if seed is None else seed, rows, w.n,
                    w.q_coords or w.doc_coords, w.q_nnz, w.q_values)


def _seed(w: Workload, base: int) -> int:
    return base + {"tiny": 1, "text": 2, "mixed": 3}.get(w.name, 9)


def scaled(w: Workload, n_docs: int, n_queries: int | None = None, **over) -> Workload:
    """The same workload shape with fewer documents/queries (parity-test sizes)."""
    d = dict(w.__dict__)
    d.update(n_docs=n_docs, n_queries=n_queries or w.n_queries, **over)
    return Workload(**d)
