"""CPU oracle for SINNAMON: plain C, FP64, written from the paper's algorithms.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and the library never calls it.

What each wrapper follows (all in ``sinn_oracle.c``):
  * ``OracleIndex.insert``   -- Alg. 5 (indexing) with the id reuse of Sec. 4.3.
  * ``OracleIndex.delete``   -- Sec. 4.3 (deletion).
  * ``OracleIndex.scores``   -- Alg. 6 (scoring), T = infinity.
  * ``OracleIndex.search``   -- Alg. 7 (ranking) over Alg. 6, FindLargest = Alg. 3.
  * ``OracleIndex.exact_topk`` -- Eq. 2 (exact MIPS) by brute force.
  * ``OracleIndex.linscan_topk`` -- Alg. 1 / Alg. 2 (LinScan), exact.
  * ``mix64`` / ``hash_table`` -- the h random mappings of Alg. 5, read as
    SplitMix64's output function of (seed ^ (o+1)*gamma ^ j), reduced mod m.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sinn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

OK, EINVAL, ENOTFOUND, ENOMEM = 0, 1, 2, 3

u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.orc_mix64.restype = C.c_uint64
        lib.orc_mix64.argtypes = [C.c_uint64]
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64]
        lib.orc_create_table.restype = vp
        lib.orc_create_table.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, u32p]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_hash_table.argtypes = [vp, u32p]
        lib.orc_n_slots.restype = C.c_uint32
        lib.orc_n_slots.argtypes = [vp]
        lib.orc_live_count.restype = C.c_uint32
        lib.orc_live_count.argtypes = [vp]
        lib.orc_is_live.restype = C.c_int
        lib.orc_is_live.argtypes = [vp, C.c_uint32]
        lib.orc_live_mask.argtypes = [vp, vp]
        lib.orc_insert.restype = C.c_int
        lib.orc_insert.argtypes = [vp, u64p, u32p, f32p, C.c_uint32, u32p]
        lib.orc_delete.restype = C.c_int
        lib.orc_delete.argtypes = [vp, u32p, C.c_uint32]
        lib.orc_sketch_column.argtypes = [vp, C.c_uint32, f64p, f64p]
        lib.orc_list_len.restype = C.c_uint32
        lib.orc_list_len.argtypes = [vp, C.c_uint32]
        lib.orc_list.argtypes = [vp, C.c_uint32, u32p]
        lib.orc_doc_nnz.restype = C.c_uint32
        lib.orc_doc_nnz.argtypes = [vp, C.c_uint32]
        lib.orc_doc.argtypes = [vp, C.c_uint32, u32p, f64p]
        lib.orc_set_sketch_bf16.restype = C.c_int
        lib.orc_set_sketch_bf16.argtypes = [vp, C.c_int]
        lib.orc_scores.restype = C.c_int
        lib.orc_scores.argtypes = [vp, u32p, f32p, C.c_uint32, f64p, vp]
        lib.orc_scores_anytime.restype = C.c_int
        lib.orc_scores_anytime.argtypes = [vp, u32p, f32p, C.c_uint32, C.c_uint64, f64p, vp]
        lib.orc_exact_scores.restype = C.c_int
        lib.orc_exact_scores.argtypes = [vp, u32p, f32p, C.c_uint32, f64p, vp]
        lib.orc_search.restype = C.c_int
        lib.orc_search.argtypes = [vp, u64p, u32p, f32p, C.c_uint32, C.c_uint32, C.c_uint32,
                                   u32p, f64p, vp, vp, vp, u32p, C.c_uint32]
        lib.orc_search_anytime.restype = C.c_int
        lib.orc_search_anytime.argtypes = [vp, u64p, u32p, f32p, C.c_uint32, C.c_uint32,
                                           C.c_uint32, C.c_uint64, u32p, f64p, vp, vp, vp,
                                           u32p, C.c_uint32]
        lib.orc_exact_topk.restype = C.c_int
        lib.orc_exact_topk.argtypes = [vp, u64p, u32p, f32p, C.c_uint32, C.c_uint32, u32p,
                                       f64p, vp, u32p, C.c_uint32]
        lib.orc_find_largest.restype = C.c_uint32
        lib.orc_find_largest.argtypes = [f64p, C.c_uint32, C.c_uint32, u32p, f64p]
        lib.orc_linscan_build.restype = vp
        lib.orc_linscan_build.argtypes = [vp]
        lib.orc_linscan_destroy.argtypes = [vp]
        lib.orc_linscan_topk.restype = C.c_int
        lib.orc_linscan_topk.argtypes = [vp, u64p, u32p, f32p, C.c_uint32, C.c_uint32, u32p,
                                         f64p, C.c_uint32]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def mix64(x: int) -> int:
    """SplitMix64's output function applied to the 64-bit word x."""
    return int(_load().orc_mix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def find_largest(values, k: int):
    """Alg. 3 on its own: the k largest (value, index) pairs, larger value first,
    equal values by smaller index.  Returns (indices, values)."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    keys = np.zeros(max(k, 1), np.uint32)
    vals = np.zeros(max(k, 1), np.float64)
    r = _load().orc_find_largest(v, v.size, k, keys, vals)
    return keys[:r].copy(), vals[:r].copy()


def _csr(indptr, indices, values):
    return (np.ascontiguousarray(indptr, dtype=np.uint64),
            np.ascontiguousarray(indices, dtype=np.uint32),
            np.ascontiguousarray(values, dtype=np.float32))


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__({EINVAL: "invalid argument", ENOTFOUND: "id not live",
                          ENOMEM: "out of memory"}.get(code, f"error {code}"))
        self.code = code


class OracleIndex:
    """A SINNAMON index held by the CPU oracle (FP64)."""

    def __init__(self, n: int, m: int, h: int, seed: int = 0x5151, table=None,
                 sketch_bf16: bool = False):
        lib = _load()
        self.n, self.m, self.h = n, m, h
        if table is None:
            self._p = lib.orc_create(n, m, h, seed)
        else:
            t = np.ascontiguousarray(table, dtype=np.uint32).reshape(-1)
            if t.size != n * h:
                raise ValueError("table must hold n*h entries")
            self._p = lib.orc_create_table(n, m, h, t)
        if not self._p:
            raise OracleError(EINVAL)
        self._lib = lib
        if sketch_bf16 and lib.orc_set_sketch_bf16(self._p, 1):
            raise OracleError(EINVAL)

    def close(self):
        if getattr(self, "_p", None):
            self._lib.orc_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state
    @property
    def n_slots(self) -> int:
        return int(self._lib.orc_n_slots(self._p))

    @property
    def live_count(self) -> int:
        return int(self._lib.orc_live_count(self._p))

    def is_live(self, i: int) -> bool:
        return bool(self._lib.orc_is_live(self._p, i))

    def live_mask(self) -> np.ndarray:
        out = np.zeros(max(self.n_slots, 1), np.uint8)
        self._lib.orc_live_mask(self._p, _ptr(out))
        return out[: self.n_slots].astype(bool)

    def live_ids(self) -> np.ndarray:
        return np.nonzero(self.live_mask())[0].astype(np.uint32)

    def hash_table(self) -> np.ndarray:
        out = np.zeros(self.n * self.h, np.uint32)
        self._lib.orc_hash_table(self._p, out)
        return out.reshape(self.n, self.h)

    def sketch_column(self, i: int):
        u = np.zeros(self.m, np.float64)
        l = np.zeros(self.m, np.float64)
        self._lib.orc_sketch_column(self._p, i, u, l)
        return u, l

    def inverted_list(self, j: int) -> np.ndarray:
        n = self._lib.orc_list_len(self._p, j)
        out = np.zeros(max(n, 1), np.uint32)
        if n:
            self._lib.orc_list(self._p, j, out)
        return out[:n].copy()

    def doc(self, i: int):
        n = self._lib.orc_doc_nnz(self._p, i)
        idx = np.zeros(max(n, 1), np.uint32)
        val = np.zeros(max(n, 1), np.float64)
        if n:
            self._lib.orc_doc(self._p, i, idx, val)
        return idx[:n].copy(), val[:n].copy()

    # ---- mutation
    def insert(self, indptr, indices, values) -> np.ndarray:
        ip, ix, vv = _csr(indptr, indices, values)
        nd = ip.size - 1
        out = np.zeros(max(nd, 1), np.uint32)
        st = self._lib.orc_insert(self._p, ip, ix, vv, nd, out)
        if st:
            raise OracleError(st)
        return out[:nd].copy()

    def delete(self, ids):
        a = np.ascontiguousarray(ids, dtype=np.uint32)
        st = self._lib.orc_delete(self._p, a, a.size)
        if st:
            raise OracleError(st)

    # ---- queries
    def scores(self, qi, qv, with_magnitude: bool = False, budget: int = 0):
        """Alg. 6 scores of every id slot; budget > 0: the anytime break after
        the term at which the postings visited reach the budget."""
        qi = np.ascontiguousarray(qi, dtype=np.uint32)
        qv = np.ascontiguousarray(qv, dtype=np.float32)
        out = np.zeros(max(self.n_slots, 1), np.float64)
        mag = np.zeros(max(self.n_slots, 1), np.float64) if with_magnitude else None
        st = self._lib.orc_scores_anytime(self._p, qi, qv, qi.size, budget, out, _ptr(mag))
        if st:
            raise OracleError(st)
        out = out[: self.n_slots]
        return (out, mag[: self.n_slots]) if with_magnitude else out

    def exact_scores(self, qi, qv, with_magnitude: bool = False):
        qi = np.ascontiguousarray(qi, dtype=np.uint32)
        qv = np.ascontiguousarray(qv, dtype=np.float32)
        out = np.zeros(max(self.n_slots, 1), np.float64)
        mag = np.zeros(max(self.n_slots, 1), np.float64) if with_magnitude else None
        st = self._lib.orc_exact_scores(self._p, qi, qv, qi.size, out, _ptr(mag))
        if st:
            raise OracleError(st)
        out = out[: self.n_slots]
        return (out, mag[: self.n_slots]) if with_magnitude else out

    def search(self, indptr, indices, values, k: int, k_prime: int, threads: int = 1,
               candidates: bool = False, budget: int = 0):
        """Alg. 6 + Alg. 7.  Returns dict with ids/scores [nq, k] and, when
        asked, cand_ids/cand_scores/cand_mag [nq, k'] (approximate scores)."""
        ip, ix, vv = _csr(indptr, indices, values)
        nq = ip.size - 1
        ids = np.zeros((max(nq, 1), k), np.uint32)
        sc = np.zeros((max(nq, 1), k), np.float64)
        cnt = np.zeros(max(nq, 1), np.uint32)
        ci = cs = cm = None
        if candidates:
            ci = np.full((max(nq, 1), k_prime), 0xFFFFFFFF, np.uint32)
            cs = np.full((max(nq, 1), k_prime), -np.inf, np.float64)
            cm = np.zeros((max(nq, 1), k_prime), np.float64)
        st = self._lib.orc_search_anytime(self._p, ip, ix, vv, nq, k, k_prime, budget, ids, sc,
                                          _ptr(ci), _ptr(cs), _ptr(cm), cnt, threads)
        if st:
            raise OracleError(st)
        res = {"ids": ids[:nq], "scores": sc[:nq], "count": cnt[:nq]}
        if candidates:
            res.update(cand_ids=ci[:nq], cand_scores=cs[:nq], cand_mag=cm[:nq])
        return res

    def search_per_query(self, indptr, indices, values, k: int, k_primes, budgets,
                         candidates: bool = False):
        """Alg. 6 + Alg. 7 with query r's own k' (k_primes[r]) and anytime
        budget (budgets[r] postings, 0 = none): one oracle search per query
        (small cases).  Candidate rows are padded to the largest k'."""
        ip = np.asarray(indptr, np.uint64)
        nq = ip.size - 1
        kpm = int(max(k_primes)) if nq else k
        ids = np.zeros((nq, k), np.uint32)
        sc = np.zeros((nq, k), np.float64)
        cnt = np.zeros(nq, np.uint32)
        ci = np.full((nq, kpm), 0xFFFFFFFF, np.uint32)
        cs = np.full((nq, kpm), -np.inf, np.float64)
        cm = np.zeros((nq, kpm), np.float64)
        for r in range(nq):
            a, b = int(ip[r]), int(ip[r + 1])
            one = self.search(np.array([0, b - a], np.uint64), indices[a:b], values[a:b], k=k,
                              k_prime=int(k_primes[r]), candidates=candidates,
                              budget=int(budgets[r]))
            ids[r], sc[r], cnt[r] = one["ids"][0], one["scores"][0], one["count"][0]
            if candidates:
                kp = int(k_primes[r])
                ci[r, :kp], cs[r, :kp], cm[r, :kp] = (one["cand_ids"][0], one["cand_scores"][0],
                                                      one["cand_mag"][0])
        res = {"ids": ids, "scores": sc, "count": cnt}
        if candidates:
            res.update(cand_ids=ci, cand_scores=cs, cand_mag=cm)
        return res

    def query_postings(self, qi, qv) -> int:
        """Postings Alg. 6 visits with no budget: the sum of |I[j]| (live ids)
        over the query's non-zeros."""
        return int(sum(self.inverted_list(int(j)).size for j, v in zip(qi, qv) if v != 0))

    def exact_topk(self, indptr, indices, values, k: int, threads: int = 1):
        ip, ix, vv = _csr(indptr, indices, values)
        nq = ip.size - 1
        ids = np.zeros((max(nq, 1), k), np.uint32)
        sc = np.zeros((max(nq, 1), k), np.float64)
        mag = np.zeros((max(nq, 1), k), np.float64)
        cnt = np.zeros(max(nq, 1), np.uint32)
        st = self._lib.orc_exact_topk(self._p, ip, ix, vv, nq, k, ids, sc, _ptr(mag), cnt,
                                      threads)
        if st:
            raise OracleError(st)
        return {"ids": ids[:nq], "scores": sc[:nq], "mag": mag[:nq], "count": cnt[:nq]}

    def linscan_topk(self, indptr, indices, values, k: int, threads: int = 1):
        ip, ix, vv = _csr(indptr, indices, values)
        nq = ip.size - 1
        ls = self._lib.orc_linscan_build(self._p)
        try:
            ids = np.zeros((max(nq, 1), k), np.uint32)
            sc = np.zeros((max(nq, 1), k), np.float64)
            st = self._lib.orc_linscan_topk(ls, ip, ix, vv, nq, k, ids, sc, threads)
            if st:
                raise OracleError(st)
        finally:
            self._lib.orc_linscan_destroy(ls)
        return {"ids": ids[:nq], "scores": sc[:nq]}
