"""Python binding of the SINNAMON C ABI (include/sinnamon.h).

Argument marshalling only: every step of insertion, deletion and search runs in
the CUDA library ``libsinnamon.so``.  The functions keep the C names; tensors
are PyTorch CUDA tensors of the index's device (device pointers of the C ABI)
unless a name says ``host``.  Unsigned C types travel in signed torch dtypes of
the same width: indptr int64, coordinates and ids int32 (id 0xFFFFFFFF, the
padding of short result rows, reads as -1).

Importing this module loads the library and fails loudly if it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

(SINN_OK, SINN_EINVAL, SINN_ENOTFOUND, SINN_ENOMEM, SINN_ECUDA, SINN_EDEVICE, SINN_ESCRATCH,
 SINN_EIO, SINN_EBUSY) = range(9)
SINN_SEQ_LATEST = 0xFFFFFFFE
SINN_FLAG_NONNEG = 1
SINN_FLAG_BF16_SKETCH = 2

# every symbol declared in include/sinnamon.h
EXPORTS = [
    "sinn_create", "sinn_create_ex", "sinn_destroy", "sinn_insert", "sinn_delete",
    "sinn_search", "sinn_search_kp", "sinn_search_host", "sinn_sync", "sinn_stats",
    "sinn_strerror", "sinn_hash_table", "sinn_sketch_columns", "sinn_inverted_list",
    "sinn_scores", "sinn_candidates", "sinn_timing_start", "sinn_timing_stop",
    "sinn_search_noalloc", "sinn_ctx_create", "sinn_ctx_destroy", "sinn_ctx_query_bytes",
    "sinn_search_ctx", "sinn_get_tuning", "sinn_set_tuning", "sinn_autotune",
    "sinn_set_budget", "sinn_get_budget", "sinn_save", "sinn_load", "sinn_debug_fail_alloc",
    "sinn_debug_wait_probe", "sinn_search_kpb", "sinn_candidates_kpb", "sinn_query_postings",
    "sinn_insert_at", "sinn_delete_at", "sinn_reclaim", "sinn_ctx_set_snapshot",
    "sinn_reserve",
    # sinnamon_kprime.h
    "sinn_kp_features", "sinn_mlp_create", "sinn_mlp_destroy", "sinn_mlp_num_params",
    "sinn_mlp_params", "sinn_mlp_set_params", "sinn_mlp_set_normalizer", "sinn_mlp_forward",
    "sinn_mlp_grad", "sinn_mlp_train_step", "sinn_search_learned", "sinn_mlp_act_bytes",
    "sinn_search_learned_ctx", "sinn_mlp_sync", "sinn_mlp_set_policy", "sinn_mlp_get_policy",
    "sinn_kp_choose", "sinn_search_learned_host",
    # sinnamon_plan.h
    "sinn_plan_create", "sinn_plan_run", "sinn_plan_recordings", "sinn_plan_destroy",
]

KP_FEATURES = 19
KP_MAX_LEVELS = 8


class SinnKpPolicy(C.Structure):
    _fields_ = [("n_levels", C.c_uint32), ("shift", C.c_uint32 * KP_MAX_LEVELS),
                ("posting_cost", C.c_float), ("margin", C.c_float)]

    def as_dict(self):
        return {"shifts": [int(self.shift[i]) for i in range(self.n_levels)],
                "posting_cost": float(self.posting_cost), "margin": float(self.margin)}

PHASES = ["prep", "score", "select", "rerank", "insert", "delete"]


class SinnConfig(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint32), ("h", C.c_uint32),
                ("tile_docs", C.c_uint32), ("seed", C.c_uint64), ("capacity_hint", C.c_uint64),
                ("table", C.c_void_p), ("max_query_nnz", C.c_uint32), ("flags", C.c_uint32),
                ("scratch_bytes", C.c_uint64)]


class SinnStats(C.Structure):
    _fields_ = [("live", C.c_uint64), ("capacity", C.c_uint64), ("next_id", C.c_uint64),
                ("postings", C.c_uint64), ("tombstones", C.c_uint64),
                ("bytes_lists", C.c_uint64), ("bytes_sketch", C.c_uint64),
                ("bytes_store", C.c_uint64), ("bytes_scratch", C.c_uint64),
                ("n", C.c_uint32), ("m", C.c_uint32), ("h", C.c_uint32),
                ("tile_docs", C.c_uint32), ("flags", C.c_uint32),
                ("pending_deletes", C.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SinnTiming(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("spans", C.c_uint64 * 6), ("launches", C.c_uint64)]

    def as_dict(self):
        return {"ms": {p: self.ms[i] for i, p in enumerate(PHASES)},
                "spans": {p: int(self.spans[i]) for i, p in enumerate(PHASES)},
                "launches": int(self.launches)}


class SinnTuning(C.Structure):
    _fields_ = [("bound_every", C.c_uint32), ("emit_min_batch", C.c_uint32),
                ("max_batch", C.c_uint32), ("rerank_blocks", C.c_uint32),
                ("dense_blocks_per_sm", C.c_uint32), ("tiles_per_block", C.c_uint32),
                ("persistent_blocks_per_sm", C.c_uint32), ("array_walk", C.c_uint32)]
    FIELDS = ["bound_every", "emit_min_batch", "max_batch", "rerank_blocks",
              "dense_blocks_per_sm", "tiles_per_block", "persistent_blocks_per_sm",
              "array_walk"]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in self.FIELDS}


class SinnError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        msg = _LIB.sinn_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")
        self.code = code


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsinnamon.so (raises if it is missing and not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"libsinnamon.so is not built ({path}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
    sig = {
        "sinn_create": ([u32, u32, u32, C.POINTER(vp)], C.c_int),
        "sinn_create_ex": ([C.POINTER(SinnConfig), C.POINTER(vp)], C.c_int),
        "sinn_destroy": ([vp], C.c_int),
        "sinn_insert": ([vp, vp, vp, vp, u32, vp, vp], C.c_int),
        "sinn_delete": ([vp, vp, u32, vp], C.c_int),
        "sinn_search": ([vp, vp, vp, vp, u32, u32, u32, vp, vp, vp], C.c_int),
        "sinn_search_kp": ([vp, vp, vp, vp, u32, u32, vp, u32, vp, vp, vp], C.c_int),
        "sinn_search_host": ([vp, vp, vp, vp, u32, u32, u32, vp, vp, vp], C.c_int),
        "sinn_sync": ([vp, vp], C.c_int),
        "sinn_stats": ([vp, C.POINTER(SinnStats)], C.c_int),
        "sinn_strerror": ([C.c_int], C.c_char_p),
        "sinn_hash_table": ([vp, vp], C.c_int),
        "sinn_sketch_columns": ([vp, vp, u32, vp, vp, vp], C.c_int),
        "sinn_inverted_list": ([vp, u32, vp, u64, C.POINTER(u64)], C.c_int),
        "sinn_scores": ([vp, vp, vp, vp, u32, vp, vp], C.c_int),
        "sinn_candidates": ([vp, vp, vp, vp, u32, u32, vp, vp, vp, vp], C.c_int),
        "sinn_timing_start": ([vp], C.c_int),
        "sinn_search_noalloc": ([vp, vp, vp, vp, u32, u32, u32, vp, vp, vp], C.c_int),
        "sinn_kp_features": ([vp, vp, vp, vp, u32, vp, vp], C.c_int),
        "sinn_ctx_create": ([vp, u64, C.POINTER(vp)], C.c_int),
        "sinn_ctx_destroy": ([vp], C.c_int),
        "sinn_ctx_query_bytes": ([vp, u32], u64),
        "sinn_search_ctx": ([vp, vp, vp, vp, u32, u32, vp, u32, vp, vp, vp], C.c_int),
        "sinn_mlp_act_bytes": ([vp, u32], u64),
        "sinn_search_learned_ctx": ([vp, vp, vp, vp, u64, vp, vp, vp, u32, u32, u32, u32, vp, vp,
                                     vp, vp], C.c_int),
        "sinn_mlp_create": ([u32, u32, u64, C.POINTER(vp)], C.c_int),
        "sinn_mlp_destroy": ([vp], C.c_int),
        "sinn_mlp_num_params": ([vp], u64),
        "sinn_mlp_params": ([vp, vp, C.c_int], C.c_int),
        "sinn_mlp_set_params": ([vp, vp], C.c_int),
        "sinn_mlp_set_normalizer": ([vp, vp, vp], C.c_int),
        "sinn_mlp_forward": ([vp, vp, u32, vp, vp], C.c_int),
        "sinn_mlp_grad": ([vp, vp, vp, u32, C.c_float, vp, vp, vp], C.c_int),
        "sinn_mlp_train_step": ([vp, vp, vp, u32, C.c_float, C.c_float, vp, vp], C.c_int),
        "sinn_search_learned": ([vp, vp, vp, vp, vp, u32, u32, u32, u32, vp, vp, vp, vp],
                                C.c_int),
        "sinn_timing_stop": ([vp, C.POINTER(SinnTiming)], C.c_int),
        "sinn_plan_create": ([vp, vp, vp, vp, vp, vp, u32, u32, u32, u32, vp, vp, vp, u64,
                              C.POINTER(vp)], C.c_int),
        "sinn_plan_run": ([vp, vp], C.c_int),
        "sinn_plan_recordings": ([vp], u64),
        "sinn_plan_destroy": ([vp], C.c_int),
        "sinn_get_tuning": ([vp, C.POINTER(SinnTuning)], C.c_int),
        "sinn_set_budget": ([vp, u64], C.c_int),
        "sinn_get_budget": ([vp], u64),
        "sinn_debug_fail_alloc": ([C.c_int64], C.c_int),
        "sinn_save": ([vp, C.c_char_p], C.c_int),
        "sinn_load": ([C.c_char_p, C.POINTER(vp)], C.c_int),
        "sinn_debug_wait_probe": ([u32, C.c_int, vp], C.c_int),
        "sinn_mlp_sync": ([vp, vp], C.c_int),
        "sinn_set_tuning": ([vp, C.POINTER(SinnTuning)], C.c_int),
        "sinn_autotune": ([vp, vp, vp, vp, u32, u32, u32, u32, C.POINTER(SinnTuning), vp],
                          C.c_int),
        "sinn_search_kpb": ([vp, vp, vp, vp, u32, u32, vp, u32, vp, vp, vp, vp], C.c_int),
        "sinn_insert_at": ([vp, vp, vp, vp, u32, vp, u32, vp], C.c_int),
        "sinn_delete_at": ([vp, vp, u32, u32, vp], C.c_int),
        "sinn_reclaim": ([vp, u32, vp], C.c_int),
        "sinn_reserve": ([vp, u64, u64], C.c_int),
        "sinn_ctx_set_snapshot": ([vp, u32], C.c_int),
        "sinn_candidates_kpb": ([vp, vp, vp, vp, u32, u32, vp, vp, vp, vp, vp], C.c_int),
        "sinn_query_postings": ([vp, vp, vp, vp, u32, vp, vp], C.c_int),
        "sinn_mlp_set_policy": ([vp, C.POINTER(SinnKpPolicy)], C.c_int),
        "sinn_mlp_get_policy": ([vp, C.POINTER(SinnKpPolicy)], C.c_int),
        "sinn_kp_choose": ([vp, vp, vp, vp, vp, u32, u32, u32, vp, vp, vp], C.c_int),
        "sinn_search_learned_host": ([vp, vp, vp, vp, vp, u32, u32, u32, u32, vp, vp, vp, vp],
                                     C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _check(code: int, where: str):
    if code != SINN_OK:
        raise SinnError(code, where)


def _p(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return C.c_void_p(t.data_ptr()) if t.numel() else C.c_void_p(t.data_ptr() or 0)
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    raise TypeError(type(t))


def _s(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t, dtype, device):
    t = torch.as_tensor(t)
    if t.dtype != dtype:
        t = t.to(dtype)
    return t.to(device).contiguous()


# ------------------------------------------------------------ C-named calls

def sinn_create(n: int, m: int, h: int):
    lib = load()
    out = C.c_void_p()
    _check(lib.sinn_create(n, m, h, C.byref(out)), "sinn_create")
    return out


def sinn_create_ex(n: int, m: int, h: int, tile_docs: int = 0, seed: int = 0,
                   capacity_hint: int = 0, table=None, max_query_nnz: int = 0,
                   scratch_bytes: int = 0, flags: int = 0):
    lib = load()
    cfg = SinnConfig(n=n, m=m, h=h, tile_docs=tile_docs, seed=seed,
                     capacity_hint=capacity_hint, max_query_nnz=max_query_nnz,
                     scratch_bytes=scratch_bytes, flags=flags)
    keep = None
    if table is not None:
        keep = np.ascontiguousarray(np.asarray(table, dtype=np.uint32).reshape(-1))
        cfg.table = keep.ctypes.data
    out = C.c_void_p()
    _check(lib.sinn_create_ex(C.byref(cfg), C.byref(out)), "sinn_create_ex")
    return out


def sinn_destroy(ix):
    _check(load().sinn_destroy(ix), "sinn_destroy")


def sinn_insert(ix, indptr, indices, values, out_ids, stream=None):
    n_docs = indptr.numel() - 1
    _check(load().sinn_insert(ix, _p(indptr), _p(indices), _p(values), n_docs, _p(out_ids),
                              _s(stream)), "sinn_insert")
    return out_ids


def sinn_delete(ix, ids, stream=None):
    _check(load().sinn_delete(ix, _p(ids), ids.numel(), _s(stream)), "sinn_delete")


def sinn_insert_at(ix, indptr, indices, values, out_ids, seq, stream=None):
    n_docs = indptr.numel() - 1
    _check(load().sinn_insert_at(ix, _p(indptr), _p(indices), _p(values), n_docs, _p(out_ids),
                                 int(seq), _s(stream)), "sinn_insert_at")
    return out_ids


def sinn_delete_at(ix, ids, seq, stream=None):
    _check(load().sinn_delete_at(ix, _p(ids), ids.numel(), int(seq), _s(stream)),
           "sinn_delete_at")


def sinn_reclaim(ix, horizon, stream=None):
    _check(load().sinn_reclaim(ix, int(horizon), _s(stream)), "sinn_reclaim")


def sinn_reserve(ix, more_ids, more_entries):
    _check(load().sinn_reserve(ix, int(more_ids), int(more_entries)), "sinn_reserve")


def sinn_search(ix, q_indptr, q_indices, q_values, k, k_prime, out_ids, out_scores,
                stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_search(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k, k_prime,
                              _p(out_ids), _p(out_scores), _s(stream)), "sinn_search")


def sinn_search_kp(ix, q_indptr, q_indices, q_values, k, k_prime, k_prime_max, out_ids,
                   out_scores, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_search_kp(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k,
                                 _p(k_prime), k_prime_max, _p(out_ids), _p(out_scores),
                                 _s(stream)), "sinn_search_kp")


def sinn_search_kpb(ix, q_indptr, q_indices, q_values, k, k_prime, k_prime_max, budget,
                    out_ids, out_scores, stream=None):
    """Per-query k' (int32 tensor or None) and per-query Alg. 6 budget in
    postings (int64 tensor or None)."""
    n_q = q_indptr.numel() - 1
    _check(load().sinn_search_kpb(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k,
                                  _p(k_prime), k_prime_max, _p(budget), _p(out_ids),
                                  _p(out_scores), _s(stream)), "sinn_search_kpb")


def sinn_candidates_kpb(ix, q_indptr, q_indices, q_values, k_prime, budget, out_ids, out_scores,
                        out_count, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_candidates_kpb(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q,
                                      k_prime, _p(budget), _p(out_ids), _p(out_scores),
                                      _p(out_count), _s(stream)), "sinn_candidates_kpb")


def sinn_query_postings(ix, q_indptr, q_indices, q_values, out, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_query_postings(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q,
                                      _p(out), _s(stream)), "sinn_query_postings")


def sinn_mlp_set_policy(mlp, shifts=None, posting_cost: float = 0.0, margin: float = 0.0):
    """shifts None clears the policy."""
    if shifts is None:
        _check(load().sinn_mlp_set_policy(mlp, None), "sinn_mlp_set_policy")
        return
    if not 0 < len(shifts) <= KP_MAX_LEVELS:
        raise SinnError(SINN_EINVAL, "sinn_mlp_set_policy")
    pol = SinnKpPolicy(n_levels=len(shifts), posting_cost=posting_cost, margin=margin)
    for i, v in enumerate(shifts):
        if not 0 <= int(v) < 2 ** 32:
            raise SinnError(SINN_EINVAL, "sinn_mlp_set_policy")
        pol.shift[i] = int(v)
    _check(load().sinn_mlp_set_policy(mlp, C.byref(pol)), "sinn_mlp_set_policy")


def sinn_mlp_get_policy(mlp) -> dict:
    pol = SinnKpPolicy()
    _check(load().sinn_mlp_get_policy(mlp, C.byref(pol)), "sinn_mlp_get_policy")
    return pol.as_dict()


def sinn_kp_choose(ix, mlp, q_indptr, q_indices, q_values, kp_min, kp_max, out_kprime,
                   out_budget, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_kp_choose(ix, mlp, _p(q_indptr), _p(q_indices), _p(q_values), n_q,
                                 kp_min, kp_max, _p(out_kprime), _p(out_budget), _s(stream)),
           "sinn_kp_choose")


def sinn_search_learned_host(ix, mlp, q_indptr, q_indices, q_values, k, kp_min, kp_max,
                             out_ids, out_scores, out_kprime=None, stream=None):
    """All buffers host (numpy arrays or CPU tensors); waits for completion."""
    n_q = (q_indptr.numel() if isinstance(q_indptr, torch.Tensor) else q_indptr.size) - 1
    _check(load().sinn_search_learned_host(ix, mlp, _p(q_indptr), _p(q_indices), _p(q_values),
                                           n_q, k, kp_min, kp_max, _p(out_ids), _p(out_scores),
                                           _p(out_kprime), _s(stream)),
           "sinn_search_learned_host")


def sinn_search_noalloc(ix, q_indptr, q_indices, q_values, k, k_prime, out_ids, out_scores,
                        stream=None):
    """sinn_search with its scratch in the library's fixed device array: no
    allocation happens during the call (for callers that cannot allocate)."""
    n_q = q_indptr.numel() - 1
    _check(load().sinn_search_noalloc(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k,
                                      k_prime, _p(out_ids), _p(out_scores), _s(stream)),
           "sinn_search_noalloc")


def sinn_search_host(ix, q_indptr, q_indices, q_values, k, k_prime, out_ids, out_scores,
                     stream=None):
    """All buffers host (CPU) tensors or numpy arrays; waits for completion."""
    n_q = (q_indptr.numel() if isinstance(q_indptr, torch.Tensor) else q_indptr.size) - 1
    _check(load().sinn_search_host(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k,
                                   k_prime, _p(out_ids), _p(out_scores), _s(stream)),
           "sinn_search_host")


def sinn_sync(ix, stream=None):
    _check(load().sinn_sync(ix, _s(stream)), "sinn_sync")


def sinn_stats(ix) -> dict:
    st = SinnStats()
    _check(load().sinn_stats(ix, C.byref(st)), "sinn_stats")
    return st.as_dict()


def sinn_strerror(code: int) -> str:
    return load().sinn_strerror(code).decode()


def sinn_hash_table(ix, n: int, h: int) -> np.ndarray:
    out = np.zeros(n * h, np.uint32)
    _check(load().sinn_hash_table(ix, _p(out)), "sinn_hash_table")
    return out.reshape(n, h)


def sinn_sketch_columns(ix, ids, u_out, l_out, stream=None):
    _check(load().sinn_sketch_columns(ix, _p(ids), ids.numel(), _p(u_out), _p(l_out),
                                      _s(stream)), "sinn_sketch_columns")


def sinn_inverted_list(ix, coord: int) -> np.ndarray:
    lib = load()
    n = C.c_uint64()
    _check(lib.sinn_inverted_list(ix, coord, None, 0, C.byref(n)), "sinn_inverted_list")
    out = np.zeros(max(n.value, 1), np.uint32)
    _check(lib.sinn_inverted_list(ix, coord, _p(out), n.value, C.byref(n)), "sinn_inverted_list")
    return out[: n.value].copy()


def sinn_scores(ix, q_indptr, q_indices, q_values, out, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_scores(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, _p(out),
                              _s(stream)), "sinn_scores")


def sinn_candidates(ix, q_indptr, q_indices, q_values, k_prime, out_ids, out_scores, out_count,
                    stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_candidates(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k_prime,
                                  _p(out_ids), _p(out_scores), _p(out_count), _s(stream)),
           "sinn_candidates")


def sinn_timing_start(ix):
    _check(load().sinn_timing_start(ix), "sinn_timing_start")


def sinn_timing_stop(ix) -> dict:
    t = SinnTiming()
    _check(load().sinn_timing_stop(ix, C.byref(t)), "sinn_timing_stop")
    return t.as_dict()


def sinn_get_tuning(ix) -> dict:
    t = SinnTuning()
    _check(load().sinn_get_tuning(ix, C.byref(t)), "sinn_get_tuning")
    return t.as_dict()


def sinn_set_tuning(ix, **fields):
    t = SinnTuning()
    _check(load().sinn_get_tuning(ix, C.byref(t)), "sinn_get_tuning")
    for f, v in fields.items():
        if f not in SinnTuning.FIELDS:
            raise KeyError(f)
        setattr(t, f, int(v))
    _check(load().sinn_set_tuning(ix, C.byref(t)), "sinn_set_tuning")


def sinn_autotune(ix, q_indptr, q_indices, q_values, k, k_prime, reps=2, stream=None) -> dict:
    t = SinnTuning()
    n_q = q_indptr.numel() - 1
    _check(load().sinn_autotune(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k, k_prime,
                                reps, C.byref(t), _s(stream)), "sinn_autotune")
    return t.as_dict()


def sinn_kp_features(ix, q_indptr, q_indices, q_values, out, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_kp_features(ix, _p(q_indptr), _p(q_indices), _p(q_values), n_q, _p(out),
                                   _s(stream)), "sinn_kp_features")


def sinn_search_learned(ix, mlp, q_indptr, q_indices, q_values, k, kp_min, kp_max, out_ids,
                        out_scores, out_kprime=None, stream=None):
    n_q = q_indptr.numel() - 1
    _check(load().sinn_search_learned(ix, mlp, _p(q_indptr), _p(q_indices), _p(q_values), n_q,
                                      k, kp_min, kp_max, _p(out_ids), _p(out_scores),
                                      _p(out_kprime), _s(stream)), "sinn_search_learned")


class Context:
    """A search context (sinn_ctx): scratch for one in-flight search, so that
    searches of one index can overlap on different streams."""

    def __init__(self, index: "Index", scratch_bytes: int, mlp=None, max_queries: int = 0):
        lib = load()
        out = C.c_void_p()
        with torch.cuda.device(index.device):
            _check(lib.sinn_ctx_create(index.handle, scratch_bytes, C.byref(out)),
                   "sinn_ctx_create")
        self._h, self.index, self.mlp = out, index, mlp
        self.act = None
        if mlp is not None and max_queries:
            nbytes = int(lib.sinn_mlp_act_bytes(mlp.handle, max_queries))
            self.act = torch.empty(nbytes, dtype=torch.uint8, device=index.device)
            self.act_rows = max_queries

    def close(self):
        if getattr(self, "_h", None):
            load().sinn_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query_bytes(self, k_prime_max: int) -> int:
        return int(load().sinn_ctx_query_bytes(self._h, k_prime_max))

    def set_snapshot(self, seq: int):
        """The sequence number this context's searches see."""
        _check(load().sinn_ctx_set_snapshot(self._h, int(seq)), "sinn_ctx_set_snapshot")

    def search(self, q_indptr, q_indices, q_values, k, k_prime_max, out_ids, out_scores,
               k_prime=None, stream=None):
        n_q = q_indptr.numel() - 1
        _check(load().sinn_search_ctx(self._h, _p(q_indptr), _p(q_indices), _p(q_values), n_q, k,
                                      _p(k_prime), k_prime_max, _p(out_ids), _p(out_scores),
                                      _s(stream)), "sinn_search_ctx")

    def search_learned(self, q_indptr, q_indices, q_values, k, kp_min, kp_max, out_ids,
                       out_scores, out_kprime=None, stream=None):
        n_q = q_indptr.numel() - 1
        assert self.act is not None and n_q <= self.act_rows
        _check(load().sinn_search_learned_ctx(
            self._h, self.index.handle, self.mlp.handle, _p(self.act), self.act.numel(),
            _p(q_indptr), _p(q_indices), _p(q_values), n_q, k, kp_min, kp_max, _p(out_ids),
            _p(out_scores), _p(out_kprime), _s(stream)), "sinn_search_learned_ctx")


class Plan:
    """A recorded search (sinn_plan): one CUDA graph replayed per run over
    fixed device buffers.  The query tensors given are kept and read at
    every run, so new queries are written into them in place (same shapes).
    k_prime: None (every query takes k_prime_max) or a device uint32 tensor
    of per-query k'; with mlp the network chooses k' in [k_prime_min,
    k_prime_max]."""

    def __init__(self, index: "Index", q_indptr, q_indices, q_values, k: int, k_prime_max: int,
                 k_prime=None, mlp=None, k_prime_min: int | None = None,
                 scratch_bytes: int = 1 << 30):
        lib = load()
        dev = index.device
        self.index, self.mlp = index, mlp
        self.q_indptr, self.q_indices, self.q_values = q_indptr, q_indices, q_values
        self.k_prime = k_prime
        n_q = q_indptr.numel() - 1
        self.out_ids = torch.empty((n_q, k), dtype=torch.int32, device=dev)
        self.out_scores = torch.empty((n_q, k), dtype=torch.float32, device=dev)
        self.out_kprime = torch.empty(n_q, dtype=torch.int32, device=dev) if mlp else None
        out = C.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.sinn_plan_create(index.handle, mlp.handle if mlp else None, _p(q_indptr),
                                        _p(q_indices), _p(q_values), _p(k_prime), n_q, k,
                                        k_prime_min if k_prime_min is not None else k,
                                        k_prime_max, _p(self.out_ids), _p(self.out_scores),
                                        _p(self.out_kprime), scratch_bytes, C.byref(out)),
                   "sinn_plan_create")
        self._h = out

    def run(self, stream=None):
        _check(load().sinn_plan_run(self._h, _s(stream)), "sinn_plan_run")
        return self.out_ids, self.out_scores

    @property
    def recordings(self) -> int:
        return int(load().sinn_plan_recordings(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().sinn_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The k' network (sinn_mlp): n_in -> hidden -> hidden -> 1."""

    def __init__(self, n_in: int = KP_FEATURES, hidden: int = 256, seed: int = 0x5151,
                 device=None):
        lib = load()
        self.device = torch.device(device or "cuda")
        out = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.sinn_mlp_create(n_in, hidden, seed, C.byref(out)), "sinn_mlp_create")
        self._h, self.n_in, self.hidden = out, n_in, hidden

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().sinn_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(load().sinn_mlp_num_params(self._h))

    def params(self, which: int = 0) -> np.ndarray:
        out = np.zeros(self.num_params, np.float32)
        _check(load().sinn_mlp_params(self._h, _p(out), which), "sinn_mlp_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        _check(load().sinn_mlp_set_params(self._h, _p(p)), "sinn_mlp_set_params")

    def set_normalizer(self, mean, std):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        _check(load().sinn_mlp_set_normalizer(self._h, _p(m), _p(s)), "sinn_mlp_set_normalizer")

    def forward(self, X, stream=None) -> torch.Tensor:
        X = _dev(X, torch.float32, self.device)
        y = torch.empty(X.shape[0], dtype=torch.float32, device=self.device)
        _check(load().sinn_mlp_forward(self._h, _p(X), X.shape[0], _p(y), _s(stream)),
               "sinn_mlp_forward")
        return y

    def grad(self, X, t, tau: float, stream=None):
        X = _dev(X, torch.float32, self.device)
        t = _dev(t, torch.float32, self.device)
        g = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _check(load().sinn_mlp_grad(self._h, _p(X), _p(t), X.shape[0], tau, _p(g), _p(loss),
                                    _s(stream)), "sinn_mlp_grad")
        return g, loss

    def train_step(self, X, t, tau: float, lr: float, stream=None) -> torch.Tensor:
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _check(load().sinn_mlp_train_step(self._h, _p(X), _p(t), X.shape[0], tau, lr, _p(loss),
                                          _s(stream)), "sinn_mlp_train_step")
        return loss

    def sync(self, stream=None):
        """Waits for the stream; raises if a GEMM's bounded wait ran out."""
        _check(load().sinn_mlp_sync(self._h, _s(stream)), "sinn_mlp_sync")

    def set_policy(self, shifts=None, posting_cost: float = 0.0, margin: float = 0.0):
        """Budget levels P_q / 2^shift (shifts[0] = 0) chosen per query by
        least posting_cost * postings + k'; None clears the policy."""
        sinn_mlp_set_policy(self._h, shifts, posting_cost, margin)

    def policy(self) -> dict:
        return sinn_mlp_get_policy(self._h)


def sinn_debug_fail_alloc(after: int):
    """The library's allocation after `after` more successful ones fails
    (SINN_ENOMEM from the call making it); after < 0 turns this off."""
    _check(load().sinn_debug_fail_alloc(int(after)), "sinn_debug_fail_alloc")


def sinn_debug_wait_probe(spins: int, arrive: bool, stream=None) -> int:
    """Status of one bounded mbarrier wait of at most `spins` polls that
    nothing completes (arrive False) or that completes (arrive True)."""
    return int(load().sinn_debug_wait_probe(int(spins), 1 if arrive else 0, _s(stream)))


# ------------------------------------------------------------- convenience

class Index:
    """A SINNAMON index on one CUDA device (owns a sinn_index handle)."""

    def __init__(self, n: int, m: int, h: int, device=None, **cfg):
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self._h = sinn_create_ex(n, m, h, **cfg)
        self.n, self.m, self.h = n, m, h
        self.flags = int(cfg.get("flags", 0))
        self.nonneg = bool(self.flags & SINN_FLAG_NONNEG)

    def close(self):
        if getattr(self, "_h", None):
            sinn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def _csr(self, indptr, indices, values):
        return (_dev(indptr, torch.int64, self.device), _dev(indices, torch.int32, self.device),
                _dev(values, torch.float32, self.device))

    def insert(self, indptr, indices, values, stream=None) -> torch.Tensor:
        ip, ix, v = self._csr(indptr, indices, values)
        out = torch.empty(ip.numel() - 1, dtype=torch.int32, device=self.device)
        sinn_insert(self._h, ip, ix, v, out, stream)
        return out

    def delete(self, ids, stream=None):
        sinn_delete(self._h, _dev(ids, torch.int32, self.device), stream)

    def insert_at(self, indptr, indices, values, seq: int, stream=None) -> torch.Tensor:
        """sinn_insert_at: the vectors are born at sequence number seq."""
        ip, ix, v = self._csr(indptr, indices, values)
        out = torch.empty(ip.numel() - 1, dtype=torch.int32, device=self.device)
        sinn_insert_at(self._h, ip, ix, v, out, seq, stream)
        return out

    def delete_at(self, ids, seq: int, stream=None):
        sinn_delete_at(self._h, _dev(ids, torch.int32, self.device), seq, stream)

    def reclaim(self, horizon: int, stream=None):
        sinn_reclaim(self._h, horizon, stream)

    def reserve(self, more_ids: int, more_entries: int):
        """sinn_reserve: room for more_ids fresh ids and more_entries store
        entries beyond those in use."""
        sinn_reserve(self._h, more_ids, more_entries)

    def search(self, indptr, indices, values, k: int, k_prime, k_prime_max: int | None = None,
               stream=None):
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        ids = torch.empty((nq, k), dtype=torch.int32, device=self.device)
        sc = torch.empty((nq, k), dtype=torch.float32, device=self.device)
        if isinstance(k_prime, int):
            sinn_search(self._h, ip, ix, v, k, k_prime, ids, sc, stream)
        else:
            kp = _dev(k_prime, torch.int32, self.device)
            sinn_search_kp(self._h, ip, ix, v, k, kp, int(k_prime_max), ids, sc, stream)
        return ids, sc

    def scores(self, indptr, indices, values, stream=None) -> torch.Tensor:
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        out = torch.empty((nq, self.stats()["capacity"]), dtype=torch.float32, device=self.device)
        sinn_scores(self._h, ip, ix, v, out, stream)
        return out

    def candidates(self, indptr, indices, values, k_prime: int, stream=None):
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        ids = torch.empty((nq, k_prime), dtype=torch.int32, device=self.device)
        sc = torch.empty((nq, k_prime), dtype=torch.float32, device=self.device)
        cnt = torch.empty(nq, dtype=torch.int32, device=self.device)
        sinn_candidates(self._h, ip, ix, v, k_prime, ids, sc, cnt, stream)
        return ids, sc, cnt

    def sketch_columns(self, ids, stream=None):
        """Columns of U and L (L is None for a SINNAMON+ index)."""
        ids = _dev(ids, torch.int32, self.device)
        u = torch.empty((ids.numel(), self.m), dtype=torch.float32, device=self.device)
        l = None if self.nonneg else torch.empty_like(u)
        sinn_sketch_columns(self._h, ids, u, l, stream)
        return u, l

    def set_budget(self, postings: int):
        """Alg. 6's anytime budget in postings (0 = none)."""
        _check(load().sinn_set_budget(self._h, int(postings)), "sinn_set_budget")

    @property
    def budget(self) -> int:
        return int(load().sinn_get_budget(self._h))

    def inverted_list(self, coord: int) -> np.ndarray:
        return sinn_inverted_list(self._h, coord)

    def hash_table(self) -> np.ndarray:
        return sinn_hash_table(self._h, self.n, self.h)

    def search_kpb(self, indptr, indices, values, k: int, k_prime=None, k_prime_max: int = 0,
                   budget=None, stream=None):
        """Search with per-query k' (None: k_prime_max for all) and per-query
        Alg. 6 budgets in postings (None: the index's budget)."""
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        ids = torch.empty((nq, k), dtype=torch.int32, device=self.device)
        sc = torch.empty((nq, k), dtype=torch.float32, device=self.device)
        kp = None if k_prime is None else _dev(k_prime, torch.int32, self.device)
        bd = None if budget is None else _dev(budget, torch.int64, self.device)
        sinn_search_kpb(self._h, ip, ix, v, k, kp, int(k_prime_max), bd, ids, sc, stream)
        return ids, sc

    def candidates_kpb(self, indptr, indices, values, k_prime: int, budget=None, stream=None):
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        ids = torch.empty((nq, k_prime), dtype=torch.int32, device=self.device)
        sc = torch.empty((nq, k_prime), dtype=torch.float32, device=self.device)
        cnt = torch.empty(nq, dtype=torch.int32, device=self.device)
        bd = None if budget is None else _dev(budget, torch.int64, self.device)
        sinn_candidates_kpb(self._h, ip, ix, v, k_prime, bd, ids, sc, cnt, stream)
        return ids, sc, cnt

    def query_postings(self, indptr, indices, values, stream=None) -> torch.Tensor:
        ip, ix, v = self._csr(indptr, indices, values)
        out = torch.empty(ip.numel() - 1, dtype=torch.int64, device=self.device)
        sinn_query_postings(self._h, ip, ix, v, out, stream)
        return out

    def kp_choose(self, mlp, indptr, indices, values, kp_min: int, kp_max: int, stream=None):
        """The learned search's (k', budget) per query."""
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        kp = torch.empty(nq, dtype=torch.int32, device=self.device)
        bd = torch.empty(nq, dtype=torch.int64, device=self.device)
        sinn_kp_choose(self._h, mlp.handle, ip, ix, v, kp_min, kp_max, kp, bd, stream)
        return kp, bd

    def kp_features(self, indptr, indices, values, stream=None) -> torch.Tensor:
        ip, ix, v = self._csr(indptr, indices, values)
        out = torch.empty((ip.numel() - 1, KP_FEATURES), dtype=torch.float32, device=self.device)
        sinn_kp_features(self._h, ip, ix, v, out, stream)
        return out

    def search_learned(self, mlp, indptr, indices, values, k: int, kp_min: int, kp_max: int,
                       stream=None):
        ip, ix, v = self._csr(indptr, indices, values)
        nq = ip.numel() - 1
        ids = torch.empty((nq, k), dtype=torch.int32, device=self.device)
        sc = torch.empty((nq, k), dtype=torch.float32, device=self.device)
        kp = torch.empty(nq, dtype=torch.int32, device=self.device)
        sinn_search_learned(self._h, mlp.handle, ip, ix, v, k, kp_min, kp_max, ids, sc, kp,
                            stream)
        return ids, sc, kp

    def tuning(self) -> dict:
        return sinn_get_tuning(self._h)

    def set_tuning(self, **fields):
        sinn_set_tuning(self._h, **fields)

    def autotune(self, indptr, indices, values, k: int, k_prime: int, reps: int = 2,
                 stream=None) -> dict:
        ip, ix, v = self._csr(indptr, indices, values)
        return sinn_autotune(self._h, ip, ix, v, k, k_prime, reps, stream)

    def sync(self, stream=None):
        sinn_sync(self._h, stream)

    def save(self, path: str):
        """Checkpoint the whole index to `path` (sinn_save)."""
        _check(load().sinn_save(self._h, os.fsencode(path)), "sinn_save")

    @classmethod
    def load(cls, path: str, device=None) -> "Index":
        """An index resumed from a sinn_save file on `device` (sinn_load)."""
        obj = cls.__new__(cls)
        obj.device = torch.device(device or "cuda")
        out = C.c_void_p()
        with torch.cuda.device(obj.device):
            _check(load().sinn_load(os.fsencode(path), C.byref(out)), "sinn_load")
        obj._h = out
        st = obj.stats()
        obj.n, obj.m, obj.h = st["n"], st["m"], st["h"]
        obj.flags = st["flags"]
        obj.nonneg = bool(obj.flags & SINN_FLAG_NONNEG)
        return obj

    def stats(self) -> dict:
        return sinn_stats(self._h)
