/*
 * sinnamon.h -- C ABI of the GB300 (sm_103a) SINNAMON library.
 *
 * SINNAMON (Bruch, Nardini, Ingber, Liberty, "An Approximate Algorithm for
 * Maximum Inner Product Search over Streaming Sparse Vectors") answers Eq. 2,
 * argmax^(k)_{x in X} <q, x>, approximately over a collection X of sparse
 * real vectors that changes online (Sec. 1: insertions and deletions arrive
 * while queries run).  The index keeps, on one GPU:
 *   - an inverted index I: coordinate -> ids of the vectors non-zero there
 *     (Alg. 5), stored per tile of T consecutive ids as a container
 *     of 16-bit local ids: a sorted array, or a T-bit bitmap when at least
 *     an eighth of the tile holds the coordinate; a deleted posting is
 *     tombstoned in place (Sec. 4.3);
 *   - the sketch matrix [U; L] (Alg. 5): 2m rows of fp32 over all id slots,
 *     row-major, so one query coordinate reads a fixed set of h rows;
 *   - the vector store S that Alg. 7 re-ranks from (Fig. 1): each vector's
 *     (coordinate, value) pairs.
 *
 * Conventions for every call:
 *   - Return value: SINN_OK (0) or one of the SINN_E* codes below.
 *     sinn_strerror() names a code.
 *   - "device" pointers are CUDA device memory of the device the index was
 *     created on (for example PyTorch CUDA tensors); "host" pointers are CPU
 *     memory.  The caller owns every buffer it passes; the library owns the
 *     index and its scratch, and never frees a caller's buffer.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; sinn_insert and sinn_delete also wait for it,
 *     because they update host-side bookkeeping (ids, sizes).
 *   - A handle is not thread-safe: calls on one handle must be serialised.
 *   - Sparse inputs are CSR: indptr[rows+1] (uint64), indices (uint32, each
 *     < n, strictly increasing within a row), values (float32, finite).
 *     Entries equal to zero are not non-zeros (Alg. 5, Alg. 6):
 *     they are neither indexed nor sketched nor scored.
 *   - Ties: every ranking puts the larger score first and, among equal
 *     scores, the smaller id first.
 */
#ifndef SINNAMON_H
#define SINNAMON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SINN_OK 0
#define SINN_EINVAL 1    /* bad argument or malformed input; nothing changed */
#define SINN_ENOTFOUND 2 /* delete of an id that is not live; nothing changed */
#define SINN_ENOMEM 3    /* device or host allocation failed */
#define SINN_ECUDA 4     /* a CUDA runtime call failed */
#define SINN_EDEVICE 5   /* a kernel reported an error (see sinn_sync) */
#define SINN_ESCRATCH 6  /* sinn_search_noalloc: one query needs more than its fixed scratch */
#define SINN_EIO 7       /* sinn_save / sinn_load: file error, or not a saved index */
#define SINN_EBUSY 8     /* sinn_insert_at: a search older than a tile's last rebuild may
                            still read it (sinn_reclaim first); sinn_save: deletions
                            not yet reclaimed */

/* Sequence numbers of snapshot searches and sequence-numbered mutations run
 * from 0 to SINN_SEQ_LATEST; a search at SINN_SEQ_LATEST (the default) sees
 * every mutation made so far. */
#define SINN_SEQ_LATEST 0xFFFFFFFEu

typedef struct sinn_index sinn_index; /* opaque; owned by the library */

/* SINNAMON+ (the Sec. 4.1 note on the non-negative orthant): only the upper
 * sketch U is kept.  Inserts with a negative value are rejected (EINVAL) and
 * queries with a negative value are malformed (their row is padded and the
 * device error set); on non-negative data the results equal SINNAMON's,
 * which never reads L for positive query entries. */
#define SINN_FLAG_NONNEG 1u

/* bfloat16 sketch (the paper stores sketches as bfloat16, Sec. 4.1 notes):
 * U and L take 2 bytes per bin instead of 4.  An upper bin holds the least
 * bfloat16 at or above its value and a lower bin the greatest at or below,
 * so decoded values remain upper / lower bounds (Thm. 1 holds); scores are
 * sums of those rounded values, so candidates can differ from the fp32
 * sketch's.  sinn_sketch_columns returns the rounded values as floats. */
#define SINN_FLAG_BF16_SKETCH 2u

/* Index parameters.  Zero fields take the defaults noted. */
typedef struct sinn_config {
  uint32_t n;              /* dimensionality; coordinates are [0, n) */
  uint32_t m;              /* sketch bins per side (U and L have m rows each), m <= 4096 */
  uint32_t h;              /* number of random mappings pi_o: [n] -> [m], 1 <= h <= min(m, 8) */
  uint32_t tile_docs;      /* ids per tile T: power of two in [1024, 16384]; 0 -> 4096 */
  uint64_t seed;           /* seed of the mappings; 0 -> 0x5151 */
  uint64_t capacity_hint;  /* id slots to reserve up front; 0 -> one tile */
  const uint32_t *table;   /* optional host table[n*h] with table[j*h+o] = pi_o(j) < m;
                              NULL -> pi_o(j) = mix64(seed ^ (o+1)*0x9E3779B97F4A7C15 ^ j) mod m,
                              mix64 being SplitMix64's output function */
  uint32_t max_query_nnz;  /* largest query non-zero count sinn_search accepts; 0 -> 1024 */
  uint32_t flags;          /* 0 or SINN_FLAG_NONNEG | SINN_FLAG_BF16_SKETCH */
  uint64_t scratch_bytes;  /* device scratch budget of one search launch; 0 -> 4 GiB */
} sinn_config;

/* Counters reported by sinn_stats. */
typedef struct sinn_stats {
  uint64_t live;           /* live vectors |X| */
  uint64_t capacity;       /* id slots with storage (a multiple of tile_docs) */
  uint64_t next_id;        /* ids ever handed out: live + free */
  uint64_t postings;       /* postings held in the inverted index, tombstones included */
  uint64_t tombstones;     /* deleted postings not yet compacted away */
  uint64_t bytes_lists;    /* device bytes of the inverted index (postings + tile offsets) */
  uint64_t bytes_sketch;   /* device bytes of U and L */
  uint64_t bytes_store;    /* device bytes of the vector store */
  uint64_t bytes_scratch;  /* device bytes of search scratch currently held */
  uint32_t n, m, h, tile_docs;
  uint32_t flags;          /* the index's SINN_FLAG_* bits */
  uint32_t pending_deletes; /* ids deleted at a sequence number, not yet reclaimed
                               (not counted in live) */
} sinn_stats_t;

/* Create an empty index on the current CUDA device with default settings.
 * n, m, h as in Alg. 5 (Sec. 4.1).  EINVAL if n = 0, m = 0, h = 0, h > m or
 * h > 8.  *out receives the handle. */
int sinn_create(uint32_t n, uint32_t m, uint32_t h, sinn_index **out);

/* Create with explicit parameters (see sinn_config). */
int sinn_create_ex(const sinn_config *cfg, sinn_index **out);

/* Release the index and all device memory it owns.  NULL is accepted. */
int sinn_destroy(sinn_index *ix);

/* Insert n_docs vectors (Alg. 5: inverted-list append and sketch columns; the
 * vectors also enter the store S).  indptr/indices/values: device CSR.
 * out_ids: device uint32[n_docs] receiving each vector's id: free ids in
 * ascending order first (Sec. 4.3 reuse), then fresh ids, in row order.
 * The whole batch is validated before anything changes (EINVAL), and every
 * allocation the insert needs is made before anything changes: on ENOMEM the
 * index holds the same vectors as before (its capacity may have grown).
 * Waits for the stream before returning. */
int sinn_insert(sinn_index *ix, const uint64_t *indptr, const uint32_t *indices,
                const float *values, uint32_t n_docs, uint32_t *out_ids, void *stream);

/* Delete n_ids vectors by id (Sec. 4.3): each id is removed from every
 * inverted list it is in (tombstoned in place), its sketch column is left as
 * it is, and the id becomes free for reuse.  ids: device uint32[n_ids].
 * ENOTFOUND if an id is not live, EINVAL if an id repeats; then nothing
 * changes.  Waits for the stream before returning. */
int sinn_delete(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, void *stream);

/* ---- Mutations while searches run (snapshots) ----------------------------
 * The paper's setting has insertions and deletions arrive while queries run
 * (Sec. 1, Sec. 4.3).  These calls let them overlap on the GPU: every
 * request gets a sequence number, and a search at sequence number s (its
 * context's snapshot, sinn_ctx_set_snapshot) counts exactly the vectors
 * inserted at numbers <= s and not deleted at numbers <= s -- the same
 * results as if it ran alone after the mutations numbered below it.
 *   - A search must be launched after the mutations numbered below its own
 *     number are enqueued, on a stream ordered after them (for example by
 *     an event); it may then run while later mutations run on other
 *     streams.
 *   - Each tile of ids has two copies of its containers; a search reads the
 *     current one, and a rebuild writes the other and then makes it current.
 *   - Deleted ids keep their postings (so older searches still score them)
 *     until sinn_reclaim removes them; only then can an insert reuse them.
 * sinn_insert and sinn_delete are the stream-ordered forms (no search may be
 * in flight); the forms below may be mixed with them. */

/* Insert as sinn_insert, the vectors born at sequence number seq (searches
 * at numbers below seq do not count them).  A tile it lands in is rebuilt
 * into the copy searches do not read; a search numbered below that tile's
 * previous sequence-numbered rebuild may still read that copy, so unless
 * every such search has been reclaimed (sinn_reclaim with a horizon at least
 * that rebuild's number) the call returns SINN_EBUSY and changes nothing.
 * seq <= SINN_SEQ_LATEST. */
int sinn_insert_at(sinn_index *ix, const uint64_t *indptr, const uint32_t *indices,
                   const float *values, uint32_t n_docs, uint32_t *out_ids, uint32_t seq,
                   void *stream);

/* Delete at sequence number seq: searches at numbers >= seq stop counting
 * the ids, older ones still do; the postings are removed and the ids freed
 * by a later sinn_reclaim.  ids: device uint32[n_ids] of live ids (ENOTFOUND
 * otherwise, EINVAL for a repeat; nothing changes then).  Waits for the
 * stream. */
int sinn_delete_at(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, uint32_t seq,
                   void *stream);

/* The caller states that every search numbered below `horizon` has finished
 * (horizon <= SINN_SEQ_LATEST + 1).  Deletions numbered at or below it are
 * then carried out (postings tombstoned, ids freed for reuse) and inserted
 * vectors numbered at or below it stop needing a snapshot check.  Horizons
 * never move back.  Waits for the stream. */
int sinn_reclaim(sinn_index *ix, uint32_t horizon, void *stream);

/* Approximate top-k search for n_q queries: Alg. 6 scoring (T = infinity),
 * then Alg. 7: the k' best approximate scores among live ids, re-ranked by
 * exact inner product <q, S.Fetch(v)>, best k returned.
 * q_indptr/q_indices/q_values: device CSR (each row <= max_query_nnz
 * non-zeros).  out_ids: device uint32[n_q*k], out_scores: device
 * float[n_q*k], row-major, best first; rows with fewer than k live vectors
 * are padded with id 0xFFFFFFFF and score -inf.  1 <= k <= 1024, k <= k'.
 * Asynchronous: a malformed query sets the device error that sinn_sync
 * returns, and that query's row is padded. */
int sinn_search(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                uint32_t *out_ids, float *out_scores, void *stream);

/* As sinn_search with a per-query k': k_prime[q] (device uint32[n_q]) is
 * clamped to [k, k_prime_max]. */
int sinn_search_kp(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                   const float *q_values, uint32_t n_q, uint32_t k, const uint32_t *k_prime,
                   uint32_t k_prime_max, uint32_t *out_ids, float *out_scores, void *stream);

/* As sinn_search_kp with, besides the per-query k' (k_prime: device
 * uint32[n_q] clamped to [k, k_prime_max], or NULL for k_prime_max
 * everywhere), a per-query anytime budget of Alg. 6: budget is device
 * uint64[n_q], budget[q] the postings query q may visit (0 = T = infinity;
 * the break follows sinn_set_budget's rule), or NULL for the index's budget.
 * The re-rank of Alg. 7 always takes every query term. */
int sinn_search_kpb(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                    const float *q_values, uint32_t n_q, uint32_t k, const uint32_t *k_prime,
                    uint32_t k_prime_max, const uint64_t *budget, uint32_t *out_ids,
                    float *out_scores, void *stream);

/* Alg. 6's postings of each query with no budget: out[q] = the sum over the
 * query's non-zeros j of |I[j]| (live postings), device uint64[n_q]; 0 for a
 * malformed row. */
int sinn_query_postings(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                        const float *q_values, uint32_t n_q, uint64_t *out, void *stream);

/* As sinn_search with every buffer in host memory: the call copies the
 * queries to the device, searches, copies the results back and waits.
 * Device errors are returned directly. */
int sinn_search_host(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                     const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                     uint32_t *out_ids, float *out_scores, void *stream);

/* sinn_search without any allocation, for callers that cannot allocate
 * device memory while they search (a memory budget fixed in advance, or a
 * serving path that must not enter the allocator, which can synchronise the
 * device or fail when memory is fragmented).  The paper has no counterpart:
 * this is a deployment variant of the same search.
 * Arguments and results are exactly those of sinn_search.  The scratch is a
 * fixed 64 MiB device array inside the library, present on every device that
 * loads it until the library is unloaded.  Queries are processed in groups
 * that fit it; SINN_ESCRATCH if even one query does not fit (one query needs
 * about 4 bytes per id slot of the index plus 1.6 MB).  Each call looks the
 * array's device address up in the current context (no allocation), except
 * on a stream being captured, where it uses the address an earlier call on
 * that device found: make the first call on a device before any stream
 * capture (SINN_ECUDA otherwise).  Every call on a device shares the array and overwrites
 * what the last call left there: calls that overlap on the GPU (on different
 * streams, or for different indexes of the same device) race, so order them.
 * The call itself allocates nothing and records no timing events. */
int sinn_search_noalloc(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                        const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                        uint32_t *out_ids, float *out_scores, void *stream);

/* ---- Search contexts: concurrent searches of one index ------------------
 * A context owns the device scratch of one search, so searches in different
 * contexts may run at the same time on different streams (a search only
 * reads the index).  Inserts and deletes of the index must be ordered
 * against every search in flight (they change the index in place).
 * scratch_bytes >= 1 MiB; sinn_ctx_query_bytes gives the scratch one query
 * needs at a given k'; a search processes as many queries at a time as fit
 * (SINN_ESCRATCH if one does not). */
typedef struct sinn_ctx sinn_ctx;
int sinn_ctx_create(sinn_index *ix, uint64_t scratch_bytes, sinn_ctx **out);

/* The sequence number the context's searches see (SINN_SEQ_LATEST after
 * creation): see "Mutations while searches run" above. */
int sinn_ctx_set_snapshot(sinn_ctx *c, uint32_t seq);
int sinn_ctx_destroy(sinn_ctx *c);
uint64_t sinn_ctx_query_bytes(sinn_ctx *c, uint32_t k_prime_max);

/* sinn_search (k_prime == NULL: k' = k_prime_max for every query) or
 * sinn_search_kp (device k_prime[n_q]) on the context's scratch. */
int sinn_search_ctx(sinn_ctx *c, const uint64_t *q_indptr, const uint32_t *q_indices,
                    const float *q_values, uint32_t n_q, uint32_t k, const uint32_t *k_prime,
                    uint32_t k_prime_max, uint32_t *out_ids, float *out_scores, void *stream);

/* Wait for the stream, then return and clear the sticky device error
 * (SINN_OK if none; SINN_EINVAL for a malformed query; SINN_EDEVICE for an
 * internal kernel error or a bounded wait inside a kernel that ran out). */
int sinn_sync(sinn_index *ix, void *stream);

/* Fill *out with the counters above (host). */
int sinn_stats(sinn_index *ix, sinn_stats_t *out);

/* Make room ahead of inserts: id slots for more_ids fresh ids beyond those
 * handed out so far (next_id) and vector-store room for more_entries
 * (coordinate, value) entries beyond those it holds, so that inserts up to
 * those sizes allocate no id-capacity arrays and no store (growing either
 * waits for every stream of the device, which a serving loop would feel as
 * a pause).  Room already there is kept; nothing else changes.  SINN_ENOMEM
 * (and no change to the part that failed) if an allocation fails; the id
 * capacity is limited as for inserts. */
int sinn_reserve(sinn_index *ix, uint64_t more_ids, uint64_t more_entries);

/* Alg. 6's anytime budget T, counted in postings (the scoring time is
 * proportional to them): each query's terms run in Alg. 6 order and scoring
 * stops after the first term at which the live postings of the lists scored
 * so far reach the budget.  0 (the default) is T = infinity.  Applies to
 * every later search, candidate and score call of the index. */
int sinn_set_budget(sinn_index *ix, uint64_t postings);

/* The current budget (0 = none); 0 for a NULL index. */
uint64_t sinn_get_budget(sinn_index *ix);

/* Checkpoint: write the whole index (parameters, mapping table, sketch,
 * lists, vector store, free ids, counters, tuning and budget) to the file at
 * `path`, replacing it.  Waits for the device.  SINN_EIO if the file cannot
 * be written.  The format is the library's own (little-endian, versioned). */
int sinn_save(sinn_index *ix, const char *path);

/* Resume: a new index on the current CUDA device holding exactly what
 * sinn_save wrote: the same live vectors under the same ids, free ids,
 * sketch, lists and store, so searches, inserts (ids included) and deletes
 * behave as they would have on the saved index.  SINN_EIO for a missing,
 * truncated or foreign file; *out is NULL on any error. */
int sinn_load(const char *path, sinn_index **out);

/* ---- Test hooks: failures made on the host, none of them faults a GPU. */

/* Allocation fault injection (process-wide): after `after` more successful
 * device or pinned-host allocations by the library, the next one fails as
 * if memory were exhausted (the call making it returns SINN_ENOMEM); then
 * injection is off again.  after < 0 turns it off.  Always SINN_OK. */
int sinn_debug_fail_alloc(int64_t after);

/* One block waits on an mbarrier with the bounded wait the tensor-core
 * kernels use, for at most `spins` polls: nothing completes the barrier
 * (arrive = 0) or the block completes it first (arrive = 1).  Waits for the
 * stream; SINN_EDEVICE if the wait ran out, SINN_OK if it completed. */
int sinn_debug_wait_probe(uint32_t spins, int arrive, void *stream);

/* ---- Launch tuning (the paper has no counterpart: these are GPU launch
 * parameters; results do not depend on them beyond fp32 summation order) -- */

/* Run-time launch parameters of the search.  Defaults come with the index;
 * sinn_autotune chooses them by timing. */
typedef struct sinn_tuning {
  uint32_t bound_every;      /* scored tiles between refreshes of a query's running
                                k'-th bound, 1..64 (default 4) */
  uint32_t emit_min_batch;   /* launches of fewer queries score densely instead of
                                emitting candidates, 1..65535 (default 32) */
  uint32_t max_batch;        /* cap on queries per internal launch, 0 = as many as the
                                scratch holds (default 0) */
  uint32_t rerank_blocks;    /* re-rank blocks per query, 1..1024, or 0 (default) for
                                one per 64 candidates of the largest k' */
  uint32_t dense_blocks_per_sm; /* grid of the dense scoring kernel (launches of few
                                   queries) per SM, 1..32 (default 8) */
  uint32_t tiles_per_block;  /* tiles one block of the batched scoring kernel covers,
                                1..64 (default 4) */
  uint32_t persistent_blocks_per_sm; /* 0 (default): one block per (query, tile group);
                                        1..4: that many resident blocks per SM take
                                        (query, tile group) items from a counter */
  uint32_t array_walk;       /* how a tile's array-container postings are shared out:
                                0 (default): each warp takes whole 32-posting chunks of
                                one term; 1: the block's threads take consecutive
                                postings across all terms (for thin lists) */
} sinn_tuning;

/* Current tuning of the index into *out (host). */
int sinn_get_tuning(sinn_index *ix, sinn_tuning *out);

/* Set the tuning; SINN_EINVAL (and no change) if a field is out of range. */
int sinn_set_tuning(sinn_index *ix, const sinn_tuning *t);

/* Choose the tuning by timing sinn_search on a sample of queries (device
 * CSR as in sinn_search, at least 1 query) with k and k_prime: coordinate
 * descent over the fields above, each candidate timed with CUDA events on
 * `stream` (best of `reps` runs, 1..8).  Leaves the fastest tuning set and
 * copies it to *out (host, may be NULL).  Synchronises the stream. */
int sinn_autotune(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                  const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                  uint32_t reps, sinn_tuning *out, void *stream);

/* Per-phase device timing, for benchmarks.  Phases: 0 query preparation,
 * 1 scoring (Alg. 6), 2 top-k' selection (Alg. 7), 3 re-rank and
 * top-k (Alg. 7), 4 insert (Alg. 5), 5 delete (Sec. 4.3).  Each phase is
 * also an NVTX range on the calling thread ("sinn score", ...), timing on
 * or off, for profilers' timelines. */
#define SINN_PHASES 6
typedef struct sinn_timing {
  double ms[SINN_PHASES];        /* summed CUDA-event durations per phase */
  uint64_t spans[SINN_PHASES];   /* timed spans per phase */
  uint64_t launches;             /* kernels the library launched meanwhile */
} sinn_timing_t;

/* Start recording: every later phase is bracketed by CUDA events on the
 * stream it runs on.  Resets the counters. */
int sinn_timing_start(sinn_index *ix);

/* Stop recording, wait for the recorded events and fill *out (host). */
int sinn_timing_stop(sinn_index *ix, sinn_timing_t *out);

/* Name of a status code (static string). */
const char *sinn_strerror(int code);

/* ---- Inspection (used by tests; not on the hot path) ------------------- */

/* Copy the mappings to host table[n*h]: table[j*h+o] = pi_o(j). */
int sinn_hash_table(sinn_index *ix, uint32_t *table);

/* Sketch columns of the given ids (Alg. 5's u and l): ids device
 * uint32[n_ids]; u_out, l_out device float[n_ids*m], row r = column ids[r].
 * A deleted id yields its stale column (Sec. 4.3 leaves it in place).
 * l_out may be NULL; it must be NULL for a SINNAMON+ index (EINVAL). */
int sinn_sketch_columns(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, float *u_out,
                        float *l_out, void *stream);

/* Live ids of inverted list I[coord] in ascending order, into host
 * out[cap]; *len receives the list length (copy truncated at cap). */
int sinn_inverted_list(sinn_index *ix, uint32_t coord, uint32_t *out, uint64_t cap,
                       uint64_t *len);

/* Alg. 6 scores of n_q queries over every id slot: device out[n_q*capacity]
 * (capacity from sinn_stats), -inf for slots that are not live. */
int sinn_scores(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                const float *q_values, uint32_t n_q, float *out, void *stream);

/* Alg. 7's candidate step only: the min(k', live) candidates of each query with their
 * approximate scores, in no particular order.  out_ids device uint32[n_q*k'],
 * out_scores device float[n_q*k'], out_count device uint32[n_q]. */
int sinn_candidates(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                    const float *q_values, uint32_t n_q, uint32_t k_prime, uint32_t *out_ids,
                    float *out_scores, uint32_t *out_count, void *stream);

/* sinn_candidates with a per-query anytime budget (device uint64[n_q] as in
 * sinn_search_kpb, or NULL for the index's budget). */
int sinn_candidates_kpb(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                        const float *q_values, uint32_t n_q, uint32_t k_prime,
                        const uint64_t *budget, uint32_t *out_ids, float *out_scores,
                        uint32_t *out_count, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SINNAMON_H */
