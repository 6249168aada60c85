/*
 * sinnamon_plan.h -- recorded searches (CUDA graphs) for the GB300 SINNAMON
 * library.  The paper has no counterpart: this is a launch mechanism.  A
 * plan records one whole batched search -- Alg. 6 scoring, Alg. 7 selection
 * and re-ranking, and for the learned variant the k' network before them --
 * into a CUDA graph once and replays it with one launch per call.
 */
#ifndef SINNAMON_PLAN_H
#define SINNAMON_PLAN_H

#include "sinnamon_kprime.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sinn_plan sinn_plan; /* opaque; owned by the library */

/* Record-once search of exactly n_q queries over caller-owned device
 * buffers, which must keep their addresses while the plan lives; the caller
 * fills the inputs before each sinn_plan_run.
 *   q_indptr/q_indices/q_values: device CSR of the n_q queries (uint64
 *     indptr[n_q+1]; the row lengths may change between runs, the total
 *     must fit the caller's index and value buffers).
 *   Mode, by the pointers given:
 *     mlp == NULL, k_prime == NULL: every query takes k' = k_prime_max
 *       (sinn_search);
 *     mlp == NULL, k_prime != NULL: device uint32[n_q] per-query k',
 *       clamped to [k, k_prime_max] (sinn_search_kp);
 *     mlp != NULL: k' from the network, clamped to [k_prime_min,
 *       k_prime_max] (sinn_search_learned); out_kprime (device uint32[n_q],
 *       may be NULL) receives it.
 *   out_ids/out_scores: device uint32[n_q*k] / float[n_q*k] as in sinn_search.
 *   scratch_bytes: the plan's own search scratch (>= 1 MiB; the batch is cut
 *     into internal launches that fit).
 * The recording is made at the first run and made again, automatically,
 * after a change that would make it stale: the index's id capacity or
 * vector store grew, the highest id entered a new tile, or the tuning
 * changed.  Inserts and deletes that reuse freed ids keep it valid while the
 * vector store (append-only, doubled when full) has room.
 * EINVAL on a bad argument, ENOMEM if the scratch cannot be allocated. */
int sinn_plan_create(sinn_index *ix, sinn_mlp *mlp, const uint64_t *q_indptr,
                     const uint32_t *q_indices, const float *q_values, const uint32_t *k_prime,
                     uint32_t n_q, uint32_t k, uint32_t k_prime_min, uint32_t k_prime_max,
                     uint32_t *out_ids, float *out_scores, uint32_t *out_kprime,
                     uint64_t scratch_bytes, sinn_plan **out);

/* Run the plan on `stream` (recording it first when needed).  With timing
 * on (sinn_timing_start) the phases inside the graph are timed too; the
 * call then waits for the graph to finish. */
int sinn_plan_run(sinn_plan *p, void *stream);

/* How many times the plan has been recorded (host). */
uint64_t sinn_plan_recordings(sinn_plan *p);

/* Release the plan (waits for the device).  NULL is accepted. */
int sinn_plan_destroy(sinn_plan *p);

#ifdef __cplusplus
}
#endif
#endif /* SINNAMON_PLAN_H */
