/*
 * sinnamon_kprime.h -- learned per-query k' for SINNAMON (C ABI).
 *
 * The paper notes that the re-ranking depth k' of Alg. 7 could be chosen per
 * query from the expected error of the sketch (end of Sec. 5.3, and the
 * question it leaves open in Sec. 7).  This part of the library learns that
 * choice: a small network reads features of a query and predicts log2 of the
 * smallest k' at which Alg. 7 still returns at least 9 of the exact top 10.
 * Conventions (status codes, device/host pointers, streams, ownership) are
 * those of sinnamon.h.
 */
#ifndef SINNAMON_KPRIME_H
#define SINNAMON_KPRIME_H

#include <stdint.h>

#include "sinnamon.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SINN_KP_TOP 16                       /* terms whose list lengths are features */
#define SINN_KP_FEATURES (3 + SINN_KP_TOP)   /* nnz, L1, L2, 16 list lengths */

typedef struct sinn_mlp sinn_mlp; /* opaque; owned by the library */

/* Per-query features for n_q queries (device CSR as in sinn_search) into
 * device out[n_q * SINN_KP_FEATURES], row-major: log2(1 + number of
 * non-zeros), the L1 and L2 norms of the non-zeros, then log2(1 + |I[j]|) for
 * the SINN_KP_TOP terms of largest |q_j| (Alg. 6 order; 0 past the last
 * term), |I[j]| counting the postings of coordinate j in the index. */
int sinn_kp_features(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                     const float *q_values, uint32_t n_q, float *out, void *stream);

/* A network n_in -> hidden -> hidden -> 1 with ReLU, fp32 master weights
 * initialised from seed (uniform, fan-in scaled), bf16 tensor-core GEMMs with
 * fp32 accumulation.  Inputs are standardised with the normaliser (mean 0,
 * stdev 1 until set).  EINVAL for n_in = 0 or > 1024, hidden = 0 or > 4096.
 * *out is NULL after any error. */
int sinn_mlp_create(uint32_t n_in, uint32_t hidden, uint64_t seed, sinn_mlp **out);
int sinn_mlp_destroy(sinn_mlp *m);

/* Number of parameters; flat order W1 [hidden x n_in], b1 [hidden],
 * W2 [hidden x hidden], b2 [hidden], w3 [hidden], b3 [1], row-major. */
uint64_t sinn_mlp_num_params(sinn_mlp *m);

/* Copy parameters (which = 0) or the last computed gradients (which = 1) to
 * host out[num_params]; waits for the device. */
int sinn_mlp_params(sinn_mlp *m, float *host_out, int which);

/* Replace the parameters from host in[num_params]. */
int sinn_mlp_set_params(sinn_mlp *m, const float *host_in);

/* Feature standardisation: x' = (x - mean) / stdev, host arrays of n_in. */
int sinn_mlp_set_normalizer(sinn_mlp *m, const float *mean, const float *stdev);

/* y[r] = network(X[r]) for B rows: device X[B * n_in], device y[B]. */
int sinn_mlp_forward(sinn_mlp *m, const float *X, uint32_t B, float *y, void *stream);

/* Gradient of the mean pinball loss at quantile tau (0 < tau < 1) of targets
 * t[B] (device) with respect to all parameters, into device
 * grad_out[num_params] (nullable) and the loss into device loss_out[1]
 * (nullable).  The pinball loss of residual u = t - y is tau*u for u >= 0 and
 * (tau-1)*u otherwise. */
int sinn_mlp_grad(sinn_mlp *m, const float *X, const float *t, uint32_t B, float tau,
                  float *grad_out, float *loss_out, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that gradient. */
int sinn_mlp_train_step(sinn_mlp *m, const float *X, const float *t, uint32_t B, float tau,
                        float lr, float *loss_out, void *stream);

/* Wait for the stream, then return and clear the network's device error:
 * SINN_EDEVICE if a bounded wait in one of its tensor-core GEMMs (forward,
 * gradient or training step) ran out since the last call, else SINN_OK.  In
 * sinn_search_learned the same errors go to the index (sinn_sync). */
int sinn_mlp_sync(sinn_mlp *m, void *stream);

/* sinn_search with k'[q] = clamp(ceil(2^network(features(q))), k_prime_min,
 * k_prime_max); the network must have n_in = SINN_KP_FEATURES.  With a
 * policy (below), the per-query k' and Alg. 6 budget the policy chooses
 * instead.  out_kprime (device uint32[n_q], nullable) receives the k' used
 * per query. */
int sinn_search_learned(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                        const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                        uint32_t k, uint32_t k_prime_min, uint32_t k_prime_max,
                        uint32_t *out_ids, float *out_scores, uint32_t *out_kprime,
                        void *stream);

/* ---- Learned Alg. 6 budget with k' --------------------------------------
 * Alg. 6 may stop scoring once a time budget is spent (its anytime break,
 * counted in postings here, as in sinn_set_budget), and Alg. 7 can recover
 * what a short budget loses with a deeper re-rank.  A policy lets the network
 * pick both per query: for each of a few budget levels it predicts the least
 * k' that keeps 9 of the exact top 10 at that level, and the query takes the
 * level of least predicted cost.
 *   Level l scores the terms of Alg. 6, in its order, until the postings
 *   visited reach ceil(P_q / 2^shift[l]), P_q being the query's postings
 *   with no budget (sinn_query_postings); shift[0] must be 0 (the whole
 *   query) and the shifts strictly increase (at most 31).
 *   The network then has n_in = SINN_KP_FEATURES + 1 inputs: the query's
 *   features followed by -shift[l], and its output for that row is log2 of
 *   that level's k'.
 *   k'_l = max(ceil(2^v), k_prime_min) with v = output + margin clamped
 *   to [0, 31] (the margin may be negative); the level is feasible when
 *   k'_l <= k_prime_max.  The feasible level of least
 *   posting_cost * (its postings) + k'_l is chosen (ties: the earlier level,
 *   the larger budget); when no level is feasible, level 0 at k_prime_max.
 *   posting_cost is the time of scoring one posting in units of the time of
 *   re-ranking one candidate (a measured ratio).
 * With a policy set, sinn_search_learned, sinn_search_learned_ctx and
 * learned plans search with the chosen per-query k' and budget (the re-rank
 * always takes every term).  Set the policy before sizing activation
 * buffers with sinn_mlp_act_bytes. */
#define SINN_KP_MAX_LEVELS 8
typedef struct sinn_kp_policy {
  uint32_t n_levels;                   /* 1..SINN_KP_MAX_LEVELS */
  uint32_t shift[SINN_KP_MAX_LEVELS];  /* budget P_q / 2^shift[l]; shift[0] = 0 */
  float posting_cost;                  /* >= 0: one posting's cost in candidates */
  float margin;                        /* added to each predicted log2 k'; finite */
} sinn_kp_policy;

/* Set (p != NULL) or clear (p == NULL) the network's policy.  EINVAL for a
 * malformed policy or a network without SINN_KP_FEATURES + 1 inputs. */
int sinn_mlp_set_policy(sinn_mlp *m, const sinn_kp_policy *p);

/* The current policy into *out (n_levels = 0: none). */
int sinn_mlp_get_policy(sinn_mlp *m, sinn_kp_policy *out);

/* The learned search's choice alone: features, network and (with a policy)
 * the level choice for n_q queries (device CSR), into device
 * out_kprime[n_q] and, nullable, device out_budget[n_q] (Alg. 6 budgets in
 * postings, 0 = the whole query; all 0 without a policy).  Searching with
 * sinn_search_kpb at these values gives sinn_search_learned's results. */
int sinn_kp_choose(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                   const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                   uint32_t k_prime_min, uint32_t k_prime_max, uint32_t *out_kprime,
                   uint64_t *out_budget, void *stream);

/* sinn_search_learned with every buffer in host memory (queries as CSR, the
 * results and, nullable, the k' per query): the call copies the queries to
 * the device, searches, copies the results back and waits for them; device
 * errors are returned directly. */
int sinn_search_learned_host(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                             const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                             uint32_t k, uint32_t k_prime_min, uint32_t k_prime_max,
                             uint32_t *out_ids, float *out_scores, uint32_t *out_kprime,
                             void *stream);

/* Device bytes of the activation buffer sinn_search_learned_ctx needs for
 * n_q queries. */
uint64_t sinn_mlp_act_bytes(sinn_mlp *m, uint32_t rows);

/* sinn_search_learned on a search context (sinnamon.h), with the network's
 * activations in the caller's device buffer act[act_bytes] so that several
 * contexts can use one network at once.  The network must not be trained
 * while such searches run. */
int sinn_search_learned_ctx(sinn_ctx *c, sinn_index *ix, sinn_mlp *m, void *act,
                            uint64_t act_bytes, const uint64_t *q_indptr,
                            const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                            uint32_t k, uint32_t k_prime_min, uint32_t k_prime_max,
                            uint32_t *out_ids, float *out_scores, uint32_t *out_kprime,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SINNAMON_KPRIME_H */
