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
 * k_prime_max); the network must have n_in = SINN_KP_FEATURES.  out_kprime
 * (device uint32[n_q], nullable) receives the k' used per query. */
int sinn_search_learned(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
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
