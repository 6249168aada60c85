// Recorded searches: one whole batched search (and for the learned variant
// the k' network before it) captured into a CUDA graph and replayed with a
// single launch.  The kernels are the ones sinn_search_ctx and
// sinn_search_learned_ctx launch; this file only records and replays them.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "../../include/sinnamon_plan.h"
#include "sinn_internal.cuh"

int sinn_mlp_refresh(sinn_mlp *m, cudaStream_t s);  // mlp.cu
uint64_t sinn_mlp_version(sinn_mlp *m);              // mlp.cu

#define CK(x)                                          \
  do {                                                 \
    if (int _st = sinn_check_cuda(x)) return _st;      \
  } while (0)

struct sinn_plan {
  sinn_index *ix = nullptr;
  sinn_mlp *m = nullptr;
  sinn_ctx *ctx = nullptr;
  void *act = nullptr;  // activations of the network (learned mode)
  uint64_t act_bytes = 0;
  const uint64_t *q_indptr = nullptr;
  const uint32_t *q_indices = nullptr;
  const float *q_values = nullptr;
  const uint32_t *k_prime = nullptr;
  uint32_t n_q = 0, k = 0, kp_min = 0, kp_max = 0;
  uint32_t *out_ids = nullptr;
  float *out_scores = nullptr;
  uint32_t *out_kprime = nullptr;
  cudaStream_t cs = nullptr;  // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t version = ~0ull;   // index shape the recording belongs to
  uint64_t mlp_version = 0;   // network policy the recording belongs to
  uint64_t launches = 0;      // kernels one replay runs
  uint64_t recordings = 0;
  std::vector<sinn_index::Span> spans;  // phase events recorded inside the graph
};

namespace {

void drop_recording(sinn_plan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto &sp : p->spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  p->exec = nullptr;
  p->graph = nullptr;
  p->spans.clear();
}

int issue(sinn_plan *p, cudaStream_t s) {
  if (p->m)
    return sinn_search_learned_ctx(p->ctx, p->ix, p->m, p->act, p->act_bytes, p->q_indptr,
                                   p->q_indices, p->q_values, p->n_q, p->k, p->kp_min,
                                   p->kp_max, p->out_ids, p->out_scores, p->out_kprime, s);
  return sinn_search_ctx(p->ctx, p->q_indptr, p->q_indices, p->q_values, p->n_q, p->k,
                         p->k_prime, p->kp_max, p->out_ids, p->out_scores, s);
}

// Capture the search on the plan's own stream.  Phase events are always
// recorded into the graph (they then belong to the plan), and the kernels
// counted while capturing are charged to each replay instead.
int record(sinn_plan *p) {
  sinn_index *ix = p->ix;
  if (p->m) {
    int st = sinn_mlp_refresh(p->m, p->cs);
    if (st) return st;
    CK(cudaStreamSynchronize(p->cs));
  }
  const bool tm = ix->tm_on;
  const size_t ns = ix->tm_spans.size();
  const uint64_t l0 = ix->launches;
  ix->tm_on = true;
  if (cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    ix->tm_on = tm;
    (void)cudaGetLastError();
    return SINN_ECUDA;
  }
  const int st = issue(p, p->cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->cs, &g);
  ix->tm_on = tm;
  std::vector<sinn_index::Span> spans(ix->tm_spans.begin() + ns, ix->tm_spans.end());
  ix->tm_spans.resize(ns);
  const uint64_t nl = ix->launches - l0;
  ix->launches = l0;
  cudaGraphExec_t x = nullptr;
  const bool ok = st == SINN_OK && e == cudaSuccess && g &&
                  cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    for (auto &sp : spans) {
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    }
    return st ? st : SINN_ECUDA;
  }
  drop_recording(p);
  p->graph = g;
  p->exec = x;
  p->spans = std::move(spans);
  p->launches = nl;
  p->version = ix->shape_version;
  p->mlp_version = sinn_mlp_version(p->m);
  p->recordings++;
  return SINN_OK;
}

}  // namespace

extern "C" int sinn_plan_create(sinn_index *ix, sinn_mlp *mlp, const uint64_t *q_indptr,
                                const uint32_t *q_indices, const float *q_values,
                                const uint32_t *k_prime, uint32_t n_q, uint32_t k,
                                uint32_t k_prime_min, uint32_t k_prime_max, uint32_t *out_ids,
                                float *out_scores, uint32_t *out_kprime, uint64_t scratch_bytes,
                                sinn_plan **out) {
  if (!ix || !out || !q_indptr || !out_ids || !out_scores || n_q == 0) return SINN_EINVAL;
  if (k == 0 || k > SINN_MAX_K || k_prime_max < k) return SINN_EINVAL;
  if (mlp && (k_prime_min < k || k_prime_max < k_prime_min)) return SINN_EINVAL;
  *out = nullptr;
  SinnDevice dev_guard_(ix->device);
  sinn_plan *p = new (std::nothrow) sinn_plan();
  if (!p) return SINN_ENOMEM;
  p->ix = ix;
  p->m = mlp;
  p->q_indptr = q_indptr;
  p->q_indices = q_indices;
  p->q_values = q_values;
  p->k_prime = mlp ? nullptr : k_prime;
  p->n_q = n_q;
  p->k = k;
  p->kp_min = k_prime_min;
  p->kp_max = k_prime_max;
  p->out_ids = out_ids;
  p->out_scores = out_scores;
  p->out_kprime = out_kprime;
  int st = sinn_ctx_create(ix, scratch_bytes, &p->ctx);
  if (!st && mlp) {
    p->act_bytes = sinn_mlp_act_bytes(mlp, n_q);
    if (sinn_dev_malloc((void **)&p->act, p->act_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      st = SINN_ENOMEM;
    }
  }
  if (!st && cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    st = SINN_ECUDA;
  }
  if (st) {
    sinn_plan_destroy(p);
    return st;
  }
  *out = p;
  return SINN_OK;
}

extern "C" int sinn_plan_run(sinn_plan *p, void *stream) {
  if (!p) return SINN_EINVAL;
  sinn_index *ix = p->ix;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  if (!p->exec || p->version != ix->shape_version || p->mlp_version != sinn_mlp_version(p->m)) {
    // the capture stream must see the caller's earlier work (index updates)
    cudaEvent_t ready;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, s));
    CK(cudaStreamWaitEvent(p->cs, ready, 0));
    cudaEventDestroy(ready);
    if (p->m && sinn_mlp_act_bytes(p->m, p->n_q) > p->act_bytes) {
      // a policy set since creation may want more network rows
      CK(cudaStreamSynchronize(p->cs));
      CK(cudaFree(p->act));
      p->act = nullptr;
      p->act_bytes = 0;
      const uint64_t need = sinn_mlp_act_bytes(p->m, p->n_q);
      CK(sinn_dev_malloc((void **)&p->act, need));
      p->act_bytes = need;
    }
    if ((st = record(p))) return st;
  }
  if (p->m && (st = sinn_mlp_refresh(p->m, s))) return st;
  CK(cudaGraphLaunch(p->exec, s));
  ix->launches += p->launches;
  if (ix->tm_on && !p->spans.empty()) {
    CK(cudaEventSynchronize(p->spans.back().b));
    for (auto &sp : p->spans) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, sp.a, sp.b));
      if (sp.phase >= 0 && sp.phase < SINN_PHASES) {
        ix->tm_acc_ms[sp.phase] += ms;
        ix->tm_acc_spans[sp.phase] += 1;
      }
    }
  }
  return SINN_OK;
}

extern "C" uint64_t sinn_plan_recordings(sinn_plan *p) { return p ? p->recordings : 0; }

extern "C" int sinn_plan_destroy(sinn_plan *p) {
  if (!p) return SINN_OK;
  SinnDevice dev_guard_(p->ix->device);
  cudaDeviceSynchronize();
  drop_recording(p);
  if (p->cs) cudaStreamDestroy(p->cs);
  if (p->act) cudaFree(p->act);
  if (p->ctx) sinn_ctx_destroy(p->ctx);
  delete p;
  return SINN_OK;
}
