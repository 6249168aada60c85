/*
 * CPU oracle for SINNAMON (Bruch, Nardini, Ingber, Liberty: "An Approximate
 * Algorithm for Maximum Inner Product Search over Streaming Sparse Vectors").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library, and the library never calls it.
 *
 * Arithmetic is FP64 throughout: document and query values arrive as fp32 and
 * are widened exactly; products and sums are formed in double.
 *
 * What each function follows:
 *   orc_mix64 / hash table   -- the paper only asks for "h independent random
 *                               mappings pi_o: [n] -> [m]" (Alg. 5 inputs,
 *                               Sec. 4.1).  Reading taken: pi_o(j) =
 *                               mix64(seed ^ ((o+1)*G) ^ j) mod m, where mix64
 *                               is the output function of SplitMix64 (Steele,
 *                               Lea, Flood, OOPSLA 2014) and G its gamma.
 *   orc_insert               -- Alg. 5 (indexing) + id reuse of Sec. 4.3;
 *                               with orc_set_sketch_bf16 the bins are stored
 *                               as bfloat16 (Sec. 4.1 notes), U rounded up
 *                               and L rounded down (a reading: bounds stay
 *                               bounds).
 *   orc_delete               -- Sec. 4.3 (remove i from every I[j], leave
 *                               column i of the sketch as it is, free id i).
 *   orc_scores               -- Alg. 6 (scoring), T = infinity.
 *   orc_scores_anytime       -- Alg. 6 with a time budget, read as postings:
 *                               terms run in Alg. 6 order and the loop breaks
 *                               after the first term at which the postings
 *                               visited so far reach the budget (the check
 *                               at the end of the term loop).
 *   find_largest             -- Alg. 3 (FindLargest, binary heap).
 *   orc_search               -- Alg. 7 (ranking: top-k' by approximate score,
 *                               exact re-rank from the vector store, top-k);
 *                               orc_search_anytime scores with a budget.
 *   orc_exact_*              -- Eq. 2 (MIPS) by brute force over the store.
 *   orc_linscan_*            -- Alg. 1 / Alg. 2 (LinScan), exact.
 *
 * Readings of points the paper leaves open (each one is a choice):
 *   - empty sketch bin: u = -inf, l = +inf (identities of max / min);
 *   - ids: a new vector takes the smallest free id, else the next fresh id;
 *   - ties everywhere: larger score first, then smaller id;
 *   - query coordinates with equal |q_j|: smaller j first;
 *   - FindLargest considers live ids only (vacant columns are not results);
 *   - zero entries are not non-zeros: they are not indexed or sketched.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOTFOUND 2
#define ORC_ENOMEM 3

/* ------------------------------------------------------------------ hash */

/* SplitMix64 output function (the "mix" step applied to the advanced state). */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static const uint64_t ORC_GAMMA = 0x9E3779B97F4A7C15ULL;

/* pi_o(j) for o in [0, h): the o-th of the h random mappings of Alg. 5. */
static uint32_t orc_pi(uint64_t seed, uint32_t o, uint32_t j, uint32_t m) {
  uint64_t x = seed ^ ((uint64_t)(o + 1) * ORC_GAMMA) ^ (uint64_t)j;
  return (uint32_t)(orc_mix64(x) % (uint64_t)m);
}

/* --------------------------------------------------------------- index */

typedef struct {
  uint32_t *ids;
  uint32_t len, cap;
} orc_plist;

typedef struct orc_index {
  uint32_t n, m, h;
  int sketch_bf16; /* bins stored as bfloat16: U rounded up, L rounded down */
  uint32_t *pi; /* n*h: pi[j*h + o] */
  /* per id slot */
  uint32_t n_slots, cap_slots; /* n_slots = next fresh id */
  uint8_t *live;
  double *U, *L;         /* column i at U[i*m .. i*m+m) */
  uint32_t **doc_idx;    /* vector store S: non-zero coordinates, ascending */
  double **doc_val;      /* and their values (fp32 inputs widened) */
  uint32_t *doc_nnz;
  uint32_t live_count;
  /* free ids: binary min-heap */
  uint32_t *free_heap;
  uint32_t n_free, cap_free;
  /* inverted index I: coordinate -> ascending list of ids */
  orc_plist *lists;
} orc_index;

/* bfloat16 storage of a sketch bin (the paper stores sketches as bfloat16,
 * Sec. 4.1 notes).  bfloat16 values are the floats whose 16 low bits are
 * zero.  Reading taken: an upper bin takes the least bfloat16 >= its value
 * and a lower bin the greatest bfloat16 <= it, so decoded values stay upper
 * / lower bounds (Thm. 1 keeps holding).  x is a float value (or +-inf). */
static double bf16_round(double x, int up) {
  float f = (float)x;
  uint32_t b;
  memcpy(&b, &f, 4);
  uint32_t t = b & 0xFFFF0000u; /* toward zero */
  float tf;
  memcpy(&tf, &t, 4);
  if (tf == f) return x;        /* representable */
  /* toward zero is up for a negative value and down for a positive one */
  int toward_zero_ok = (f < 0.0f) ? up : !up;
  if (!toward_zero_ok) t += 0x10000u; /* one bfloat16 step away from zero */
  memcpy(&tf, &t, 4);
  return (double)tf;
}

/* Store bins as bfloat16 from now on (only on an empty index). */
int orc_set_sketch_bf16(orc_index *ix, int on);

static void *xrealloc(void *p, size_t bytes) {
  void *q = realloc(p, bytes ? bytes : 1);
  return q;
}

static orc_index *orc_alloc(uint32_t n, uint32_t m, uint32_t h) {
  if (n == 0 || m == 0 || h == 0 || h > m) return NULL;
  orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
  if (!ix) return NULL;
  ix->n = n;
  ix->m = m;
  ix->h = h;
  ix->pi = (uint32_t *)calloc((size_t)n * h, sizeof(uint32_t));
  ix->lists = (orc_plist *)calloc(n, sizeof(orc_plist));
  if (!ix->pi || !ix->lists) {
    free(ix->pi);
    free(ix->lists);
    free(ix);
    return NULL;
  }
  return ix;
}

orc_index *orc_create(uint32_t n, uint32_t m, uint32_t h, uint64_t seed) {
  orc_index *ix = orc_alloc(n, m, h);
  if (!ix) return NULL;
  for (uint32_t j = 0; j < n; ++j)
    for (uint32_t o = 0; o < h; ++o) ix->pi[(size_t)j * h + o] = orc_pi(seed, o, j, m);
  return ix;
}

/* Same as orc_create with the mappings given explicitly (table[j*h+o] < m);
 * used by tests that need, e.g., an injective mapping. */
orc_index *orc_create_table(uint32_t n, uint32_t m, uint32_t h, const uint32_t *table) {
  orc_index *ix = orc_alloc(n, m, h);
  if (!ix) return NULL;
  for (size_t t = 0; t < (size_t)n * h; ++t) {
    if (table[t] >= m) {
      free(ix->pi);
      free(ix->lists);
      free(ix);
      return NULL;
    }
    ix->pi[t] = table[t];
  }
  return ix;
}

void orc_destroy(orc_index *ix) {
  if (!ix) return;
  for (uint32_t j = 0; j < ix->n; ++j) free(ix->lists[j].ids);
  for (uint32_t i = 0; i < ix->n_slots; ++i) {
    free(ix->doc_idx[i]);
    free(ix->doc_val[i]);
  }
  free(ix->lists);
  free(ix->pi);
  free(ix->live);
  free(ix->U);
  free(ix->L);
  free(ix->doc_idx);
  free(ix->doc_val);
  free(ix->doc_nnz);
  free(ix->free_heap);
  free(ix);
}

int orc_set_sketch_bf16(orc_index *ix, int on) {
  if (ix->n_slots) return ORC_EINVAL;
  ix->sketch_bf16 = on ? 1 : 0;
  return ORC_OK;
}

void orc_hash_table(const orc_index *ix, uint32_t *out) {
  memcpy(out, ix->pi, (size_t)ix->n * ix->h * sizeof(uint32_t));
}

uint32_t orc_n_slots(const orc_index *ix) { return ix->n_slots; }
uint32_t orc_live_count(const orc_index *ix) { return ix->live_count; }
int orc_is_live(const orc_index *ix, uint32_t id) { return id < ix->n_slots && ix->live[id]; }
void orc_live_mask(const orc_index *ix, uint8_t *out) { memcpy(out, ix->live, ix->n_slots); }

/* free-id min-heap */
static void heap_push_u32(orc_index *ix, uint32_t v) {
  if (ix->n_free == ix->cap_free) {
    ix->cap_free = ix->cap_free ? 2 * ix->cap_free : 64;
    ix->free_heap = (uint32_t *)xrealloc(ix->free_heap, ix->cap_free * sizeof(uint32_t));
  }
  uint32_t c = ix->n_free++;
  ix->free_heap[c] = v;
  while (c > 0) {
    uint32_t p = (c - 1) / 2;
    if (ix->free_heap[p] <= ix->free_heap[c]) break;
    uint32_t t = ix->free_heap[p];
    ix->free_heap[p] = ix->free_heap[c];
    ix->free_heap[c] = t;
    c = p;
  }
}

static uint32_t heap_pop_u32(orc_index *ix) {
  uint32_t top = ix->free_heap[0];
  ix->free_heap[0] = ix->free_heap[--ix->n_free];
  uint32_t c = 0;
  for (;;) {
    uint32_t l = 2 * c + 1, r = l + 1, s = c;
    if (l < ix->n_free && ix->free_heap[l] < ix->free_heap[s]) s = l;
    if (r < ix->n_free && ix->free_heap[r] < ix->free_heap[s]) s = r;
    if (s == c) break;
    uint32_t t = ix->free_heap[s];
    ix->free_heap[s] = ix->free_heap[c];
    ix->free_heap[c] = t;
    c = s;
  }
  return top;
}

static int grow_slots(orc_index *ix, uint32_t need) {
  if (need <= ix->cap_slots) return ORC_OK;
  uint32_t nc = ix->cap_slots ? ix->cap_slots : 1024;
  while (nc < need) nc *= 2;
  ix->live = (uint8_t *)xrealloc(ix->live, nc);
  ix->U = (double *)xrealloc(ix->U, (size_t)nc * ix->m * sizeof(double));
  ix->L = (double *)xrealloc(ix->L, (size_t)nc * ix->m * sizeof(double));
  ix->doc_idx = (uint32_t **)xrealloc(ix->doc_idx, nc * sizeof(uint32_t *));
  ix->doc_val = (double **)xrealloc(ix->doc_val, nc * sizeof(double *));
  ix->doc_nnz = (uint32_t *)xrealloc(ix->doc_nnz, nc * sizeof(uint32_t));
  if (!ix->live || !ix->U || !ix->L || !ix->doc_idx || !ix->doc_val || !ix->doc_nnz)
    return ORC_ENOMEM;
  for (uint32_t i = ix->cap_slots; i < nc; ++i) {
    ix->live[i] = 0;
    ix->doc_idx[i] = NULL;
    ix->doc_val[i] = NULL;
    ix->doc_nnz[i] = 0;
  }
  ix->cap_slots = nc;
  return ORC_OK;
}

/* Insert id into the ascending list (no duplicates by construction). */
static void list_insert(orc_plist *li, uint32_t id) {
  if (li->len == li->cap) {
    li->cap = li->cap ? 2 * li->cap : 8;
    li->ids = (uint32_t *)xrealloc(li->ids, li->cap * sizeof(uint32_t));
  }
  uint32_t lo = 0, hi = li->len; /* first position with ids[pos] > id */
  if (li->len == 0 || li->ids[li->len - 1] < id) {
    lo = li->len;
  } else {
    while (lo < hi) {
      uint32_t mid = (lo + hi) / 2;
      if (li->ids[mid] < id) lo = mid + 1;
      else hi = mid;
    }
  }
  memmove(li->ids + lo + 1, li->ids + lo, (size_t)(li->len - lo) * sizeof(uint32_t));
  li->ids[lo] = id;
  li->len++;
}

static int list_remove(orc_plist *li, uint32_t id) {
  uint32_t lo = 0, hi = li->len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) / 2;
    if (li->ids[mid] < id) lo = mid + 1;
    else hi = mid;
  }
  if (lo >= li->len || li->ids[lo] != id) return ORC_ENOTFOUND;
  memmove(li->ids + lo, li->ids + lo + 1, (size_t)(li->len - lo - 1) * sizeof(uint32_t));
  li->len--;
  return ORC_OK;
}

/* Validate one CSR batch: coordinates < n and strictly increasing per row,
 * values finite.  Nothing is changed when this fails. */
static int validate_csr(uint32_t n, const uint64_t *indptr, const uint32_t *indices,
                        const float *values, uint32_t rows) {
  for (uint32_t r = 0; r < rows; ++r) {
    if (indptr[r + 1] < indptr[r]) return ORC_EINVAL;
    for (uint64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
      if (indices[p] >= n) return ORC_EINVAL;
      if (p > indptr[r] && indices[p] <= indices[p - 1]) return ORC_EINVAL;
      if (!isfinite(values[p])) return ORC_EINVAL;
    }
  }
  return ORC_OK;
}

/* Alg. 5 for each row of the batch, in batch order.  out_ids[r] receives the
 * id given to row r: the smallest free id if any (Sec. 4.3), else a fresh one. */
int orc_insert(orc_index *ix, const uint64_t *indptr, const uint32_t *indices,
               const float *values, uint32_t n_docs, uint32_t *out_ids) {
  int st = validate_csr(ix->n, indptr, indices, values, n_docs);
  if (st) return st;
  for (uint32_t r = 0; r < n_docs; ++r) {
    uint32_t id;
    if (ix->n_free > 0) {
      id = heap_pop_u32(ix);
    } else {
      if (ix->n_slots == 0xFFFFFFFEu) return ORC_ENOMEM;
      if (grow_slots(ix, ix->n_slots + 1)) return ORC_ENOMEM;
      id = ix->n_slots++;
    }
    if (out_ids) out_ids[r] = id;

    /* nz(x_i) = { j : x_i[j] != 0 } (Alg. 5); the vector is kept in
     * the store S for re-ranking. */
    uint32_t cnt = 0;
    for (uint64_t p = indptr[r]; p < indptr[r + 1]; ++p)
      if (values[p] != 0.0f) cnt++;
    free(ix->doc_idx[id]);
    free(ix->doc_val[id]);
    ix->doc_idx[id] = (uint32_t *)malloc((cnt ? cnt : 1) * sizeof(uint32_t));
    ix->doc_val[id] = (double *)malloc((cnt ? cnt : 1) * sizeof(double));
    ix->doc_nnz[id] = cnt;
    uint32_t c = 0;
    for (uint64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
      if (values[p] == 0.0f) continue;
      ix->doc_idx[id][c] = indices[p];
      ix->doc_val[id][c] = (double)values[p];
      c++;
    }

    /* I[j].Insert(i) for all j in nz(x_i) (Alg. 5). */
    for (uint32_t t = 0; t < cnt; ++t) list_insert(&ix->lists[ix->doc_idx[id][t]], id);

    /* Alg. 5, sketch: u[k] is the max and l[k] the min of x_i[j] over the
     * non-zeros j that some mapping sends to k.  Visiting each (j, o) pair
     * once and folding x_i[j] into bin pi_o(j) forms exactly these set
     * maxima / minima.  A bin no non-zero reaches keeps -inf / +inf. */
    double *u = ix->U + (size_t)id * ix->m;
    double *l = ix->L + (size_t)id * ix->m;
    for (uint32_t k = 0; k < ix->m; ++k) {
      u[k] = -INFINITY;
      l[k] = INFINITY;
    }
    for (uint32_t t = 0; t < cnt; ++t) {
      uint32_t j = ix->doc_idx[id][t];
      double v = ix->doc_val[id][t];
      for (uint32_t o = 0; o < ix->h; ++o) {
        uint32_t k = ix->pi[(size_t)j * ix->h + o];
        if (v > u[k]) u[k] = v;
        if (v < l[k]) l[k] = v;
      }
    }
    if (ix->sketch_bf16)
      for (uint32_t k = 0; k < ix->m; ++k) {
        u[k] = bf16_round(u[k], 1);
        l[k] = bf16_round(l[k], 0);
      }
    ix->live[id] = 1;
    ix->live_count++;
  }
  return ORC_OK;
}

/* Sec. 4.3: remove i from every inverted list, leave column i of the sketch
 * untouched, and make i available again.  The whole batch is checked first
 * (every id live, no repeats); nothing changes if the check fails. */
int orc_delete(orc_index *ix, const uint32_t *ids, uint32_t n_ids) {
  for (uint32_t a = 0; a < n_ids; ++a) {
    if (!orc_is_live(ix, ids[a])) return ORC_ENOTFOUND;
    for (uint32_t b = 0; b < a; ++b)
      if (ids[b] == ids[a]) return ORC_EINVAL;
  }
  for (uint32_t a = 0; a < n_ids; ++a) {
    uint32_t id = ids[a];
    for (uint32_t t = 0; t < ix->doc_nnz[id]; ++t) list_remove(&ix->lists[ix->doc_idx[id][t]], id);
    free(ix->doc_idx[id]);
    free(ix->doc_val[id]);
    ix->doc_idx[id] = NULL;
    ix->doc_val[id] = NULL;
    ix->doc_nnz[id] = 0;
    ix->live[id] = 0;
    ix->live_count--;
    heap_push_u32(ix, id);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ inspection */

void orc_sketch_column(const orc_index *ix, uint32_t id, double *u, double *l) {
  memcpy(u, ix->U + (size_t)id * ix->m, ix->m * sizeof(double));
  memcpy(l, ix->L + (size_t)id * ix->m, ix->m * sizeof(double));
}

uint32_t orc_list_len(const orc_index *ix, uint32_t j) { return ix->lists[j].len; }

void orc_list(const orc_index *ix, uint32_t j, uint32_t *out) {
  memcpy(out, ix->lists[j].ids, ix->lists[j].len * sizeof(uint32_t));
}

uint32_t orc_doc_nnz(const orc_index *ix, uint32_t id) { return ix->doc_nnz[id]; }

void orc_doc(const orc_index *ix, uint32_t id, uint32_t *idx, double *val) {
  memcpy(idx, ix->doc_idx[id], ix->doc_nnz[id] * sizeof(uint32_t));
  memcpy(val, ix->doc_val[id], ix->doc_nnz[id] * sizeof(double));
}

/* --------------------------------------------------------------- queries */

typedef struct {
  uint32_t j;
  double v;
} orc_qterm;

/* Alg. 6: query terms by descending |q_j|; equal magnitudes by ascending j. */
static int qterm_cmp(const void *a, const void *b) {
  const orc_qterm *x = (const orc_qterm *)a, *y = (const orc_qterm *)b;
  double ax = fabs(x->v), ay = fabs(y->v);
  if (ax > ay) return -1;
  if (ax < ay) return 1;
  return (x->j < y->j) ? -1 : (x->j > y->j);
}

/* nz(q), sorted as Alg. 6 asks.  Returns the number of terms. */
static uint32_t query_terms(const uint32_t *qi, const float *qv, uint32_t qnnz, orc_qterm *out) {
  uint32_t c = 0;
  for (uint32_t t = 0; t < qnnz; ++t) {
    if (qv[t] == 0.0f) continue;
    out[c].j = qi[t];
    out[c].v = (double)qv[t];
    c++;
  }
  qsort(out, c, sizeof(orc_qterm), qterm_cmp);
  return c;
}

static int validate_query(const orc_index *ix, const uint32_t *qi, const float *qv, uint32_t qnnz) {
  uint64_t ip[2] = {0, qnnz};
  return validate_csr(ix->n, ip, qi, qv, 1);
}

/* Alg. 6 with T = infinity.  scores[i] for every id slot i < n_slots
 * (vacant slots are 0: no list holds them).  If mag is given, mag[i] receives
 * sum |q_j * x~_j(i)| over the same terms, the magnitude that floating-point
 * error in scores[i] scales with. */
static void alg6_scores(const orc_index *ix, const orc_qterm *terms, uint32_t nt, double *scores,
                        double *mag) {
  memset(scores, 0, (size_t)ix->n_slots * sizeof(double));
  if (mag) memset(mag, 0, (size_t)ix->n_slots * sizeof(double));
  for (uint32_t t = 0; t < nt; ++t) {
    uint32_t j = terms[t].j;
    double qj = terms[t].v;
    const uint32_t *K = ix->pi + (size_t)j * ix->h; /* K = {pi_o(j)} */
    const orc_plist *li = &ix->lists[j];
    for (uint32_t p = 0; p < li->len; ++p) {
      uint32_t i = li->ids[p];
      double xt;
      if (qj > 0) { /* least upper bound */
        xt = INFINITY;
        for (uint32_t o = 0; o < ix->h; ++o) {
          double c = ix->U[(size_t)i * ix->m + K[o]];
          if (c < xt) xt = c;
        }
      } else { /* greatest lower bound */
        xt = -INFINITY;
        for (uint32_t o = 0; o < ix->h; ++o) {
          double c = ix->L[(size_t)i * ix->m + K[o]];
          if (c > xt) xt = c;
        }
      }
      double s = qj * xt;
      scores[i] += s;
      if (mag) mag[i] += fabs(s);
    }
  }
}

/* The anytime break of Alg. 6 with the budget counted in postings: the
 * number of sorted terms scored.  Budget 0 means T = infinity. */
static uint32_t anytime_terms(const orc_index *ix, const orc_qterm *terms, uint32_t nt,
                              uint64_t budget) {
  if (budget == 0) return nt;
  uint64_t visited = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    visited += ix->lists[terms[t].j].len;
    if (visited >= budget) return t + 1; /* break after this term */
  }
  return nt;
}

int orc_scores_anytime(const orc_index *ix, const uint32_t *qi, const float *qv, uint32_t qnnz,
                       uint64_t budget, double *scores, double *mag) {
  if (validate_query(ix, qi, qv, qnnz)) return ORC_EINVAL;
  orc_qterm *terms = (orc_qterm *)malloc((qnnz ? qnnz : 1) * sizeof(orc_qterm));
  uint32_t nt = query_terms(qi, qv, qnnz, terms);
  alg6_scores(ix, terms, anytime_terms(ix, terms, nt, budget), scores, mag);
  free(terms);
  return ORC_OK;
}

int orc_scores(const orc_index *ix, const uint32_t *qi, const float *qv, uint32_t qnnz,
               double *scores, double *mag) {
  return orc_scores_anytime(ix, qi, qv, qnnz, 0, scores, mag);
}

/* ---- Alg. 3: FindLargest with a binary heap -----------------------------
 * Items are (value, key) pairs.  "a ranks above b" means a larger value, or an
 * equal value and a smaller key.  The heap keeps the k items that rank highest;
 * its root is the lowest-ranked of them. */
typedef struct {
  double value;
  uint32_t key;
} orc_item;

static int ranks_above(orc_item a, orc_item b) {
  if (a.value > b.value) return 1;
  if (a.value < b.value) return 0;
  return a.key < b.key;
}

typedef struct {
  orc_item *a;
  uint32_t len;
} orc_heap;

static void oh_push(orc_heap *hp, orc_item it) {
  uint32_t c = hp->len++;
  hp->a[c] = it;
  while (c > 0) {
    uint32_t p = (c - 1) / 2;
    if (!ranks_above(hp->a[p], hp->a[c])) break; /* parent already lower */
    orc_item t = hp->a[p];
    hp->a[p] = hp->a[c];
    hp->a[c] = t;
    c = p;
  }
}

static orc_item oh_pop(orc_heap *hp) {
  orc_item top = hp->a[0];
  hp->a[0] = hp->a[--hp->len];
  uint32_t c = 0;
  for (;;) {
    uint32_t l = 2 * c + 1, r = l + 1, s = c;
    if (l < hp->len && ranks_above(hp->a[s], hp->a[l])) s = l;
    if (r < hp->len && ranks_above(hp->a[s], hp->a[r])) s = r;
    if (s == c) break;
    orc_item t = hp->a[s];
    hp->a[s] = hp->a[c];
    hp->a[c] = t;
    c = s;
  }
  return top;
}

static int item_cmp_desc(const void *x, const void *y) {
  orc_item a = *(const orc_item *)x, b = *(const orc_item *)y;
  if (ranks_above(a, b)) return -1;
  if (ranks_above(b, a)) return 1;
  return 0;
}

/* Alg. 3 over items[0..cnt): keeps the k highest-ranked, returned in out
 * sorted from highest to lowest.  Returns min(k, cnt). */
static uint32_t find_largest(const orc_item *items, uint32_t cnt, uint32_t k, orc_item *out) {
  if (k == 0) return 0;
  orc_heap hp;
  hp.a = (orc_item *)malloc(((size_t)k + 1) * sizeof(orc_item));
  hp.len = 0;
  int have_theta = 0;
  orc_item theta = {0, 0};
  for (uint32_t i = 0; i < cnt; ++i) {
    if (have_theta && !ranks_above(items[i], theta)) continue; /* not above theta */
    oh_push(&hp, items[i]);
    if (hp.len > k) {
      theta = oh_pop(&hp);
      have_theta = 1;
    }
  }
  uint32_t r = hp.len;
  memcpy(out, hp.a, r * sizeof(orc_item));
  free(hp.a);
  qsort(out, r, sizeof(orc_item), item_cmp_desc);
  return r;
}

/* <q, x_i> from the vector store, in FP64.  qdense is q scattered over [n]. */
static double exact_dot(const orc_index *ix, const double *qdense, uint32_t id, double *mag) {
  double s = 0.0, a = 0.0;
  for (uint32_t t = 0; t < ix->doc_nnz[id]; ++t) {
    double p = qdense[ix->doc_idx[id][t]] * ix->doc_val[id][t];
    s += p;
    a += fabs(p);
  }
  if (mag) *mag = a;
  return s;
}

typedef struct {
  double *scores; /* n_slots */
  double *mag;
  orc_item *items; /* n_slots */
  orc_item *cand;  /* k' */
  orc_item *top;   /* k */
  double *qdense;  /* n */
  orc_qterm *terms;
  uint32_t terms_cap;
} orc_ws;

static void ws_init(orc_ws *w, const orc_index *ix, uint32_t kp, uint32_t k) {
  size_t ns = ix->n_slots ? ix->n_slots : 1;
  w->scores = (double *)malloc(ns * sizeof(double));
  w->mag = (double *)malloc(ns * sizeof(double));
  w->items = (orc_item *)malloc(ns * sizeof(orc_item));
  w->cand = (orc_item *)malloc(((size_t)kp + 1) * sizeof(orc_item));
  w->top = (orc_item *)malloc(((size_t)k + 1) * sizeof(orc_item));
  w->qdense = (double *)calloc(ix->n, sizeof(double));
  w->terms = NULL;
  w->terms_cap = 0;
}

static void ws_free(orc_ws *w) {
  free(w->scores);
  free(w->mag);
  free(w->items);
  free(w->cand);
  free(w->top);
  free(w->qdense);
  free(w->terms);
}

/* Alg. 6 then Alg. 7 for one query.  Returns the number of results r =
 * min(k, live).  out_ids/out_scores get the top-k by exact score (padding
 * beyond r: id 0xFFFFFFFF, score -inf).  If cand_ids is given it receives the
 * min(k', live) candidates V of Alg. 7 in rank order, with their
 * approximate scores and magnitudes. */
static uint32_t search_one(const orc_index *ix, orc_ws *w, const uint32_t *qi, const float *qv,
                           uint32_t qnnz, uint32_t k, uint32_t kp, uint64_t budget,
                           uint32_t *out_ids, double *out_scores, uint32_t *cand_ids,
                           double *cand_scores, double *cand_mag) {
  if (qnnz > w->terms_cap) {
    w->terms_cap = qnnz;
    w->terms = (orc_qterm *)xrealloc(w->terms, qnnz * sizeof(orc_qterm));
  }
  uint32_t nt = query_terms(qi, qv, qnnz, w->terms);
  alg6_scores(ix, w->terms, anytime_terms(ix, w->terms, nt, budget), w->scores, w->mag);

  /* Alg. 7, candidates: V = FindLargest(scores, k') over the live ids. */
  uint32_t cnt = 0;
  for (uint32_t i = 0; i < ix->n_slots; ++i) {
    if (!ix->live[i]) continue;
    w->items[cnt].value = w->scores[i];
    w->items[cnt].key = i;
    cnt++;
  }
  uint32_t nv = find_largest(w->items, cnt, kp, w->cand);
  if (cand_ids) {
    for (uint32_t t = 0; t < nv; ++t) {
      cand_ids[t] = w->cand[t].key;
      if (cand_scores) cand_scores[t] = w->cand[t].value;
      if (cand_mag) cand_mag[t] = w->mag[w->cand[t].key];
    }
  }

  /* Alg. 7, re-rank: s_v = <q, S.Fetch(v)> exactly. */
  for (uint32_t t = 0; t < nt; ++t) w->qdense[w->terms[t].j] = w->terms[t].v;
  for (uint32_t t = 0; t < nv; ++t) w->cand[t].value = exact_dot(ix, w->qdense, w->cand[t].key, NULL);
  for (uint32_t t = 0; t < nt; ++t) w->qdense[w->terms[t].j] = 0.0;

  /* Alg. 7, result: FindLargest({s_v}, k). */
  uint32_t r = find_largest(w->cand, nv, k, w->top);
  for (uint32_t t = 0; t < k; ++t) {
    out_ids[t] = t < r ? w->top[t].key : 0xFFFFFFFFu;
    out_scores[t] = t < r ? w->top[t].value : -INFINITY;
  }
  return r;
}

/* Exact top-k (Eq. 2) by brute force over every live vector in the store. */
static uint32_t exact_one(const orc_index *ix, orc_ws *w, const uint32_t *qi, const float *qv,
                          uint32_t qnnz, uint32_t k, uint32_t *out_ids, double *out_scores,
                          double *out_mag) {
  for (uint32_t t = 0; t < qnnz; ++t) w->qdense[qi[t]] = (double)qv[t];
  uint32_t cnt = 0;
  for (uint32_t i = 0; i < ix->n_slots; ++i) {
    if (!ix->live[i]) continue;
    w->items[cnt].value = exact_dot(ix, w->qdense, i, &w->mag[i]);
    w->items[cnt].key = i;
    cnt++;
  }
  for (uint32_t t = 0; t < qnnz; ++t) w->qdense[qi[t]] = 0.0;
  uint32_t r = find_largest(w->items, cnt, k, w->top);
  for (uint32_t t = 0; t < k; ++t) {
    out_ids[t] = t < r ? w->top[t].key : 0xFFFFFFFFu;
    out_scores[t] = t < r ? w->top[t].value : -INFINITY;
    if (out_mag) out_mag[t] = t < r ? w->mag[w->top[t].key] : 0.0;
  }
  return r;
}

/* -------------------------------------------------- batched entry points */

typedef struct {
  const orc_index *ix;
  const uint64_t *indptr;
  const uint32_t *indices;
  const float *values;
  uint32_t q0, q1, k, kp, mode;
  uint64_t budget;
  uint32_t *out_ids;
  double *out_scores;
  uint32_t *cand_ids;
  double *cand_scores;
  double *cand_mag;
  double *out_mag;
  uint32_t *out_count;
} orc_job;

static void *run_job(void *arg) {
  orc_job *jb = (orc_job *)arg;
  orc_ws w;
  ws_init(&w, jb->ix, jb->kp, jb->k);
  for (uint32_t q = jb->q0; q < jb->q1; ++q) {
    const uint32_t *qi = jb->indices + jb->indptr[q];
    const float *qv = jb->values + jb->indptr[q];
    uint32_t qn = (uint32_t)(jb->indptr[q + 1] - jb->indptr[q]);
    uint32_t r;
    if (jb->mode == 0) {
      r = search_one(jb->ix, &w, qi, qv, qn, jb->k, jb->kp, jb->budget,
                     jb->out_ids + (size_t)q * jb->k,
                     jb->out_scores + (size_t)q * jb->k,
                     jb->cand_ids ? jb->cand_ids + (size_t)q * jb->kp : NULL,
                     jb->cand_scores ? jb->cand_scores + (size_t)q * jb->kp : NULL,
                     jb->cand_mag ? jb->cand_mag + (size_t)q * jb->kp : NULL);
    } else {
      r = exact_one(jb->ix, &w, qi, qv, qn, jb->k, jb->out_ids + (size_t)q * jb->k,
                    jb->out_scores + (size_t)q * jb->k,
                    jb->out_mag ? jb->out_mag + (size_t)q * jb->k : NULL);
    }
    if (jb->out_count) jb->out_count[q] = r;
  }
  ws_free(&w);
  return NULL;
}

static int run_batch(orc_job proto, uint32_t n_q, uint32_t n_threads) {
  for (uint32_t q = 0; q < n_q; ++q) {
    uint64_t ip[2] = {0, proto.indptr[q + 1] - proto.indptr[q]};
    if (proto.indptr[q + 1] < proto.indptr[q]) return ORC_EINVAL;
    if (validate_csr(proto.ix->n, ip, proto.indices + proto.indptr[q],
                     proto.values + proto.indptr[q], 1))
      return ORC_EINVAL;
  }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_q) n_threads = n_q ? n_q : 1;
  pthread_t *th = (pthread_t *)malloc(n_threads * sizeof(pthread_t));
  orc_job *jobs = (orc_job *)malloc(n_threads * sizeof(orc_job));
  for (uint32_t t = 0; t < n_threads; ++t) {
    jobs[t] = proto;
    jobs[t].q0 = (uint32_t)((uint64_t)n_q * t / n_threads);
    jobs[t].q1 = (uint32_t)((uint64_t)n_q * (t + 1) / n_threads);
  }
  if (n_threads == 1) {
    run_job(&jobs[0]);
  } else {
    for (uint32_t t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    for (uint32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  free(th);
  free(jobs);
  return ORC_OK;
}

/* SINNAMON retrieval (Alg. 6 with the anytime budget, then Alg. 7) for a
 * CSR batch of queries; budget 0 means T = infinity. */
int orc_search_anytime(const orc_index *ix, const uint64_t *indptr, const uint32_t *indices,
                       const float *values, uint32_t n_q, uint32_t k, uint32_t kp,
                       uint64_t budget, uint32_t *out_ids, double *out_scores,
                       uint32_t *cand_ids, double *cand_scores, double *cand_mag,
                       uint32_t *out_count, uint32_t n_threads) {
  if (k == 0 || kp < k) return ORC_EINVAL;
  orc_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.budget = budget;
  jb.ix = ix;
  jb.indptr = indptr;
  jb.indices = indices;
  jb.values = values;
  jb.k = k;
  jb.kp = kp;
  jb.mode = 0;
  jb.out_ids = out_ids;
  jb.out_scores = out_scores;
  jb.cand_ids = cand_ids;
  jb.cand_scores = cand_scores;
  jb.cand_mag = cand_mag;
  jb.out_count = out_count;
  return run_batch(jb, n_q, n_threads);
}

/* SINNAMON retrieval (Alg. 6 + Alg. 7), T = infinity. */
int orc_search(const orc_index *ix, const uint64_t *indptr, const uint32_t *indices,
               const float *values, uint32_t n_q, uint32_t k, uint32_t kp, uint32_t *out_ids,
               double *out_scores, uint32_t *cand_ids, double *cand_scores, double *cand_mag,
               uint32_t *out_count, uint32_t n_threads) {
  return orc_search_anytime(ix, indptr, indices, values, n_q, k, kp, 0, out_ids, out_scores,
                            cand_ids, cand_scores, cand_mag, out_count, n_threads);
}

/* Exact MIPS (Eq. 2) by brute force, for a CSR batch of queries. */
int orc_exact_topk(const orc_index *ix, const uint64_t *indptr, const uint32_t *indices,
                   const float *values, uint32_t n_q, uint32_t k, uint32_t *out_ids,
                   double *out_scores, double *out_mag, uint32_t *out_count, uint32_t n_threads) {
  if (k == 0) return ORC_EINVAL;
  orc_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.ix = ix;
  jb.indptr = indptr;
  jb.indices = indices;
  jb.values = values;
  jb.k = k;
  jb.kp = k;
  jb.mode = 1;
  jb.out_ids = out_ids;
  jb.out_scores = out_scores;
  jb.out_mag = out_mag;
  jb.out_count = out_count;
  return run_batch(jb, n_q, n_threads);
}

/* Dense exact scores <q, x_i> for every slot (0 for vacant slots); if mag is
 * given it receives sum_j |q_j * x_i[j]| per slot. */
int orc_exact_scores(const orc_index *ix, const uint32_t *qi, const float *qv, uint32_t qnnz,
                     double *scores, double *mag) {
  if (validate_query(ix, qi, qv, qnnz)) return ORC_EINVAL;
  double *qd = (double *)calloc(ix->n, sizeof(double));
  for (uint32_t t = 0; t < qnnz; ++t) qd[qi[t]] = (double)qv[t];
  for (uint32_t i = 0; i < ix->n_slots; ++i) {
    double a = 0.0;
    scores[i] = ix->live[i] ? exact_dot(ix, qd, i, &a) : 0.0;
    if (mag) mag[i] = a;
  }
  free(qd);
  return ORC_OK;
}

/* FindLargest (Alg. 3) exposed on its own: top-k of (values[i], i), i < cnt. */
uint32_t orc_find_largest(const double *values, uint32_t cnt, uint32_t k, uint32_t *out_keys,
                          double *out_values) {
  orc_item *items = (orc_item *)malloc((cnt ? cnt : 1) * sizeof(orc_item));
  orc_item *out = (orc_item *)malloc(((size_t)k + 1) * sizeof(orc_item));
  for (uint32_t i = 0; i < cnt; ++i) {
    items[i].value = values[i];
    items[i].key = i;
  }
  uint32_t r = find_largest(items, cnt, k, out);
  for (uint32_t t = 0; t < r; ++t) {
    out_keys[t] = out[t].key;
    out_values[t] = out[t].value;
  }
  free(items);
  free(out);
  return r;
}

/* ------------------------------------------------------------- LinScan */
/* Alg. 1 (indexing) builds, per coordinate, parallel arrays of ids and values;
 * Alg. 2 (retrieval) accumulates exact scores coordinate at a time and ends
 * with FindLargest.  Built from the live vectors of a SINNAMON oracle index so
 * both indexes hold the same collection. */
typedef struct orc_linscan {
  uint32_t n, n_slots;
  uint32_t **ids;
  double **vals;
  uint32_t *len;
  uint8_t *live;
} orc_linscan;

orc_linscan *orc_linscan_build(const orc_index *ix) {
  orc_linscan *ls = (orc_linscan *)calloc(1, sizeof(orc_linscan));
  ls->n = ix->n;
  ls->n_slots = ix->n_slots;
  ls->ids = (uint32_t **)calloc(ix->n, sizeof(uint32_t *));
  ls->vals = (double **)calloc(ix->n, sizeof(double *));
  ls->len = (uint32_t *)calloc(ix->n, sizeof(uint32_t));
  ls->live = (uint8_t *)malloc(ix->n_slots ? ix->n_slots : 1);
  memcpy(ls->live, ix->live, ix->n_slots);
  for (uint32_t i = 0; i < ix->n_slots; ++i)
    if (ix->live[i])
      for (uint32_t t = 0; t < ix->doc_nnz[i]; ++t) ls->len[ix->doc_idx[i][t]]++;
  for (uint32_t j = 0; j < ix->n; ++j) {
    ls->ids[j] = (uint32_t *)malloc((ls->len[j] ? ls->len[j] : 1) * sizeof(uint32_t));
    ls->vals[j] = (double *)malloc((ls->len[j] ? ls->len[j] : 1) * sizeof(double));
    ls->len[j] = 0;
  }
  for (uint32_t i = 0; i < ix->n_slots; ++i) { /* ascending i: Alg. 1 per vector */
    if (!ix->live[i]) continue;
    for (uint32_t t = 0; t < ix->doc_nnz[i]; ++t) {
      uint32_t j = ix->doc_idx[i][t];
      ls->ids[j][ls->len[j]] = i;
      ls->vals[j][ls->len[j]] = ix->doc_val[i][t];
      ls->len[j]++;
    }
  }
  return ls;
}

void orc_linscan_destroy(orc_linscan *ls) {
  if (!ls) return;
  for (uint32_t j = 0; j < ls->n; ++j) {
    free(ls->ids[j]);
    free(ls->vals[j]);
  }
  free(ls->ids);
  free(ls->vals);
  free(ls->len);
  free(ls->live);
  free(ls);
}

typedef struct {
  const orc_linscan *ls;
  const uint64_t *indptr;
  const uint32_t *indices;
  const float *values;
  uint32_t q0, q1, k;
  uint32_t *out_ids;
  double *out_scores;
} orc_lsjob;

static void *run_lsjob(void *arg) {
  orc_lsjob *jb = (orc_lsjob *)arg;
  const orc_linscan *ls = jb->ls;
  size_t ns = ls->n_slots ? ls->n_slots : 1;
  double *scores = (double *)malloc(ns * sizeof(double));
  orc_item *items = (orc_item *)malloc(ns * sizeof(orc_item));
  orc_item *top = (orc_item *)malloc(((size_t)jb->k + 1) * sizeof(orc_item));
  for (uint32_t q = jb->q0; q < jb->q1; ++q) {
    memset(scores, 0, ns * sizeof(double)); /* Alg. 2: scores start at zero */
    for (uint64_t p = jb->indptr[q]; p < jb->indptr[q + 1]; ++p) {
      uint32_t j = jb->indices[p];
      double qj = (double)jb->values[p];
      if (qj == 0.0) continue;
      for (uint32_t t = 0; t < ls->len[j]; ++t) scores[ls->ids[j][t]] += ls->vals[j][t] * qj;
    }
    uint32_t cnt = 0;
    for (uint32_t i = 0; i < ls->n_slots; ++i) {
      if (!ls->live[i]) continue;
      items[cnt].value = scores[i];
      items[cnt].key = i;
      cnt++;
    }
    uint32_t r = find_largest(items, cnt, jb->k, top);
    for (uint32_t t = 0; t < jb->k; ++t) {
      jb->out_ids[(size_t)q * jb->k + t] = t < r ? top[t].key : 0xFFFFFFFFu;
      jb->out_scores[(size_t)q * jb->k + t] = t < r ? top[t].value : -INFINITY;
    }
  }
  free(scores);
  free(items);
  free(top);
  return NULL;
}

int orc_linscan_topk(const orc_linscan *ls, const uint64_t *indptr, const uint32_t *indices,
                     const float *values, uint32_t n_q, uint32_t k, uint32_t *out_ids,
                     double *out_scores, uint32_t n_threads) {
  if (k == 0) return ORC_EINVAL;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_q) n_threads = n_q ? n_q : 1;
  pthread_t *th = (pthread_t *)malloc(n_threads * sizeof(pthread_t));
  orc_lsjob *jobs = (orc_lsjob *)malloc(n_threads * sizeof(orc_lsjob));
  for (uint32_t t = 0; t < n_threads; ++t) {
    orc_lsjob j = {ls, indptr, indices, values, 0, 0, k, out_ids, out_scores};
    j.q0 = (uint32_t)((uint64_t)n_q * t / n_threads);
    j.q1 = (uint32_t)((uint64_t)n_q * (t + 1) / n_threads);
    jobs[t] = j;
  }
  if (n_threads == 1) {
    run_lsjob(&jobs[0]);
  } else {
    for (uint32_t t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, run_lsjob, &jobs[t]);
    for (uint32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  free(th);
  free(jobs);
  return ORC_OK;
}
