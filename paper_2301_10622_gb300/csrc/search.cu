// Retrieval on the GPU: Alg. 6 (scoring) and Alg. 7 (ranking) of SINNAMON.
//
// One search launch handles a batch of B queries:
//   k_qprep      nz(q), sorted by |q_j| descending, ties by j (Alg. 6)
//   k_score_emit grid (query, group of tiles), queries fastest so the blocks
//                resident at any time share the tiles' lists and sketch rows
//                in L2: walks the query's lists inside each tile of T ids,
//                decodes each posting from the sketch (least upper bound from
//                U for q_j > 0, greatest lower bound from L for q_j < 0,
//                Alg. 6) and accumulates q_j * x~ in shared memory.  Score
//                keys at or above the query's running bound are counted in its
//                4096-bin histogram (top 12 bits) and emitted as candidates;
//                every few tiles a block turns the histogram into a new lower
//                bound on the k'-th best score (at least k' scores already seen
//                are at or above it).
//   k_pick_list/k_compact_list/k_refine
//                FindLargest(scores, k') of Alg. 7 as a radix select:
//                the complete histogram gives the bin holding the k'-th best;
//                emitted keys above it are in, the rest of that bin is picked
//                by (score, -id).
//   fallback     a query whose emitted list overflows, or whose boundary bin
//                is huge (massive ties), is rescored densely (one key per id)
//                and selected with finer histogram levels (k_hist_level) or,
//                for exact ties beyond the buffer, by id order.
//   k_rerank     s_v = <q, S.Fetch(v)> for every candidate (Alg. 7)
//   k_final      FindLargest({s_v}, k) (Alg. 7), sorted best first
// Ties rank the smaller id first: keys carry ~id in their low 32 bits.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "sinn_internal.cuh"

#define CK(x)                                          \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) return sinn_check_cuda(e_); \
  } while (0)

namespace {

constexpr uint32_t kBoundCap = 65536;   // boundary-bin entries kept per query
constexpr uint32_t kEmitCap = 131072;   // emitted candidates kept per query
constexpr uint32_t kScoreThreads = 512;
constexpr uint32_t kChunk = 2048;       // keys per block in the dense select passes
constexpr uint32_t kTermBatch = 64;     // query terms staged in shared memory at a time
constexpr uint32_t kBmGroups = 2;       // 4-id groups per thread a bitmap term pass holds
constexpr uint32_t kFbBlocks = 1024;    // blocks of the fallback kernels
constexpr uint32_t kTouchCap = 2048;    // ids a touched-list tile may list
constexpr uint32_t kZeroBin = 0x800u;   // key bin (top 12 bits) of a zero score
constexpr uint32_t kFuseQueries = 4;    // launches of at most this many queries fuse steps

enum SelMode : uint32_t { SEL_DONE = 0, SEL_L1 = 1, SEL_L2 = 2, SEL_COMPACT = 3, SEL_TIES = 4 };

struct SelState {
  uint32_t mode;    // SelMode
  uint32_t prefix;  // top pbits of the boundary key
  uint32_t pbits;
  uint32_t rem;     // keys still to take from the boundary bin
  uint32_t cnt;     // keys in the boundary bin
  uint32_t kq;      // candidates wanted: min(k', live)
  uint32_t ncand;   // candidates collected so far
  uint32_t nbnd;    // boundary keys collected
  uint32_t dense;   // 1: selected from dense keys (fallback), 0: from the emitted list
  uint32_t pad[3];
};

struct QTerm {
  uint32_t j;
  float v;
};

struct Batch {  // device scratch views of one launch
  QTerm *terms;     // B x qmax
  uint32_t *nt;     // B: query terms (the re-rank uses them all)
  uint32_t *ns;     // B: terms scored (fewer under an anytime budget)
  uint32_t *keys;   // B x cap
  uint32_t *hist0;  // B x 4096
  uint32_t *hist1;  // B x 4096
  uint32_t *hist2;  // B x 256
  SelState *sel;    // B
  uint64_t *cand;   // B x kpmax
  uint64_t *bnd;    // B x kBoundCap
  uint64_t *ekeys;  // B x kpmax
  uint64_t *elist;  // B x kEmitCap: emitted (key << 32 | ~id)
  uint32_t *ecnt;   // B: emitted count (may exceed kEmitCap: overflow)
  uint32_t *bound;  // B: lower-bound bin of the k'-th best key
  uint32_t *tdone;  // B: tiles finished
  uint32_t *rdone;  // B: re-rank blocks finished
  uint32_t *flagged;  // B: queries taking the dense fallback
  uint32_t *nflag;    // 1
  uint32_t *tick;     // 4: blocks finished of the kernels that end in a pick or refine
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  return (1u << (threadIdx.x & 31)) - 1u;
}

// Warp-aggregated append: returns the slot for lanes with pred set.
__device__ __forceinline__ uint32_t warp_append(bool pred, uint32_t *counter) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, pred);
  if (!m) return 0;
  const uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((threadIdx.x & 31) == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  return base + __popc(m & lanemask_lt());
}

// True in every thread of the block that is the last of `total` blocks to
// count on *ctr (zeroed by the query prep); every block fences its writes
// before counting, and the last one fences after, so it sees them all.
// Reads of data other blocks wrote in the same launch go through L2
// (__ldcg): this SM's L1 may hold older copies.
__device__ bool last_block(uint32_t *ctr, uint32_t total) {
  __shared__ uint32_t s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) + 1u == total ? 1u : 0u;
  __syncthreads();
  const bool last = s_last != 0u;
  if (last) __threadfence();
  return last;
}

// --------------------------------------------------------------- query prep
__global__ void k_qprep(const uint64_t *__restrict__ q_indptr, const uint32_t *__restrict__ q_idx,
                        const float *__restrict__ q_val, uint32_t q0, uint32_t n, uint32_t qmax,
                        uint32_t kp_scalar, const uint32_t *__restrict__ kp_arr, uint32_t kp_min,
                        uint32_t kp_max, const uint64_t *live_count, Batch bt,
                        const uint32_t *__restrict__ coord_len, uint64_t budget,
                        const uint64_t *__restrict__ budget_arr, int nonneg, int dense_all,
                        uint32_t *err) {
  extern __shared__ uint32_t sq[];
  uint32_t *sj = sq;                  // qmax
  float *sv = (float *)(sq + qmax);   // qmax
  __shared__ uint32_t s_cnt, s_bad;
  const uint32_t b = blockIdx.x, q = q0 + b;
  // the slot's selection state starts empty: histograms, emitted count,
  // running bound, tiles done; block 0 also resets the launch's counters
  // (flagged queries, the persistent kernel's work counter)
  {
    uint4 *h0 = (uint4 *)(bt.hist0 + (uint64_t)b * 4096), *h1 = (uint4 *)(bt.hist1 + (uint64_t)b * 4096);
    uint4 *h2 = (uint4 *)(bt.hist2 + (uint64_t)b * 256);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) {
      h0[i] = z;
      h1[i] = z;
    }
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) h2[i] = z;
  }
  if (threadIdx.x == 0) {
    bt.ecnt[b] = 0u;
    bt.bound[b] = 0u;
    bt.tdone[b] = 0u;
    bt.rdone[b] = 0u;
    if (dense_all) bt.flagged[b] = b;  // every query of the launch scores densely
    if (b == 0) {
      *bt.nflag = dense_all ? gridDim.x : 0u;
      *(unsigned long long *)(((uintptr_t)(bt.nflag + 1) + 7) & ~(uintptr_t)7) = 0ull;
      for (uint32_t i = 0; i < 4; ++i) bt.tick[i] = 0u;
    }
  }
  const uint64_t s = q_indptr[q], e = q_indptr[q + 1];
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_bad = (e < s || e - s > qmax) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_bad) {
    for (uint64_t p = s + threadIdx.x; p < e; p += blockDim.x) {
      uint32_t c = q_idx[p];
      float v = q_val[p];
      bool bad = c >= n || !isfinite(v) || (p > s && q_idx[p - 1] >= c) || (nonneg && v < 0.0f);
      if (bad) atomicOr(&s_bad, 1u);
      if (v != 0.0f && !bad) {
        uint32_t slot = atomicAdd(&s_cnt, 1u);
        sj[slot] = c;
        sv[slot] = v;
      }
    }
  }
  __syncthreads();
  const uint32_t cnt = s_bad ? 0u : s_cnt;
  QTerm *out = bt.terms + (uint64_t)b * qmax;
  // Alg. 6: terms ranked by |q_j| descending, ties by j ascending
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const float ai = fabsf(sv[i]);
    const uint32_t ji = sj[i];
    uint32_t r = 0;
    for (uint32_t t = 0; t < cnt; ++t) {
      float at = fabsf(sv[t]);
      r += (at > ai) || (at == ai && sj[t] < ji);
    }
    out[r].j = ji;
    out[r].v = sv[i];
  }
  if (budget || budget_arr) __syncthreads();  // thread 0 reads the sorted terms
  if (threadIdx.x == 0) {
    // Alg. 6's anytime break, the budget counted in postings (the index's, or
    // this query's own when per-query budgets are given): score the terms up
    // to the first one at which the postings visited reach the budget (the
    // re-rank still takes every term: Alg. 7's exact inner product)
    if (budget_arr) budget = budget_arr[q];
    uint32_t scored = cnt;
    if (budget) {
      uint64_t visited = 0;
      scored = 0;
      while (scored < cnt) {
        visited += coord_len[out[scored].j];
        ++scored;
        if (visited >= budget) break;
      }
    }
    if (s_bad) atomicOr(err, SINN_DERR_QUERY);
    bt.nt[b] = cnt;
    bt.ns[b] = scored;
    uint32_t kp = kp_arr ? min(max(kp_arr[q], kp_min), kp_max) : kp_scalar;
    SelState st;
    st.mode = SEL_DONE;
    st.prefix = 0;
    st.pbits = 0;
    st.rem = 0;
    st.cnt = 0;
    const uint64_t lc = *live_count;
    st.kq = s_bad ? 0u : (uint32_t)(lc < kp ? lc : (uint64_t)kp);
    st.ncand = 0;
    st.nbnd = 0;
    st.dense = dense_all ? 1u : 0u;
    bt.sel[b] = st;
  }
}

// ------------------------------------------------------------------ scoring
// Alg. 6 for one (tile, query) pair.  The block first stages the query terms
// that have postings in this tile, then walks the flattened (term, posting)
// space so every thread stays busy whatever the list lengths.
struct ScoreArgs {
  const uint2 *tile_dir;        // copy v of tile t at (2t + v) n
  uint16_t *const *tile_post;   // storage of copy v of tile t at 2t + v
  const uint32_t *sel;          // per tile: the copy to read
  const uint32_t *recent;       // ids whose visibility depends on the snapshot
  const uint32_t *born, *died;  // their birth and death sequence numbers
  uint32_t seq;                 // the search's snapshot
  const void *U;  // sketch planes: fp32 or bfloat16 bits (S below)
  const void *L;
  const uint32_t *pi;
  const uint32_t *live;
  uint64_t cap;
  uint32_t n, h, T, log2T, qmax, tiles;
  uint32_t bound_every;  // tiles between refreshes of the running bound
  uint32_t tpb;          // tiles per block of the batched kernel
  uint32_t *err;         // sticky device error bits (bounds-check builds)
  uint32_t m;            // sketch rows per plane (bounds-check builds)
};

// Lower-bound bin of the kq-th largest key from a (partial) histogram: the
// highest bin b with sum_{i >= b} hist[i] >= kq, or 0 if the counts fall short.
// Counts only grow, so a stale read gives a lower (still valid) bound.  Only
// bins at or above lb (the bound already known) are read: a new bound below
// it would not raise it.
__device__ uint32_t bound_from_hist(const uint32_t *gh, uint32_t kq, uint32_t lb,
                                   uint32_t *part) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr uint32_t per = 4096 / kScoreThreads;  // thread tid owns the tid-th group from the top
  const uint32_t top = 4096 - tid * per;
  uint32_t c[per], s = 0;
#pragma unroll
  for (uint32_t i = 0; i < per; ++i) {
    c[i] = top - 1 - i >= lb ? __ldcg(gh + top - 1 - i) : 0u;
    s += c[i];
  }
  uint32_t x = s;  // inclusive scan over threads (top groups first)
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) part[wid] = x;
  __syncthreads();
  if (tid == 0) {
    uint32_t r = 0;
    for (uint32_t w = 0; w < kScoreThreads / 32; ++w) {
      uint32_t v = part[w];
      part[w] = r;
      r += v;
    }
    part[kScoreThreads / 32] = 0;  // result slot
  }
  __syncthreads();
  const uint32_t before = part[wid] + x - s;
  if (before < kq && before + s >= kq) {
    uint32_t run = before, bin = top - 1;
#pragma unroll
    for (uint32_t i = 0; i < per; ++i) {
      if (run + c[i] >= kq) {
        bin = top - 1 - i;
        break;
      }
      run += c[i];
    }
    part[kScoreThreads / 32] = bin;
  }
  __syncthreads();
  const uint32_t r = part[kScoreThreads / 32];
  __syncthreads();
  return r;
}

// Decoded value x~ of one posting (Alg. 6): the least upper bound
// over the term's h rows of U (q_j > 0) or the greatest lower bound over its
// rows of L (q_j < 0).  row[o] already points at the tile's slice of the row.
__device__ __forceinline__ float sk_load(const float *p) { return __ldg(p); }
__device__ __forceinline__ float sk_load(const uint16_t *p) { return sinn_bf16_f(__ldg(p)); }
__device__ __forceinline__ float4 sk_load4(const float *p) { return __ldg((const float4 *)p); }
__device__ __forceinline__ float4 sk_load4(const uint16_t *p) {
  const uint2 v = __ldg((const uint2 *)p);  // 4 bins, 8-byte aligned
  return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xFFFF0000u),
                     __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xFFFF0000u));
}

template <int H, typename S>
__device__ __forceinline__ float decode(const S *const *row, uint32_t h, bool pos, uint32_t d) {
  float y = sk_load(row[0] + d);
  const uint32_t hh = H > 0 ? (uint32_t)H : h;
#pragma unroll
  for (uint32_t o = 1; o < (H > 0 ? (uint32_t)H : (uint32_t)SINN_MAX_H); ++o) {
    if (o >= hh) break;
    const float z = sk_load(row[o] + d);
    y = pos ? fminf(y, z) : fmaxf(y, z);
  }
  return y;
}

// Sketch values of 4 consecutive ids (16-byte aligned: rows start on tile
// boundaries): least upper bound over the rows for q_j > 0, greatest lower
// bound for q_j < 0 (Alg. 6).
template <int H, typename S>
__device__ __forceinline__ float4 decode4(const S *const *row, uint32_t h, bool pos,
                                          uint32_t d0) {
  float4 y = sk_load4(row[0] + d0);
  const uint32_t hh = H > 0 ? (uint32_t)H : h;
#pragma unroll
  for (uint32_t o = 1; o < (H > 0 ? (uint32_t)H : (uint32_t)SINN_MAX_H); ++o) {
    if (o >= hh) break;
    const float4 z = sk_load4(row[o] + d0);
    if (pos) {
      y.x = fminf(y.x, z.x); y.y = fminf(y.y, z.y); y.z = fminf(y.z, z.z); y.w = fminf(y.w, z.w);
    } else {
      y.x = fmaxf(y.x, z.x); y.y = fmaxf(y.y, z.y); y.z = fmaxf(y.z, z.z); y.w = fmaxf(y.w, z.w);
    }
  }
  return y;
}

// One warp: start the copies of the directory entries {start, count} of the
// first nt query terms (coordinates tj, in shared memory) in tile t into dst
// (8 bytes each, cp.async), from the tile's current copy, whose number goes
// to *ver.
__device__ __forceinline__ void dir_fetch(const ScoreArgs &a, const uint32_t *tj, uint32_t nt,
                                          uint32_t t, uint2 *dst, uint32_t *ver, uint32_t lane) {
  // one load for the warp: every lane reads the same copy of the tile
  const uint32_t v = __ldcg(a.sel + t);
  if (lane == 0) *ver = v;
  const uint2 *dir = a.tile_dir + ((uint64_t)t * 2 + v) * a.n;
  for (uint32_t k = lane; k < nt; k += 32) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(dst + k);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(dir + tj[k])
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// The recent bits of this thread's 4 ids (id a multiple of 4; the warp's
// lanes cover consecutive ids, 8 lanes per 32-bit word) among the live ones
// in lwv, read by one lane per word once a live bit was seen; 0 when the
// index keeps no snapshot words.  Every lane of the warp takes part.
__device__ __forceinline__ uint32_t recent_bits4(const ScoreArgs &a, uint64_t id, uint32_t lwv,
                                                 uint32_t lane) {
  if (!a.recent || !__any_sync(0xFFFFFFFFu, lwv != 0u)) return 0u;
  uint32_t w = 0u;
  if ((lane & 7u) == 0u) w = sinn_ld_gpu(a.recent + (id >> 5));
  w = __shfl_sync(0xFFFFFFFFu, w, lane & ~7u);
  return (w >> (id & 31)) & lwv;
}

// Live ids of this thread's 4 (bits of lwv) that the search's snapshot counts.
__device__ __forceinline__ uint32_t visible4(const ScoreArgs &a, uint64_t id, uint32_t lwv,
                                             uint32_t lane) {
  const uint32_t rwv = recent_bits4(a, id, lwv, lane);
  if (rwv)
    for (uint32_t q = 0; q < 4; ++q)
      if (((rwv >> q) & 1u) && !sinn_visible_recent(a.born, a.died, a.seq, id + q))
        lwv &= ~(1u << q);
  return lwv;
}

// Alg. 6 for query slot b over tiles [t_beg, t_end).  A query term's postings
// inside a tile sit in one container: a bitmap of T bits when at least an
// eighth of the tile's ids hold the coordinate, else a sorted array of 16-bit
// local ids.  The query's coordinates, weights and sketch bins are staged
// once for all the block's tiles (queries of at most kTermBatch terms; longer
// ones restage each batch of terms per tile).  Per tile, for each batch:
//   Staging (warp 0): the terms' directory entries (fetched a tile ahead with
//   cp.async when the query has a single batch), the prefix of the array
//   terms' chunk counts and the list of bitmap terms.
//   Bitmap terms: thread t owns the 4 consecutive ids 4t..4t+3 of each
//   2048-id slice, holds their partial scores in registers and, per term,
//   reads one bitmap word and one 16-byte group of sketch values; no atomics.
//   The sums go to a second accumulator only the owner touches, so no
//   barrier separates them from the array terms.
//   Array terms: their postings are cut into chunks of 32 (one per lane),
//   numbered in term order; each warp takes a contiguous range of chunks (so
//   it finds a chunk's term by advancing one pointer) and adds q_j * x~ into
//   shared memory with atomics (two terms may share an id).
// The epilogue adds the two accumulators and leaves them zero for the next
// tile: ids whose score key reaches the query's running bound are counted in
// the histogram and emitted as candidates.  Counted keys go straight to the
// query's global histogram; the bound is refreshed from it once per block.
// Touched-list tiles: when a tile holds only array containers of the query
// and the running bound is above the bin of a zero score, an id no posting
// reached scores 0 and cannot be a candidate.  Each array posting then also
// marks its id in a T-bit bitmap, the first mark appending the id to a list,
// and the epilogue visits the listed ids only (instead of all T).
template <int H, typename S, bool WALK>
__device__ void score_tiles(const ScoreArgs &a, const Batch &bt, uint32_t b, uint32_t t_beg,
                            uint32_t t_end, uint32_t *sm) {
  constexpr uint32_t NW = kScoreThreads / 32;
  constexpr uint32_t HS = H > 0 ? (uint32_t)H : (uint32_t)SINN_MAX_H;
  const uint32_t T = a.T, BMIN = T >> SINN_BITMAP_SHIFT;
  float *acc = (float *)sm;                          // T: array terms (atomics)
  float *bacc = acc + T;                             // T: bitmap terms (owner only)
  uint32_t *touched = sm + 2 * T;                    // T/32: ids an array posting reached
  uint16_t *tlist = (uint16_t *)(touched + T / 32);  // kTouchCap: those ids, first touch order
  uint32_t *t_start = (uint32_t *)(tlist + kTouchCap);  // kTermBatch
  uint32_t *t_cnt = t_start + kTermBatch;            // kTermBatch
  uint32_t *t_cp = t_cnt + kTermBatch;               // kTermBatch+1: chunk prefix (arrays)
  float *t_v = (float *)(t_cp + kTermBatch + 1);     // kTermBatch
  uint32_t *t_j = (uint32_t *)(t_v + kTermBatch);    // kTermBatch: coordinates
  uint32_t *t_bin = t_j + kTermBatch;                // kTermBatch * h
  __shared__ uint32_t part[NW + 2];
  __shared__ uint32_t s_nbm, s_lb, s_ntl, s_apost, s_dirty;
  __shared__ uint8_t t_bl[kTermBatch];  // bitmap terms of the batch, in order
  // directory entries of the query's terms for this tile and the next one
  // (queries of at most kTermBatch terms: fetched a tile ahead by cp.async)
  __shared__ uint2 s_dir[2][kTermBatch];
  __shared__ uint32_t s_ver[2], s_vt;  // copies of the prefetched entries; of this tile

  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t nt = bt.ns[b];  // Alg. 6 scores the budget's prefix
  const QTerm *terms = bt.terms + (uint64_t)b * a.qmax;
  // the query's histogram of key bins, counted in place with L2 atomics:
  // past the first tiles only the keys at or above the running bound are
  // counted, too few to need a per-block copy (whose shared memory is worth
  // more as L1 for the sketch gathers)
  uint32_t *gh = bt.hist0 + (uint64_t)b * 4096;
  uint64_t *el = bt.elist + (uint64_t)b * kEmitCap;
  const uint32_t nbatch = nt == 0 ? 1 : (nt + kTermBatch - 1) / kTermBatch;

  // the block starts with zero accumulators and no marks; every epilogue
  // leaves them so
  for (uint32_t d = 4 * tid; d < T; d += 4 * kScoreThreads) {
    *(float4 *)(acc + d) = make_float4(0.f, 0.f, 0.f, 0.f);
    *(float4 *)(bacc + d) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (uint32_t w = tid; w < T / 32; w += kScoreThreads) touched[w] = 0u;
  if (tid == 0) s_lb = __ldcg(&bt.bound[b]);
  if (nbatch == 1 && wid == 0) {
    // the query's coordinates, weights and bins, the same for every tile
    for (uint32_t k = lane; k < nt; k += 32) {
      const uint32_t j = terms[k].j;
      t_j[k] = j;
      t_v[k] = terms[k].v;
      for (uint32_t o = 0; o < a.h; ++o) {
        const uint32_t bin = a.pi[(uint64_t)j * a.h + o];
        t_bin[k * a.h + o] = SINN_IN_BOUNDS(bin < a.m, a.err) ? bin : 0u;
      }
    }
    __syncwarp();
    if (t_beg < t_end) dir_fetch(a, t_j, nt, t_beg, s_dir[0], &s_ver[0], lane);
  }
  __syncthreads();
  // keys below the bound are neither counted nor emitted
  const uint32_t lb = s_lb;
  for (uint32_t t = t_beg; t < t_end; ++t) {
    const uint64_t id0 = (uint64_t)t << a.log2T;
    __syncthreads();  // the previous tile's epilogue is done with acc, bacc and the list
    bool touch = false;
    for (uint32_t bi = 0; bi < nbatch; ++bi) {
      const uint32_t i0 = bi * kTermBatch;
      const uint32_t nb = nt > i0 ? min(kTermBatch, nt - i0) : 0u;
      if (bi > 0) __syncthreads();  // the previous batch is consumed
      if (wid == 0) {
        // the batch's directory entries, then the exclusive prefix of the
        // array chunk counts and the list of bitmap terms
        const uint32_t pb = (t - t_beg) & 1u;
        if (nbatch == 1) {
          asm volatile("cp.async.wait_all;\n" ::: "memory");  // this tile's entries
          __syncwarp();
        }
        // the tile's copy: the one its entries were prefetched from, or (terms
        // restaged per batch) the current one, read once for all batches
        const uint32_t vt = nbatch == 1 ? s_ver[pb] : (bi == 0 ? __ldcg(a.sel + t) : s_vt);
        const uint2 *dir = a.tile_dir + ((uint64_t)t * 2 + vt) * a.n;
        __syncwarp();
        if (lane == 0) s_vt = vt;
        for (uint32_t k = lane; k < nb; k += 32) {
          uint2 de;
          if (nbatch == 1) {
            de = s_dir[pb][k];
          } else {
            const uint32_t j = terms[i0 + k].j;
            de = dir[j];
            t_v[k] = terms[i0 + k].v;
            for (uint32_t o = 0; o < a.h; ++o) {
              const uint32_t bin = a.pi[(uint64_t)j * a.h + o];
              t_bin[k * a.h + o] = SINN_IN_BOUNDS(bin < a.m, a.err) ? bin : 0u;
            }
          }
          t_start[k] = de.x;
          t_cnt[k] = de.y;
          // array terms' chunks of 32 postings (walk 0) or postings (walk 1)
          t_cp[k] = de.y >= BMIN ? 0u : (WALK ? de.y : (de.y + 31) >> 5);
        }
        // the next tile's entries arrive while this tile is scored
        if (nbatch == 1 && t + 1 < t_end)
          dir_fetch(a, t_j, nb, t + 1, s_dir[pb ^ 1u], &s_ver[pb ^ 1u], lane);
        __syncwarp();
        uint32_t run = 0, nbm = 0, apost = 0;
        for (uint32_t base = 0; base < nb; base += 32) {
          const uint32_t i = base + lane;
          const uint32_t v = i < nb ? t_cp[i] : 0;
          const bool isbm = i < nb && t_cnt[i] >= BMIN;
          const uint32_t isb = __ballot_sync(0xFFFFFFFFu, isbm);
          if (isbm) t_bl[nbm + __popc(isb & ((1u << lane) - 1u))] = (uint8_t)i;
          nbm += __popc(isb);
          uint32_t ap = (i < nb && !isbm) ? t_cnt[i] : 0u;
          for (int dd = 16; dd > 0; dd >>= 1) ap += __shfl_xor_sync(0xFFFFFFFFu, ap, dd);
          apost += ap;
          uint32_t x = v;
          for (int dd = 1; dd < 32; dd <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, dd);
            if (lane >= (uint32_t)dd) x += y;
          }
          if (i < nb) t_cp[i] = run + x - v;
          run += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
        if (lane == 0) {
          t_cp[nb] = run;
          part[0] = run;
          s_nbm = nbm;
          s_apost = apost;
          s_ntl = 0;
          // accumulators the tile writes: 1 acc (array terms), 2 bacc (bitmaps)
          s_dirty = (bi ? s_dirty : 0u) | (run ? 1u : 0u) | (nbm ? 2u : 0u);
        }
      }
      __syncthreads();
      const uint16_t *post = a.tile_post[(uint64_t)t * 2 + s_vt];
      // a touched-list tile (block-uniform): arrays only, bound above zero
      touch = nbatch == 1 && s_nbm == 0 && lb > kZeroBin && s_apost <= kTouchCap;
      // bitmap terms: thread tid owns ids 4*tid + 4*kScoreThreads*g .. +3;
      // their partial sums go to bacc, which only the owner touches, so the
      // array terms need not wait for them
      const uint32_t nbm = s_nbm;
      for (uint32_t g0 = 0; g0 < T && nbm > 0; g0 += 4 * kScoreThreads * kBmGroups) {
        float4 r[kBmGroups];
#pragma unroll
        for (uint32_t g = 0; g < kBmGroups; ++g) {
          const uint32_t d0 = g0 + g * 4 * kScoreThreads + 4 * tid;
          r[g] = d0 < T ? *(const float4 *)(bacc + d0) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (uint32_t kk = 0; kk < nbm; ++kk) {
          const uint32_t k = t_bl[kk];
          const float v = t_v[k];
          const bool pos = v > 0.0f;
          const S *plane = (const S *)(pos ? a.U : a.L);
          const S *row[HS];
#pragma unroll
          for (uint32_t o = 0; o < HS; ++o)
            if (o < a.h) row[o] = plane + (uint64_t)t_bin[k * a.h + o] * a.cap + id0;
          const uint32_t *bm = (const uint32_t *)(post + t_start[k]);
#pragma unroll
          for (uint32_t g = 0; g < kBmGroups; ++g) {
            const uint32_t d0 = g0 + g * 4 * kScoreThreads + 4 * tid;
            if (d0 < T) {
              const uint32_t bits = __ldg(bm + (d0 >> 5)) >> (d0 & 31);
              const float4 x = decode4<H, S>(row, a.h, pos, d0);
              if (bits & 1u) r[g].x = fmaf(v, x.x, r[g].x);
              if (bits & 2u) r[g].y = fmaf(v, x.y, r[g].y);
              if (bits & 4u) r[g].z = fmaf(v, x.z, r[g].z);
              if (bits & 8u) r[g].w = fmaf(v, x.w, r[g].w);
            }
          }
        }
#pragma unroll
        for (uint32_t g = 0; g < kBmGroups; ++g) {
          const uint32_t d0 = g0 + g * 4 * kScoreThreads + 4 * tid;
          if (d0 < T) *(float4 *)(bacc + d0) = r[g];
        }
      }
      // array terms; on a touched-list tile each first mark of an id lists it
      auto add = [&](uint32_t d, float x) {
        atomicAdd(&acc[d], x);
        if (touch) {
          const uint32_t bit = 1u << (d & 31);
          if (!(atomicOr(&touched[d >> 5], bit) & bit)) tlist[atomicAdd(&s_ntl, 1u)] = (uint16_t)d;
        }
      };
      const uint32_t C = part[0];
      if (WALK) {
        // walk 1: the batch's array postings as one sequence, thread tid taking
        // postings tid, tid + kScoreThreads, ... (4 per pass, loads in flight
        // together); a posting's term is the last i with t_cp[i] <= p
        for (uint32_t q0 = tid; q0 < C; q0 += 4 * kScoreThreads) {
          uint32_t d[4], ti[4];
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t p = q0 + u * kScoreThreads;
            d[u] = SINN_TOMB;
            ti[u] = 0;
            if (p < C) {
              uint32_t i = 0, hi = nb;
              while (hi - i > 1) {
                const uint32_t mid = (i + hi) >> 1;
                if (t_cp[mid] <= p) i = mid;
                else hi = mid;
              }
              ti[u] = i;
              d[u] = (uint32_t)__ldg(post + t_start[i] + (p - t_cp[i]));
              if (!(d[u] & SINN_TOMB) && !SINN_IN_BOUNDS(d[u] < T, a.err)) d[u] = SINN_TOMB;
            }
          }
          float x[4];
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) {
            x[u] = 0.0f;
            if (d[u] & SINN_TOMB) continue;
            const uint32_t k = ti[u];
            const float v = t_v[k];
            const bool pos = v > 0.0f;
            const S *plane = (const S *)(pos ? a.U : a.L);
            const S *row[HS];
#pragma unroll
            for (uint32_t o = 0; o < HS; ++o)
              if (o < a.h) row[o] = plane + (uint64_t)t_bin[k * a.h + o] * a.cap + id0;
            x[u] = v * decode<H, S>(row, a.h, pos, d[u]);
          }
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u)
            if (!(d[u] & SINN_TOMB)) add(d[u], x[u]);
        }
      }
      const uint32_t c_beg = WALK ? 0u : (uint32_t)((uint64_t)C * wid / NW);
      const uint32_t c_end = WALK ? 0u : (uint32_t)((uint64_t)C * (wid + 1) / NW);
      if (c_beg < c_end) {
        uint32_t i = 0, hi = nb;  // term of c_beg: last i with t_cp[i] <= c_beg
        while (hi - i > 1) {
          const uint32_t mid = (i + hi) >> 1;
          if (t_cp[mid] <= c_beg) i = mid;
          else hi = mid;
        }
        uint32_t c_start = 0, c_next = 0, lo = 0, len = 0;
        float v = 0.0f;
        bool pos = true;
        const S *row[HS];
        auto load_term = [&]() {
          c_start = t_cp[i];
          c_next = t_cp[i + 1];
          lo = t_start[i];
          len = t_cnt[i];
          v = t_v[i];
          pos = v > 0.0f;
          const S *plane = (const S *)(pos ? a.U : a.L);
#pragma unroll
          for (uint32_t o = 0; o < HS; ++o)
            if (o < a.h) row[o] = plane + (uint64_t)t_bin[i * a.h + o] * a.cap + id0;
        };
        load_term();
        for (uint32_t c = c_beg; c < c_end;) {
          while (c >= c_next) {
            ++i;
            load_term();
          }
          const uint32_t nck = min(min(4u, c_end - c), c_next - c);
          const uint32_t p0 = (c - c_start) * 32 + lane;
          uint32_t d[4];
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t p = p0 + u * 32;
            d[u] = (u < nck && p < len) ? (uint32_t)__ldg(post + lo + p) : SINN_TOMB;
            if (!(d[u] & SINN_TOMB) && !SINN_IN_BOUNDS(d[u] < T, a.err)) d[u] = SINN_TOMB;
          }
          float x[4];
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u)
            x[u] = (d[u] & SINN_TOMB) ? 0.0f : decode<H, S>(row, a.h, pos, d[u]);
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u)
            if (!(d[u] & SINN_TOMB)) add(d[u], v * x[u]);
          c += nck;
        }
      }
    }
    __syncthreads();  // the array terms' atomics are complete
    if (touch) {
      // touched-list epilogue: the ids an array posting reached, each read,
      // cleared and, at or above the bound, counted and emitted
      const uint32_t ntl = s_ntl;
      for (uint32_t base = 0; base < ntl; base += kScoreThreads) {
        const uint32_t i = base + tid;
        const bool in = i < ntl;
        const uint32_t d = in ? tlist[i] : 0u;
        float sc = 0.0f;
        if (in) {
          sc = acc[d];
          acc[d] = 0.0f;
          touched[d >> 5] = 0u;
        }
        const uint32_t key = sinn_f2key(sc + 0.0f);
        const uint64_t id = id0 + d;
        const bool em = in && sinn_is_live(a.live, id) && (key >> 20) >= lb &&
                        (!a.recent || !((sinn_ld_gpu(a.recent + (id >> 5)) >> (id & 31)) & 1u) ||
                         sinn_visible_recent(a.born, a.died, a.seq, id));
        if (em) atomicAdd(&gh[key >> 20], 1u);
        if (__any_sync(0xFFFFFFFFu, em)) {
          const uint32_t p = warp_append(em, &bt.ecnt[b]);
          if (em && p < kEmitCap) el[p] = ((uint64_t)key << 32) | (uint32_t)~(uint32_t)(id0 + d);
        }
      }
      continue;
    }
    // epilogue, 4 consecutive ids per thread: score = array part + bitmap part
    const uint32_t dirty = s_dirty;
    for (uint32_t g0 = 0; g0 < T; g0 += 4 * kScoreThreads) {
      const uint32_t d0 = g0 + 4 * tid;
      const bool in = d0 < T;
      float4 sa = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (dirty & 1u) {
          sa = *(const float4 *)(acc + d0);
          *(float4 *)(acc + d0) = z;
        }
        if (dirty & 2u) {
          const float4 y = *(const float4 *)(bacc + d0);
          *(float4 *)(bacc + d0) = z;
          sa = make_float4(sa.x + y.x, sa.y + y.y, sa.z + y.z, sa.w + y.w);
        }
      }
      // live ids, less those the search's snapshot does not count
      const uint32_t lwv =
          visible4(a, id0 + d0, in ? (__ldg(a.live + ((id0 + d0) >> 5)) >> (d0 & 31)) & 15u : 0u,
                   lane);
      const float rv[4] = {sa.x, sa.y, sa.z, sa.w};
      // ids at or above the running bound count and are emitted
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t key = sinn_f2key(rv[q] + 0.0f);
        const bool em = ((lwv >> q) & 1u) && (key >> 20) >= lb;
        if (em) atomicAdd(&gh[key >> 20], 1u);
        if (__any_sync(0xFFFFFFFFu, em)) {
          const uint32_t p = warp_append(em, &bt.ecnt[b]);
          if (em && p < kEmitCap)
            el[p] = ((uint64_t)key << 32) | (uint32_t)~(uint32_t)(id0 + d0 + q);
        }
      }
    }
  }
  // The final boundary bin is never below any bound used, so the
  // histogram stays exact from the boundary bin up and every candidate is
  // emitted.  Refresh the query's bound each time the tiles done cross a
  // multiple of bound_every.
  __threadfence();  // every count is visible before the tiles are reported done
  __syncthreads();
  if (tid == 0) part[NW + 1] = atomicAdd(&bt.tdone[b], t_end - t_beg);
  __syncthreads();
  const uint32_t kq = bt.sel[b].kq;
  const uint32_t done0 = part[NW + 1], done1 = done0 + (t_end - t_beg);
  if (done1 / a.bound_every > done0 / a.bound_every && kq > 0) {
    const uint32_t nbnd = bound_from_hist(gh, kq, lb, part);
    if (tid == 0 && nbnd > 0) atomicMax(&bt.bound[b], nbnd);
  }
}

// Grid (query, group of tiles_per_block tiles), queries fastest.
template <int H, typename S, bool WALK>
__global__ void __launch_bounds__(kScoreThreads, 4) k_score_emit(ScoreArgs a, Batch bt) {
  extern __shared__ uint32_t sm[];
  const uint32_t t0 = blockIdx.y * a.tpb;
  score_tiles<H, S, WALK>(a, bt, blockIdx.x, t0, min(a.tiles, t0 + a.tpb), sm);
}

// The same work as k_score_emit from a fixed grid of blocks: each block takes
// (query, group) items from a counter in the same query-fastest order until
// none is left.
template <int H, typename S, bool WALK>
__global__ void __launch_bounds__(kScoreThreads, 4)
    k_score_emit_persistent(ScoreArgs a, Batch bt, uint32_t nb, unsigned long long *next) {
  extern __shared__ uint32_t sm[];
  __shared__ unsigned long long s_item;
  const uint64_t groups = (a.tiles + a.tpb - 1) / a.tpb, total = groups * nb;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1ull);
    __syncthreads();
    const uint64_t item = s_item;
    __syncthreads();  // every thread has read the item before the next draw
    if (item >= total) break;
    const uint32_t b = (uint32_t)(item % nb), t0 = (uint32_t)(item / nb) * a.tpb;
    score_tiles<H, S, WALK>(a, bt, b, t0, min(a.tiles, t0 + a.tpb), sm);
  }
}

// Dense scoring of the flagged queries: launches of few queries, and the
// fallback of batched ones.  Work items are (query, tile, slice of
// kLoneSlice ids), queries fastest so the blocks resident together share a
// tile's lists and sketch rows, and one query alone still fills the GPU
// (T / kLoneSlice items per tile).  A block stages the query's terms for
// the item's tile (directory entries, weights, bins), then:
//   bitmap terms: thread t owns ids 4t..4t+3 of the slice and keeps their
//   partial scores in registers; terms are taken four at a time (h = 1) or
//   two at a time so their bitmap words and sketch values are in flight
//   together;
//   array terms: warp w takes terms w, w + 8, ...; its lanes read the
//   container's postings and add those inside the slice into shared memory
//   with atomics.
// Every live id's key is written (0 for a slot that is not live) and its bin
// counted in a shared histogram, added to the query's global one when the
// block moves to another query or ends (few global atomics per bin, where
// one histogram for the whole grid would serialise on the popular bins).
constexpr uint32_t kLoneThreads = 256;
constexpr uint32_t kLoneSlice = 4 * kLoneThreads;

template <int H, typename S>
__device__ __forceinline__ void lone_bitmap_term(const ScoreArgs &a, const uint16_t *post,
                                                 const uint32_t *t_start, const float *t_v,
                                                 const uint32_t *t_bin, uint32_t k, uint64_t id0,
                                                 uint32_t d0, uint32_t *bits, float4 *x,
                                                 float *v) {
  constexpr uint32_t HS = H > 0 ? (uint32_t)H : (uint32_t)SINN_MAX_H;
  *v = t_v[k];
  const bool pos = *v > 0.0f;
  const S *plane = (const S *)(pos ? a.U : a.L);
  const S *row[HS];
#pragma unroll
  for (uint32_t o = 0; o < HS; ++o)
    if (o < a.h) row[o] = plane + (uint64_t)t_bin[k * a.h + o] * a.cap + id0;
  *bits = __ldg((const uint32_t *)(post + t_start[k]) + (d0 >> 5)) >> (d0 & 31);
  *x = decode4<H, S>(row, a.h, pos, d0);
}

__device__ __forceinline__ void lone_fma(float4 &r, uint32_t bits, float4 x, float v) {
  if (bits & 1u) r.x = fmaf(v, x.x, r.x);
  if (bits & 2u) r.y = fmaf(v, x.y, r.y);
  if (bits & 4u) r.z = fmaf(v, x.z, r.z);
  if (bits & 8u) r.w = fmaf(v, x.w, r.w);
}

__device__ __noinline__ void pick_all(Batch bt, uint32_t level);

template <int H, typename S>
__global__ void __launch_bounds__(kLoneThreads, 8) k_score_lone(ScoreArgs a, Batch bt,
                                                                uint32_t fuse_pick) {
  constexpr uint32_t HS = H > 0 ? (uint32_t)H : (uint32_t)SINN_MAX_H;
  constexpr uint32_t NW = kLoneThreads / 32;
  __shared__ float4 acc4[kLoneSlice / 4];  // array terms of the slice (atomics)
  __shared__ uint32_t hist[4096];          // key bins of the block's current query
  __shared__ uint32_t t_start[kTermBatch], t_cnt[kTermBatch];
  __shared__ uint32_t t_bin[kTermBatch * SINN_MAX_H];
  __shared__ float t_v[kTermBatch];
  __shared__ uint8_t t_bl[kTermBatch], t_al[kTermBatch];  // bitmap / array terms
  __shared__ uint32_t s_nbm, s_nal, s_v;
  float *acc = (float *)acc4;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t T = a.T, BMIN = T >> SINN_BITMAP_SHIFT, spt = T / kLoneSlice;
  const uint32_t nf = *bt.nflag;
  const uint64_t items = (uint64_t)nf * a.tiles * spt;
  for (uint32_t i = tid; i < 4096; i += kLoneThreads) hist[i] = 0u;
  uint32_t cur = 0xFFFFFFFFu;  // query whose counts the histogram holds
  auto flush = [&]() {
    uint32_t *gh = bt.hist0 + (uint64_t)cur * 4096;
    for (uint32_t i = tid; i < 4096; i += kLoneThreads) {
      const uint32_t c = hist[i];
      if (c) {
        atomicAdd(&gh[i], c);
        hist[i] = 0u;
      }
    }
  };
  for (uint64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const uint32_t b = bt.flagged[w % nf];
    const uint64_t r0 = w / nf;
    const uint32_t t = (uint32_t)(r0 / spt), s0 = (uint32_t)(r0 % spt) * kLoneSlice;
    __syncthreads();  // the previous item is done with the shared state
    if (b != cur) {   // block-uniform
      if (cur != 0xFFFFFFFFu) flush();
      cur = b;
      __syncthreads();
    }
    const uint32_t nt = bt.ns[b];  // Alg. 6 scores the budget's prefix
    const QTerm *terms = bt.terms + (uint64_t)b * a.qmax;
    const uint64_t id0 = (uint64_t)t << a.log2T;
    const uint32_t d0 = s0 + 4 * tid;  // this thread's 4 ids
    if (tid == 0) s_v = __ldcg(a.sel + t);  // the tile's copy, for the whole item
    __syncthreads();
    const uint2 *dir = a.tile_dir + ((uint64_t)t * 2 + s_v) * a.n;
    const uint16_t *post = a.tile_post[(uint64_t)t * 2 + s_v];
    acc4[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t i0 = 0; i0 < nt; i0 += kTermBatch) {
      const uint32_t nb = min(kTermBatch, nt - i0);
      if (i0) __syncthreads();  // the previous batch is consumed
      if (wid == 0) {
        for (uint32_t k = lane; k < nb; k += 32) {
          const QTerm q = terms[i0 + k];
          const uint2 de = dir[q.j];
          t_start[k] = de.x;
          t_cnt[k] = de.y;
          t_v[k] = q.v;
          for (uint32_t o = 0; o < a.h; ++o) {
            const uint32_t bin = a.pi[(uint64_t)q.j * a.h + o];
            t_bin[k * a.h + o] = SINN_IN_BOUNDS(bin < a.m, a.err) ? bin : 0u;
          }
        }
        __syncwarp();
        uint32_t nbm = 0, nal = 0;
        for (uint32_t base = 0; base < nb; base += 32) {
          const uint32_t i = base + lane;
          const uint32_t c = i < nb ? t_cnt[i] : 0u;
          const uint32_t mb = __ballot_sync(0xFFFFFFFFu, c >= BMIN);
          const uint32_t ma = __ballot_sync(0xFFFFFFFFu, c > 0 && c < BMIN);
          const uint32_t below = (1u << lane) - 1u;
          if (c >= BMIN) t_bl[nbm + __popc(mb & below)] = (uint8_t)i;
          if (c > 0 && c < BMIN) t_al[nal + __popc(ma & below)] = (uint8_t)i;
          nbm += __popc(mb);
          nal += __popc(ma);
        }
        if (lane == 0) {
          s_nbm = nbm;
          s_nal = nal;
        }
      }
      __syncthreads();  // also orders the zeroed accumulator before the atomics
      const uint32_t nbm = s_nbm;
      uint32_t kk = 0;
      // (four terms in flight fit the registers with one sketch row per term)
      for (; H == 1 && kk + 3 < nbm; kk += 4) {
        uint32_t b0, b1, b2, b3;
        float4 x0, x1, x2, x3;
        float v0, v1, v2, v3;
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk], id0, d0, &b0, &x0, &v0);
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk + 1], id0, d0, &b1, &x1,
                               &v1);
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk + 2], id0, d0, &b2, &x2,
                               &v2);
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk + 3], id0, d0, &b3, &x3,
                               &v3);
        lone_fma(r, b0, x0, v0);
        lone_fma(r, b1, x1, v1);
        lone_fma(r, b2, x2, v2);
        lone_fma(r, b3, x3, v3);
      }
      for (; kk + 1 < nbm; kk += 2) {
        uint32_t b0, b1;
        float4 x0, x1;
        float v0, v1;
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk], id0, d0, &b0, &x0, &v0);
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk + 1], id0, d0, &b1, &x1,
                               &v1);
        lone_fma(r, b0, x0, v0);
        lone_fma(r, b1, x1, v1);
      }
      if (kk < nbm) {
        uint32_t b0;
        float4 x0;
        float v0;
        lone_bitmap_term<H, S>(a, post, t_start, t_v, t_bin, t_bl[kk], id0, d0, &b0, &x0, &v0);
        lone_fma(r, b0, x0, v0);
      }
      const uint32_t nal = s_nal;
      for (uint32_t ai = wid; ai < nal; ai += NW) {
        const uint32_t k = t_al[ai];
        const uint32_t lo = t_start[k], cnt = t_cnt[k];
        const float v = t_v[k];
        const bool pos = v > 0.0f;
        const S *plane = (const S *)(pos ? a.U : a.L);
        const S *row[HS];
#pragma unroll
        for (uint32_t o = 0; o < HS; ++o)
          if (o < a.h) row[o] = plane + (uint64_t)t_bin[k * a.h + o] * a.cap + id0;
        for (uint32_t p = lane; p < cnt; p += 32) {
          const uint32_t dd = __ldg(post + lo + p);
          if (dd & SINN_TOMB) continue;
          if (!SINN_IN_BOUNDS(dd < T, a.err)) continue;
          if (dd - s0 >= kLoneSlice) continue;  // outside the slice
          atomicAdd(&acc[dd - s0], v * decode<H, S>(row, a.h, pos, dd));
        }
      }
    }
    __syncthreads();  // the array terms' atomics are complete
    const float4 x = acc4[tid];
    const float rv[4] = {r.x + x.x, r.y + x.y, r.z + x.z, r.w + x.w};
    // live ids, less those the search's snapshot does not count
    const uint32_t lwv =
        visible4(a, id0 + d0, (__ldg(a.live + ((id0 + d0) >> 5)) >> (d0 & 31)) & 15u, lane);
    uint32_t kv[4];
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const bool lv = (lwv >> q) & 1u;
      const uint32_t key = sinn_f2key(rv[q] + 0.0f);
      kv[q] = lv ? key : 0u;
      if (lv) atomicAdd(&hist[key >> 20], 1u);
    }
    *(uint4 *)(bt.keys + (uint64_t)b * a.cap + id0 + d0) = make_uint4(kv[0], kv[1], kv[2], kv[3]);
  }
  __syncthreads();
  if (cur != 0xFFFFFFFFu) flush();
  // with fuse_pick, the launch's last block makes the level-0 picks
  if (fuse_pick && last_block(bt.tick, gridDim.x)) pick_all(bt, 0);
}

// Kernels specialised for h = 1 and h = 2 (the common sketch shapes); other h
// use the general loop.
struct ScoreKernels {
  void (*emit)(ScoreArgs, Batch);
  void (*dense)(ScoreArgs, Batch, uint32_t);
  void (*persistent)(ScoreArgs, Batch, uint32_t, unsigned long long *);
};

template <typename S, bool WALK>
ScoreKernels score_kernels_for(uint32_t h) {
  if (h == 1)
    return {k_score_emit<1, S, WALK>, k_score_lone<1, S>, k_score_emit_persistent<1, S, WALK>};
  if (h == 2)
    return {k_score_emit<2, S, WALK>, k_score_lone<2, S>, k_score_emit_persistent<2, S, WALK>};
  return {k_score_emit<0, S, WALK>, k_score_lone<0, S>, k_score_emit_persistent<0, S, WALK>};
}

// Sketch bins as fp32 or as bfloat16 bits; array postings of the batched
// kernels walked in per-term chunks or spread over the block.
ScoreKernels score_kernels(uint32_t h, bool bf16, bool walk) {
  if (bf16) return walk ? score_kernels_for<uint16_t, true>(h) : score_kernels_for<uint16_t, false>(h);
  return walk ? score_kernels_for<float, true>(h) : score_kernels_for<float, false>(h);
}

// ------------------------------------------------------------------ select
// Find, scanning bins from the top, the bin where the running count reaches
// rem.  Returns (bin, count above the bin).  Block of at least 128 threads
// (the first 128 read); the counts are read from L2.
__device__ void find_bin(const uint32_t *hist, uint32_t nb, uint32_t rem, uint32_t *out_bin,
                         uint32_t *out_above) {
  __shared__ uint32_t sums[128];
  __shared__ uint32_t res[2];
  const uint32_t tid = threadIdx.x, per = nb / 128;
  if (tid < 128) {
    // thread tid owns bins [nb - (tid+1)*per, nb - tid*per), highest first
    const uint32_t hi = nb - tid * per;
    uint32_t s = 0;
    for (uint32_t i = 0; i < per; ++i) s += __ldcg(hist + hi - 1 - i);
    sums[tid] = s;
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0, found = 0;
    for (uint32_t w = 0; w < 128 && !found; ++w) {
      if (run + sums[w] >= rem) {
        uint32_t top = nb - w * per;
        for (uint32_t i = 0; i < per; ++i) {
          uint32_t c = __ldcg(hist + top - 1 - i);
          if (run + c >= rem) {
            res[0] = top - 1 - i;
            res[1] = run;
            found = 1;
            break;
          }
          run += c;
        }
      } else {
        run += sums[w];
      }
    }
    if (!found) {  // cannot happen when rem <= sum(hist)
      res[0] = 0;
      res[1] = run;
    }
  }
  __syncthreads();
  *out_bin = res[0];
  *out_above = res[1];
}

// Level-0 pick for every query of the batch from its complete histogram.
// Emitted lists hold every key at or above the final boundary bin (the
// running bound never exceeds it), so the list path suffices unless the list
// overflowed or the boundary bin is too large to buffer: then the query is
// flagged for the dense fallback.
__global__ void k_pick_list(Batch bt) {
  const uint32_t b = blockIdx.x;
  SelState st = bt.sel[b];
  if (st.kq == 0) return;
  uint32_t bin, above;
  find_bin(bt.hist0 + (uint64_t)b * 4096, 4096, st.kq, &bin, &above);
  if (threadIdx.x == 0) {
    const uint32_t cnt = bt.hist0[(uint64_t)b * 4096 + bin];
    // the dense fallback also takes a histogram short of kq keys (not
    // expected: every live id at or above the running bound is counted)
    if (bt.ecnt[b] > kEmitCap || cnt > kBoundCap || above + cnt < st.kq) {
      bt.flagged[atomicAdd(bt.nflag, 1u)] = b;
      st.dense = 1;
      st.mode = SEL_DONE;
    } else {
      st.prefix = bin;
      st.pbits = 12;
      st.rem = st.kq - above;
      st.cnt = cnt;
      st.mode = SEL_COMPACT;
      st.dense = 0;
    }
    bt.sel[b] = st;
  }
}

// Split each emitted list: keys above the boundary bin are candidates, keys in
// it go to the boundary buffer.
__global__ void k_compact_list(Batch bt, uint32_t kpmax) {
  const uint32_t b = blockIdx.x;
  const SelState st = bt.sel[b];
  if (st.mode != SEL_COMPACT || st.dense) return;
  const uint32_t ne = min(bt.ecnt[b], kEmitCap);
  const uint64_t *el = bt.elist + (uint64_t)b * kEmitCap;
  uint64_t *cand = bt.cand + (uint64_t)b * kpmax;
  uint64_t *bnd = bt.bnd + (uint64_t)b * kBoundCap;
  uint32_t *ncand = &bt.sel[b].ncand, *nbnd = &bt.sel[b].nbnd;
  for (uint32_t i0 = 0; i0 < ne; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const uint64_t k64 = i < ne ? el[i] : 0ull;
    const uint32_t top = (uint32_t)(k64 >> 52);
    const bool up = i < ne && top > st.prefix;
    const bool eq = i < ne && top == st.prefix;
    uint32_t p = warp_append(up, ncand);
    if (up && p < kpmax) cand[p] = k64;
    p = warp_append(eq, nbnd);
    if (eq && p < kBoundCap) bnd[p] = k64;
  }
}

// Fallback: reset the flagged queries' histogram (their keys are recomputed).
__global__ void k_fb_reset(Batch bt) {
  const uint32_t nf = *bt.nflag;
  for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
    const uint32_t b = bt.flagged[f];
    for (uint32_t i = threadIdx.x; i < 4096; i += blockDim.x) {
      bt.hist0[(uint64_t)b * 4096 + i] = 0;
      bt.hist1[(uint64_t)b * 4096 + i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) bt.hist2[(uint64_t)b * 256 + i] = 0;
  }
}

// Dense-path pick at a level for flagged query b (one block; the counts
// may come from the same launch, so they are read from L2).
__device__ void pick_one(Batch bt, uint32_t b, uint32_t level) {
  SelState st = bt.sel[b];
  if (level == 0) {
    // the dense histogram counts every id the search sees: a snapshot may
    // see fewer than the live count that bounded kq
    __shared__ uint32_t s_tot;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    uint32_t c = 0;
    for (uint32_t i = threadIdx.x; i < 4096; i += blockDim.x)
      c += __ldcg(bt.hist0 + (uint64_t)b * 4096 + i);
    atomicAdd(&s_tot, c);
    __syncthreads();
    const uint32_t tot = s_tot;
    __syncthreads();
    if (tot < st.kq) {
      st.kq = tot;
      if (threadIdx.x == 0) bt.sel[b].kq = tot;
    }
    if (st.kq == 0) {
      if (threadIdx.x == 0) {
        st.mode = SEL_DONE;
        bt.sel[b] = st;
      }
      __syncthreads();
      return;
    }
    st.rem = st.kq;
    st.prefix = 0;
    st.pbits = 0;
  } else if ((level == 1 && st.mode != SEL_L1) || (level == 2 && st.mode != SEL_L2)) {
    return;
  }
  const uint32_t nb = level == 2 ? 256u : 4096u;
  const uint32_t *h = level == 0 ? bt.hist0 + (uint64_t)b * 4096
                                 : level == 1 ? bt.hist1 + (uint64_t)b * 4096
                                              : bt.hist2 + (uint64_t)b * 256;
  uint32_t bin, above;
  find_bin(h, nb, st.rem, &bin, &above);
  if (threadIdx.x == 0) {
    const uint32_t digits = level == 2 ? 8u : 12u;
    st.prefix = (st.prefix << digits) | bin;
    st.pbits += digits;
    st.rem -= above;
    st.cnt = __ldcg(h + bin);
    if (st.cnt <= kBoundCap) st.mode = SEL_COMPACT;
    else st.mode = level == 0 ? SEL_L1 : level == 1 ? SEL_L2 : SEL_TIES;
    bt.sel[b] = st;
  }
  __syncthreads();
}

// The pick at a level for every flagged query, by one block (the last of a
// launch that produced the counts).
__device__ __noinline__ void pick_all(Batch bt, uint32_t level) {
  const uint32_t nf = __ldcg(bt.nflag);
  for (uint32_t f = 0; f < nf; ++f) pick_one(bt, __ldcg(bt.flagged + f), level);
}

// Dense-path pick at a level for the flagged queries.
__global__ void k_pick(Batch bt, uint32_t level) {
  const uint32_t nf = *bt.nflag;
  for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) pick_one(bt, bt.flagged[f], level);
}

// Counts of the next digit (level 1: 12 bits, level 2: 8 bits) of query b's
// dense keys in [beg, end) that match its current prefix, added into the
// query's histogram of that level (hist: the block's shared scratch).
__device__ void hist_keys(Batch bt, uint32_t b, const SelState &st, uint64_t cap, uint64_t beg,
                          uint64_t end, uint32_t level, uint32_t *hist) {
  const uint32_t nb = level == 1 ? 4096u : 256u;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint32_t shift_p = 32 - st.pbits;  // 20 or 8
  const uint32_t shift_d = level == 1 ? 8u : 0u;
  const uint32_t dmask = nb - 1;
  const uint32_t *keys = bt.keys + (uint64_t)b * cap;
  for (uint64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const uint32_t key = keys[i];
    if (key != 0u && (key >> shift_p) == st.prefix) atomicAdd(&hist[(key >> shift_d) & dmask], 1u);
  }
  __syncthreads();
  uint32_t *gh = level == 1 ? bt.hist1 + (uint64_t)b * 4096 : bt.hist2 + (uint64_t)b * 256;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
    if (hist[i]) atomicAdd(&gh[i], hist[i]);
  __syncthreads();
}

// Histogram of the next digit over dense keys matching the current prefix.
// With fuse set, the launch's last block then makes the level's pick; with
// fuse = 2 (level 1 only) that block also counts and picks level 2 for any
// query whose boundary bin is still too large (rare: massive ties), so one
// launch covers both levels.
__global__ void k_hist_level(Batch bt, uint64_t cap, uint64_t span, uint32_t level,
                             uint32_t fuse) {
  __shared__ uint32_t hist[4096];
  __shared__ uint32_t s_any;
  __shared__ SelState s_st;
  const uint32_t nf = *bt.nflag;
  const uint64_t chunks = (span + kChunk - 1) / kChunk;
  const SelMode want = level == 1 ? SEL_L1 : SEL_L2;
  // the level is needed only for a boundary bin too large to buffer: look
  // once before walking the keys
  if (threadIdx.x == 0) s_any = 0u;
  __syncthreads();
  for (uint32_t f = threadIdx.x; f < nf; f += blockDim.x)
    if (bt.sel[bt.flagged[f]].mode == want) s_any = 1u;
  __syncthreads();
  for (uint64_t w = blockIdx.x; s_any && w < nf * chunks; w += gridDim.x) {
    const uint32_t b = bt.flagged[w / chunks];
    const SelState st = bt.sel[b];
    if (st.mode != want) continue;
    const uint64_t beg = (w % chunks) * kChunk;
    hist_keys(bt, b, st, cap, beg, (beg + kChunk < span) ? beg + kChunk : span, level, hist);
  }
  if (fuse && last_block(bt.tick + level, gridDim.x)) {
    pick_all(bt, level);
    if (fuse == 2 && level == 1) {
      const uint32_t nf2 = __ldcg(bt.nflag);
      for (uint32_t f = 0; f < nf2; ++f) {
        const uint32_t b = __ldcg(bt.flagged + f);
        if (threadIdx.x < sizeof(SelState) / 4)
          ((uint32_t *)&s_st)[threadIdx.x] = __ldcg((const uint32_t *)&bt.sel[b] + threadIdx.x);
        __syncthreads();
        if (s_st.mode == SEL_L2) hist_keys(bt, b, s_st, cap, 0, span, 2, hist);
        __syncthreads();  // s_st is read again for the next query
      }
      pick_all(bt, 2);
    }
  }
}

// Dense-path collection: keys above the boundary bin are candidates; in
// COMPACT mode the boundary bin's keys are buffered too.  A block takes a
// chunk of kChunk keys, 8 per thread, counts its hits, reserves room for the
// whole block with one atomic per list and writes them.
__device__ void refine_one(Batch bt, uint32_t b, uint64_t cap, uint64_t span, uint32_t kpmax);

// With refine_nb > 0, the launch's last block then refines queries
// 0 .. refine_nb - 1 (the work of k_refine).
__global__ void __launch_bounds__(256) k_compact(Batch bt, uint64_t cap, uint64_t span,
                                                 uint32_t kpmax, uint32_t refine_nb) {
  constexpr uint32_t PER = kChunk / 256;
  __shared__ uint32_t wsum[2][8], s_base[2];
  const uint32_t nf = *bt.nflag;
  const uint64_t chunks = (span + kChunk - 1) / kChunk;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (uint64_t w = blockIdx.x; w < nf * chunks; w += gridDim.x) {
    const uint32_t b = bt.flagged[w % nf];
    const SelState st = bt.sel[b];  // block-uniform
    if (st.mode != SEL_COMPACT && st.mode != SEL_TIES) continue;
    const uint32_t shift = 32 - st.pbits;
    const uint32_t *keys = bt.keys + (uint64_t)b * cap;
    uint64_t *cand = bt.cand + (uint64_t)b * kpmax;
    uint64_t *bnd = bt.bnd + (uint64_t)b * kBoundCap;
    uint32_t *ncand = &bt.sel[b].ncand, *nbnd = &bt.sel[b].nbnd;
    const uint64_t beg = (w / nf) * kChunk + (uint64_t)tid * PER;
    uint32_t key[PER];
    uint32_t nu = 0, ne = 0, fu = 0, fe = 0;  // counts and flag bits (up, equal)
#pragma unroll
    for (uint32_t q = 0; q < PER; q += 4) {
      const uint4 v = beg + q + 4 <= span ? *(const uint4 *)(keys + beg + q)
                                          : make_uint4(0u, 0u, 0u, 0u);
      key[q] = v.x;
      key[q + 1] = v.y;
      key[q + 2] = v.z;
      key[q + 3] = v.w;
    }
#pragma unroll
    for (uint32_t q = 0; q < PER; ++q) {
      const uint32_t top = shift == 32 ? 0u : (key[q] >> shift);
      const bool up = key[q] != 0u && top > st.prefix;
      const bool eq = key[q] != 0u && top == st.prefix && st.mode == SEL_COMPACT;
      fu |= (up ? 1u : 0u) << q;
      fe |= (eq ? 1u : 0u) << q;
      nu += up;
      ne += eq;
    }
    // block prefix of the counts: within warps, then over warps
    uint32_t xu = nu, xe = ne;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t yu = __shfl_up_sync(0xFFFFFFFFu, xu, d);
      const uint32_t ye = __shfl_up_sync(0xFFFFFFFFu, xe, d);
      if (lane >= (uint32_t)d) {
        xu += yu;
        xe += ye;
      }
    }
    if (lane == 31) {
      wsum[0][wid] = xu;
      wsum[1][wid] = xe;
    }
    __syncthreads();
    if (tid < 2) {
      uint32_t tot = 0;
      for (uint32_t i = 0; i < 8; ++i) {
        const uint32_t v = wsum[tid][i];
        wsum[tid][i] = tot;
        tot += v;
      }
      s_base[tid] = tot ? atomicAdd(tid == 0 ? ncand : nbnd, tot) : 0u;
    }
    __syncthreads();
    uint32_t pu = s_base[0] + wsum[0][wid] + xu - nu;
    uint32_t pe = s_base[1] + wsum[1][wid] + xe - ne;
#pragma unroll
    for (uint32_t q = 0; q < PER; ++q) {
      const uint64_t i = beg + q;
      const uint64_t k64 = ((uint64_t)key[q] << 32) | (uint32_t)~(uint32_t)i;
      if ((fu >> q) & 1u) {
        if (pu < kpmax) cand[pu] = k64;
        ++pu;
      }
      if ((fe >> q) & 1u) {
        if (pe < kBoundCap) bnd[pe] = k64;
        ++pe;
      }
    }
    __syncthreads();  // wsum and s_base are reused by the next chunk
  }
  if (refine_nb && last_block(bt.tick + 3, gridDim.x))
    for (uint32_t b = 0; b < refine_nb; ++b) refine_one(bt, b, cap, span, kpmax);
}

// Block-level selection of the r largest of n distinct 64-bit keys held in
// global memory (read from L2: they may come from the same launch): one
// 8-bit digit per pass from the top, stopping early once the prefix pins
// down exactly r keys.  Returns (prefix, mask): the selected
// keys are those with (key & mask) >= prefix.
__device__ void block_select_u64(const uint64_t *keys, uint32_t n, uint32_t r,
                                 uint64_t *out_prefix, uint64_t *out_mask) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_rem, s_stop;
  __shared__ uint64_t s_prefix, s_mask;
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_rem = r;
    s_stop = (r >= n) ? 1u : 0u;
  }
  __syncthreads();
  for (int shift = 56; shift >= 0 && !s_stop; shift -= 8) {
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint64_t pre = s_prefix, msk = s_mask;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint64_t k = __ldcg(keys + i);
      if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // the digit where the count from the top reaches rem: lane l sums the
      // 8 digits 255 - 8l ... 248 - 8l, a scan over lanes finds the lane
      // holding it, that lane finds the digit
      const uint32_t lane = threadIdx.x, top = 255 - 8 * lane, rem = s_rem;
      uint32_t c[8], sum = 0;
#pragma unroll
      for (uint32_t i = 0; i < 8; ++i) {
        c[i] = hist[top - i];
        sum += c[i];
      }
      uint32_t x = sum;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
      }
      const uint32_t before = x - sum;
      if (before < rem && x >= rem) {
        uint32_t run = before, dsel = top;
#pragma unroll
        for (uint32_t i = 0; i < 8; ++i) {
          if (run + c[i] >= rem) {
            dsel = top - i;
            break;
          }
          run += c[i];
        }
        s_rem = rem - run;
        s_prefix = pre | ((uint64_t)dsel << shift);
        s_mask = msk | (0xFFull << shift);
        if (hist[dsel] == rem - run) s_stop = 1u;  // the whole digit bucket is in
      }
    }
    __syncthreads();
  }
  *out_prefix = s_prefix;
  *out_mask = s_mask;
  __syncthreads();
}

// Rest of the boundary bin of query b: the rem best of its keys (COMPACT), or
// in TIES mode the rem smallest ids whose key equals the boundary value
// exactly.  One block of up to 512 threads; the state and the boundary keys
// may come from the same launch (read from L2).
__device__ void refine_one(Batch bt, uint32_t b, uint64_t cap, uint64_t span, uint32_t kpmax) {
  __shared__ SelState st;
  __shared__ uint32_t s_base, wsum[16];
  __syncthreads();  // st and s_base may still be read for the previous query
  if (threadIdx.x < sizeof(SelState) / 4)
    ((uint32_t *)&st)[threadIdx.x] = __ldcg((const uint32_t *)&bt.sel[b] + threadIdx.x);
  __syncthreads();
  if (st.mode != SEL_COMPACT && st.mode != SEL_TIES) return;
  uint64_t *cand = bt.cand + (uint64_t)b * kpmax;
  uint32_t *ncand = &bt.sel[b].ncand;
  if (st.mode == SEL_COMPACT) {
    const uint64_t *bnd = bt.bnd + (uint64_t)b * kBoundCap;
    const uint32_t nb = min(st.nbnd, kBoundCap);
    uint64_t pre, msk;
    block_select_u64(bnd, nb, st.rem, &pre, &msk);
    for (uint32_t i0 = 0; i0 < nb; i0 += blockDim.x) {
      const uint32_t i = i0 + threadIdx.x;
      const uint64_t k = i < nb ? __ldcg(bnd + i) : 0ull;
      const bool take = i < nb && (k & msk) >= pre;
      const uint32_t p = warp_append(take, ncand);
      if (take && p < kpmax) cand[p] = k;
    }
    return;
  }
  // SEL_TIES: ordered scan in id order
  const uint32_t *keys = bt.keys + (uint64_t)b * cap;
  const uint32_t tau = st.prefix;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t i0 = 0; i0 < span && s_base < st.rem; i0 += blockDim.x) {
    const uint64_t i = i0 + threadIdx.x;
    const bool m = i < span && keys[i] == tau;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, m);
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    uint32_t before = s_base;
    for (uint32_t w = 0; w < wid; ++w) before += wsum[w];
    before += __popc(bal & lanemask_lt());
    if (m && before < st.rem) {
      const uint32_t p = atomicAdd(ncand, 1u);
      if (p < kpmax) cand[p] = ((uint64_t)tau << 32) | (uint32_t)~(uint32_t)i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (uint32_t w = 0; w < blockDim.x / 32; ++w) tot += wsum[w];
      s_base += tot;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) k_refine(Batch bt, uint64_t cap, uint64_t span,
                                                uint32_t kpmax) {
  refine_one(bt, blockIdx.x, cap, span, kpmax);
}

// ------------------------------------------------------------------ re-rank
struct RerankArgs {
  const uint64_t *fwd_off;
  const uint32_t *fwd_nnz;
  const uint2 *fwd;
  uint64_t cap;
  uint64_t fwd_cap;  // entries of the vector store (bounds-check builds)
  uint32_t *err;
  uint32_t qmax, kpmax;
};

// Candidates a query's selection produced.  Equal to kq by construction (the
// histogram is exact from the boundary bin up); the minimum keeps every later
// read inside what was written even if that ever failed, and the re-rank
// raises the internal-error flag then.
__device__ __forceinline__ uint32_t n_selected(const SelState &st, uint32_t kpmax) {
  return min(min(st.kq, st.ncand), kpmax);
}

__device__ __forceinline__ uint32_t hslot(uint32_t c, uint32_t mask) {
  return (c * 0x9E3779B1u) >> 7 & mask;
}

// Alg. 7, result: best k of query b's re-ranked candidates, sorted best
// first.  One block; the re-ranked keys may come from the same launch (read
// from L2).
__device__ void final_one(Batch bt, uint32_t b, uint32_t kpmax, uint32_t k, uint32_t q0,
                          uint32_t *out_ids, float *out_scores) {
  __shared__ uint64_t sk[SINN_MAX_K];
  __shared__ uint32_t s_cnt;
  const uint32_t kq = n_selected(bt.sel[b], kpmax);
  const uint32_t r = min(k, kq);
  const uint64_t *ek = bt.ekeys + (uint64_t)b * kpmax;
  uint64_t pre = 0, msk = 0;
  if (kq > 0) block_select_u64(ek, kq, r, &pre, &msk);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kq; i += blockDim.x) {
    const uint64_t key = __ldcg(ek + i);
    if ((key & msk) >= pre) {
      const uint32_t p = atomicAdd(&s_cnt, 1u);
      if (p < SINN_MAX_K) sk[p] = key;
    }
  }
  // bitonic sort, descending, of the r keys padded to the next power of two
  uint32_t P = 1;
  while (P < r) P <<= 1;
  for (uint32_t i = r + threadIdx.x; i < P; i += blockDim.x) sk[i] = 0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const uint64_t x = sk[i], y = sk[j];
          if (desc ? (x < y) : (x > y)) {
            sk[i] = y;
            sk[j] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  const uint64_t ob = (uint64_t)(q0 + b) * k;
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    if (i < r) {
      out_ids[ob + i] = ~(uint32_t)sk[i];
      out_scores[ob + i] = sinn_key2f((uint32_t)(sk[i] >> 32));
    } else {
      out_ids[ob + i] = 0xFFFFFFFFu;
      out_scores[ob + i] = -INFINITY;
    }
  }
}

// One block's share of query b's re-rank (Alg. 7: exact <q, x_v> from the
// vector store for each candidate v).  The query lives in a shared-memory
// hash table; one warp per candidate, lanes over the vector's entries,
// fixed-order reduction.
__device__ void rerank_part(const RerankArgs &a, Batch bt, uint32_t b, uint32_t kq,
                            uint32_t *hs) {
  const uint32_t nt = bt.nt[b];
  uint32_t tsz = 64;
  while (tsz < 2 * nt) tsz <<= 1;
  const uint32_t mask = tsz - 1;
  uint32_t *hk = hs;
  float *hv = (float *)(hs + tsz);
  for (uint32_t i = threadIdx.x; i < tsz; i += blockDim.x) hk[i] = 0xFFFFFFFFu;
  __syncthreads();
  const QTerm *terms = bt.terms + (uint64_t)b * a.qmax;
  for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) {
    uint32_t c = terms[i].j, s = hslot(c, mask);
    while (atomicCAS(&hk[s], 0xFFFFFFFFu, c) != 0xFFFFFFFFu) s = (s + 1) & mask;
    hv[s] = terms[i].v;
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t *cand = bt.cand + (uint64_t)b * a.kpmax;
  uint64_t *ek = bt.ekeys + (uint64_t)b * a.kpmax;
  for (uint32_t c = blockIdx.x * nw + wid; c < kq; c += gridDim.x * nw) {
    const uint32_t id = ~(uint32_t)cand[c];
    if (id >= a.cap) {  // cannot happen: selected keys carry live ids
      if (lane == 0) {
        ek[c] = 0ull;
        atomicOr(a.err, SINN_DERR_INTERNAL);
      }
      continue;
    }
    const uint64_t fo = a.fwd_off[id];
    uint32_t nz = a.fwd_nnz[id];
    if (!SINN_IN_BOUNDS(fo + nz <= a.fwd_cap, a.err)) nz = 0;
    float s = 0.0f;
    // four entries per lane in flight, then their look-ups; the sum keeps
    // the entries' order within each lane
    for (uint32_t e0 = 0; e0 < nz; e0 += 128) {
      uint2 pr[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t e = e0 + u * 32 + lane;
        pr[u] = e < nz ? __ldg(a.fwd + fo + e) : make_uint2(0xFFFFFFFFu, 0u);
      }
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        if (pr[u].x == 0xFFFFFFFFu) continue;
        uint32_t h = hslot(pr[u].x, mask);
        float qv = 0.0f;
        while (true) {
          const uint32_t kk = hk[h];
          if (kk == pr[u].x) {
            qv = hv[h];
            break;
          }
          if (kk == 0xFFFFFFFFu) break;
          h = (h + 1) & mask;
        }
        s = fmaf(qv, __uint_as_float(pr[u].y), s);
      }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) ek[c] = ((uint64_t)sinn_f2key(s + 0.0f) << 32) | (uint32_t)~id;
  }
}

// Alg. 7, re-rank; with fuse set, the last of a query's blocks to finish
// then takes its best k (otherwise k_final does).
__global__ void k_rerank(RerankArgs a, Batch bt, uint32_t fuse, uint32_t k, uint32_t q0,
                         uint32_t *out_ids, float *out_scores) {
  extern __shared__ uint32_t hs[];
  const uint32_t b = blockIdx.y;
  const SelState st = bt.sel[b];
  const uint32_t kq = n_selected(st, a.kpmax);
  if (blockIdx.x == 0 && threadIdx.x == 0 && st.ncand != st.kq) atomicOr(a.err, SINN_DERR_INTERNAL);
  if (blockIdx.x * (blockDim.x >> 5) < kq) rerank_part(a, bt, b, kq, hs);
  if (fuse && last_block(bt.rdone + b, gridDim.x))
    final_one(bt, b, a.kpmax, k, q0, out_ids, out_scores);
}

// Alg. 7, result, for a launch of many queries: one block per query.
__global__ void __launch_bounds__(1024) k_final(Batch bt, uint32_t kpmax, uint32_t k, uint32_t q0,
                                                uint32_t *out_ids, float *out_scores) {
  final_one(bt, blockIdx.x, kpmax, k, q0, out_ids, out_scores);
}

__global__ void k_keys_to_scores(const uint32_t *__restrict__ keys, uint64_t cnt, float *out) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  uint32_t k = keys[i];
  out[i] = k ? sinn_key2f(k) : -INFINITY;
}

__global__ void k_cand_out(Batch bt, uint32_t kpmax, uint32_t q0, uint32_t *out_ids,
                           float *out_scores, uint32_t *out_count) {
  const uint32_t b = blockIdx.x;
  const uint32_t kq = n_selected(bt.sel[b], kpmax);
  const uint64_t *cand = bt.cand + (uint64_t)b * kpmax;
  const uint64_t ob = (uint64_t)(q0 + b) * kpmax;
  for (uint32_t i = threadIdx.x; i < kpmax; i += blockDim.x) {
    if (i < kq) {
      out_ids[ob + i] = ~(uint32_t)cand[i];
      out_scores[ob + i] = sinn_key2f((uint32_t)(cand[i] >> 32));
    } else {
      out_ids[ob + i] = 0xFFFFFFFFu;
      out_scores[ob + i] = -INFINITY;
    }
  }
  if (threadIdx.x == 0) out_count[q0 + b] = kq;
}

// ------------------------------------------------------------- host driver
struct Layout {
  size_t terms, nt, keys, hist, sel, cand, bnd, ekeys, elist, ctr, flagged, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Layout layout_for(const sinn_index *ix, uint32_t B, uint32_t kpmax) {
  Layout L;
  size_t o = 0;
  L.terms = o;   o = align256(o + (size_t)B * ix->max_qnnz * sizeof(QTerm));
  L.nt = o;      o = align256(o + (size_t)B * 8);
  L.keys = o;    o = align256(o + (size_t)B * ix->cap * 4);
  L.hist = o;    o = align256(o + (size_t)B * (4096 + 4096 + 256) * 4);
  L.sel = o;     o = align256(o + (size_t)B * sizeof(SelState));
  L.cand = o;    o = align256(o + (size_t)B * kpmax * 8);
  L.bnd = o;     o = align256(o + (size_t)B * kBoundCap * 8);
  L.ekeys = o;   o = align256(o + (size_t)B * kpmax * 8);
  L.elist = o;   o = align256(o + (size_t)B * kEmitCap * 8);
  L.ctr = o;     o = align256(o + ((size_t)4 * B + 8) * 4);
  L.flagged = o; o = align256(o + (size_t)B * 4);
  L.total = o;
  return L;
}

Batch views(void *base, const Layout &L, uint32_t B) {
  char *p = (char *)base;
  Batch bt;
  bt.terms = (QTerm *)(p + L.terms);
  bt.nt = (uint32_t *)(p + L.nt);
  bt.ns = bt.nt + B;
  bt.keys = (uint32_t *)(p + L.keys);
  bt.hist0 = (uint32_t *)(p + L.hist);
  bt.hist1 = bt.hist0 + (size_t)B * 4096;
  bt.hist2 = bt.hist1 + (size_t)B * 4096;
  bt.sel = (SelState *)(p + L.sel);
  bt.cand = (uint64_t *)(p + L.cand);
  bt.bnd = (uint64_t *)(p + L.bnd);
  bt.ekeys = (uint64_t *)(p + L.ekeys);
  bt.elist = (uint64_t *)(p + L.elist);
  bt.ecnt = (uint32_t *)(p + L.ctr);
  bt.bound = bt.ecnt + B;
  bt.tdone = bt.bound + B;
  bt.rdone = bt.tdone + B;
  bt.nflag = bt.rdone + B;  // then the persistent kernel's 8-byte counter
  bt.tick = bt.nflag + 4;
  bt.flagged = (uint32_t *)(p + L.flagged);
  return bt;
}

enum class Stage { kScores, kCandidates, kFull };

struct SearchReq {
  const uint64_t *q_indptr;
  const uint32_t *q_idx;
  const float *q_val;
  uint32_t n_q, k, kp, kp_min, kp_max;
  const uint32_t *kp_arr;
  const uint64_t *budget_arr;  // per-query Alg. 6 budgets (0 = none), or null: the index's
  uint32_t seq = SINN_SEQ_LATEST;  // snapshot: the ids the search counts
  uint32_t *out_ids;
  float *out_scores;
  uint32_t *out_count;
  float *out_dense;
  Stage stage;
};

size_t score_smem(const sinn_index *ix) {
  // two T-float accumulators, the T-bit touched marks and list, the staged
  // terms (start, count, chunk prefix + 1, weight, coordinate, h bins)
  return (size_t)ix->T * 8 + (size_t)ix->T / 8 + (size_t)kTouchCap * 2 +
         (size_t)kTermBatch * (4 + 4 + 4 + 4 + 4 + 4 * ix->h) + 4;
}

// The dynamic shared memory a kernel may use, raised only when a launch
// needs more than was set before (the attribute belongs to the function and
// persists; setting it on every search costs a driver call per kernel).
cudaError_t set_dyn_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> done;
  std::lock_guard<std::mutex> g(mu);
  auto it = done.find(fn);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
  if (e == cudaSuccess) done[fn] = bytes;
  return e;
}

// Multiprocessor count of a device, asked once.
int sm_count(int dev) {
  static std::mutex mu;
  static std::unordered_map<int, int> sms;
  std::lock_guard<std::mutex> g(mu);
  auto it = sms.find(dev);
  if (it != sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 1;
  }
  sms[dev] = n;
  return n;
}

// Scratch supplied by the caller instead of the index's own (grown) buffer.
struct FixedScratch {
  void *base;
  size_t bytes;
};

int run_search(sinn_index *ix, const SearchReq &r, cudaStream_t s,
               const FixedScratch *fixed = nullptr) {
  const uint32_t kpmax = r.kp_max;
  const Layout one = layout_for(ix, 1, kpmax);
  const uint64_t budget = fixed ? fixed->bytes : ix->scratch_budget;
  uint64_t B = std::max<uint64_t>(1, budget / one.total);
  B = std::min<uint64_t>(B, r.n_q);
  B = std::min<uint64_t>(B, 65535);
  if (ix->tune.max_batch) B = std::min<uint64_t>(B, ix->tune.max_batch);
  Layout L = layout_for(ix, (uint32_t)B, kpmax);
  if (fixed && L.total > fixed->bytes) return SINN_ESCRATCH;
  if (!fixed) {
    int st = sinn_ensure_scratch(ix, L.total);
    if (st) return st;
  }
  Batch bt = views(fixed ? fixed->base : ix->scratch, L, (uint32_t)B);
  const size_t ssm = score_smem(ix);
  const ScoreKernels sk = score_kernels(ix->h, ix->sk_elem == 2, ix->tune.array_walk != 0);
  CK(set_dyn_smem((const void *)sk.emit, ssm));
  CK(set_dyn_smem((const void *)sk.persistent, ssm));
  ScoreArgs sa;
  sa.tile_dir = ix->d_tile_dir;
  sa.tile_post = ix->d_tile_post;
  sa.sel = ix->d_tile_sel;
  // without sequence-numbered mutations every live id counts for every search
  sa.recent = ix->snapshots ? ix->d_recent : nullptr;
  sa.born = ix->d_born;
  sa.died = ix->d_died;
  sa.seq = r.seq;
  sa.U = ix->d_U;
  sa.L = ix->d_L;
  sa.pi = ix->d_pi;
  sa.live = ix->d_live;
  sa.cap = ix->cap;
  sa.n = ix->n;
  sa.h = ix->h;
  sa.T = ix->T;
  sa.log2T = ix->log2T;
  sa.qmax = ix->max_qnnz;
  // ids at or above next_id were never assigned: search covers the tiles
  // below it (the keys keep the capacity as their row stride)
  const uint64_t used_tiles =
      std::max<uint64_t>(1, std::min<uint64_t>(ix->cap / ix->T, (ix->next_id + ix->T - 1) / ix->T));
  const uint64_t span = r.stage == Stage::kScores ? ix->cap : used_tiles * ix->T;
  sa.tiles = (uint32_t)(span / ix->T);
  sa.bound_every = ix->tune.bound_every;
  sa.tpb = ix->tune.tiles_per_block;
  sa.err = ix->d_err;
  sa.m = ix->m;
  RerankArgs ra;
  ra.fwd_off = ix->d_fwd_off;
  ra.fwd_nnz = ix->d_fwd_nnz;
  ra.fwd = ix->d_fwd;
  ra.qmax = ix->max_qnnz;
  ra.kpmax = kpmax;
  ra.cap = ix->cap;
  ra.fwd_cap = ix->fwd_cap;
  ra.err = ix->d_err;
  uint32_t tsz = 64;
  while (tsz < 2 * ix->max_qnnz) tsz <<= 1;
  const int sms = sm_count(ix->device);
  const uint32_t fb_score_blocks = (uint32_t)std::max(1, sms) * ix->tune.dense_blocks_per_sm;
  for (uint32_t q0 = 0; q0 < r.n_q; q0 += (uint32_t)B) {
    const uint32_t nb = (uint32_t)std::min<uint64_t>(B, r.n_q - q0);
    // a launch of a few queries ends its scoring, histogram and compaction
    // kernels with the next step's pick or refine (the last block to finish
    // makes it for every query, one after another) instead of launching it
    const uint32_t fuse = nb <= kFuseQueries ? 1u : 0u;
    {
      SinnPhase ph(ix, s, 0);
      ix->launches++;
      // launches of fewer than emit_min_batch queries (and the dense score
      // output) score every query densely
      const bool dense = r.stage == Stage::kScores || nb < ix->tune.emit_min_batch;
      k_qprep<<<nb, 128, (size_t)ix->max_qnnz * 8, s>>>(r.q_indptr, r.q_idx, r.q_val, q0,
                                                         ix->n, ix->max_qnnz, r.kp, r.kp_arr,
                                                         r.kp_min, r.kp_max, ix->d_live_count, bt,
                                                         ix->d_coord_len, ix->budget,
                                                         r.budget_arr,
                                                         (ix->flags & SINN_FLAG_NONNEG) ? 1 : 0,
                                                         dense ? 1 : 0, ix->d_err);
      CK(cudaGetLastError());
    }
    if (r.stage == Stage::kScores) {  // dense keys for every query
      ix->launches += 1 + nb;
      sk.dense<<<fb_score_blocks, kLoneThreads, 0, s>>>(sa, bt, 0u);
      for (uint32_t b = 0; b < nb; ++b) {
        uint64_t cnt = ix->cap;
        k_keys_to_scores<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
            bt.keys + (uint64_t)b * ix->cap, cnt, r.out_dense + (uint64_t)(q0 + b) * ix->cap);
      }
      CK(cudaGetLastError());
      continue;
    }
    const bool dense_all = nb < ix->tune.emit_min_batch;
    {
      SinnPhase ph(ix, s, 1);
      if (dense_all) {
        ix->launches++;
        sk.dense<<<fb_score_blocks, kLoneThreads, 0, s>>>(sa, bt, fuse);
      } else {
        ix->launches++;
        if (ix->tune.persistent_blocks_per_sm) {
          // 8-byte aligned work counter after the nflag word
          unsigned long long *next =
              (unsigned long long *)(((uintptr_t)(bt.nflag + 1) + 7) & ~(uintptr_t)7);
          sk.persistent<<<(unsigned)sms * ix->tune.persistent_blocks_per_sm, kScoreThreads, ssm,
                          s>>>(sa, bt, nb, next);
        } else {
          sk.emit<<<dim3(nb, (sa.tiles + sa.tpb - 1) / sa.tpb), kScoreThreads, ssm, s>>>(sa, bt);
        }
      }
      CK(cudaGetLastError());
    }
    {
      SinnPhase ph(ix, s, 2);
      if (!dense_all) {
        // list path, then the dense fallback for flagged queries (no work
        // when none is flagged)
        ix->launches += 4;
        k_pick_list<<<nb, 128, 0, s>>>(bt);
        k_compact_list<<<nb, 512, 0, s>>>(bt, kpmax);
        k_fb_reset<<<std::min(nb, kFbBlocks), 256, 0, s>>>(bt);
        sk.dense<<<fb_score_blocks, kLoneThreads, 0, s>>>(sa, bt, fuse);
      }
      // grids no larger than the work (the flagged queries are at most nb)
      const uint32_t gq = std::min(nb, kFbBlocks);
      const uint32_t gc = (uint32_t)std::min<uint64_t>(
          (uint64_t)nb * ((span + kChunk - 1) / kChunk), (uint64_t)fb_score_blocks * 2);
      // the finer levels only run for a boundary bin too large to buffer
      // (massive ties): a smaller grid keeps the common no-op launch cheap
      const uint32_t gh = std::min<uint32_t>(gc, nb * 64);
      if (fuse) {
        ix->launches += 2;
        k_hist_level<<<gh, 256, 0, s>>>(bt, ix->cap, span, 1, 2u);
        k_compact<<<gc, 256, 0, s>>>(bt, ix->cap, span, kpmax, nb);
      } else {
        ix->launches += 7;
        k_pick<<<gq, 128, 0, s>>>(bt, 0);
        k_hist_level<<<gh, 256, 0, s>>>(bt, ix->cap, span, 1, 0u);
        k_pick<<<gq, 128, 0, s>>>(bt, 1);
        k_hist_level<<<gh, 256, 0, s>>>(bt, ix->cap, span, 2, 0u);
        k_pick<<<gq, 128, 0, s>>>(bt, 2);
        k_compact<<<gc, 256, 0, s>>>(bt, ix->cap, span, kpmax, 0u);
        k_refine<<<nb, 512, 0, s>>>(bt, ix->cap, span, kpmax);
      }
      CK(cudaGetLastError());
    }
    if (r.stage == Stage::kCandidates) {
      ix->launches++;
      k_cand_out<<<nb, 256, 0, s>>>(bt, kpmax, q0, r.out_ids, r.out_scores, r.out_count);
      CK(cudaGetLastError());
      continue;
    }
    {
      SinnPhase ph(ix, s, 3);
      ix->launches += fuse ? 1 : 2;
      // blocks per query: the tuning's count, or (0) about 64 candidates each
      // (for a launch of few queries, enough blocks to fill the GPU, down to
      // one warp per candidate)
      uint32_t rb = ix->tune.rerank_blocks ? ix->tune.rerank_blocks : (kpmax + 63) / 64;
      if (!ix->tune.rerank_blocks)
        rb = std::max<uint32_t>(rb, ((uint32_t)sms * 8 + nb - 1) / nb);
      k_rerank<<<dim3(std::min<uint32_t>(rb, (kpmax + 7) / 8), nb), 256,
                 (size_t)tsz * 8, s>>>(ra, bt, fuse, r.k, q0, r.out_ids, r.out_scores);
      if (!fuse) k_final<<<nb, 1024, 0, s>>>(bt, kpmax, r.k, q0, r.out_ids, r.out_scores);
      CK(cudaGetLastError());
    }
  }
  return SINN_OK;
}

int check_query_args(sinn_index *ix, const uint64_t *ip, uint32_t n_q) {
  if (!ix) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!ip) return SINN_EINVAL;
  return SINN_OK;
}

}  // namespace

extern "C" int sinn_search(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                           const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                           uint32_t *out_ids, float *out_scores, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k == 0 || k > SINN_MAX_K || k_prime < k) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = k;
  r.kp = k_prime;
  r.kp_min = k;
  r.kp_max = k_prime;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.stage = Stage::kFull;
  return run_search(ix, r, (cudaStream_t)stream);
}

extern "C" int sinn_search_kp(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                              const float *q_values, uint32_t n_q, uint32_t k,
                              const uint32_t *k_prime, uint32_t k_prime_max, uint32_t *out_ids,
                              float *out_scores, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k == 0 || k > SINN_MAX_K || k_prime_max < k || !k_prime) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = k;
  r.kp = k_prime_max;
  r.kp_arr = k_prime;
  r.kp_min = k;
  r.kp_max = k_prime_max;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.stage = Stage::kFull;
  return run_search(ix, r, (cudaStream_t)stream);
}

extern "C" int sinn_scores(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                           const float *q_values, uint32_t n_q, float *out, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (n_q == 0) return SINN_OK;
  if (!out) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = 1;
  r.kp = 1;
  r.kp_min = 1;
  r.kp_max = 1;
  r.out_dense = out;
  r.stage = Stage::kScores;
  return run_search(ix, r, (cudaStream_t)stream);
}

extern "C" int sinn_candidates(sinn_index *ix, const uint64_t *q_indptr,
                               const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                               uint32_t k_prime, uint32_t *out_ids, float *out_scores,
                               uint32_t *out_count, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k_prime == 0) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores || !out_count) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = 1;
  r.kp = k_prime;
  r.kp_min = 1;
  r.kp_max = k_prime;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.out_count = out_count;
  r.stage = Stage::kCandidates;
  return run_search(ix, r, (cudaStream_t)stream);
}

extern "C" int sinn_search_host(sinn_index *ix, const uint64_t *q_indptr,
                                const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                                uint32_t k, uint32_t k_prime, uint32_t *out_ids,
                                float *out_scores, void *stream) {
  if (!ix) return SINN_EINVAL;
  if (k == 0 || k > SINN_MAX_K || k_prime < k) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!q_indptr || !out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t nnz = q_indptr[n_q] - q_indptr[0];
  if (nnz && (!q_indices || !q_values)) return SINN_EINVAL;
  const size_t b_ip = align256(((size_t)n_q + 1) * 8), b_ix = align256(nnz * 4),
               b_v = align256(nnz * 4), b_oi = align256((size_t)n_q * k * 4),
               b_os = align256((size_t)n_q * k * 4);
  const size_t need = b_ip + b_ix + b_v + b_oi + b_os;
  if (need > ix->hstage_size) {
    if (ix->hstage) {
      CK(cudaStreamSynchronize(s));
      CK(cudaFree(ix->hstage));
      ix->hstage = nullptr;
      ix->hstage_size = 0;
    }
    CK(sinn_dev_malloc((void **)&ix->hstage, need));
    ix->hstage_size = need;
  }
  char *p = (char *)ix->hstage;
  uint64_t *d_ip = (uint64_t *)p;
  uint32_t *d_ix = (uint32_t *)(p + b_ip);
  float *d_v = (float *)(p + b_ip + b_ix);
  uint32_t *d_oi = (uint32_t *)(p + b_ip + b_ix + b_v);
  float *d_os = (float *)(p + b_ip + b_ix + b_v + b_oi);
  // row pointers rebased to zero on the device side
  std::vector<uint64_t> ip(q_indptr, q_indptr + n_q + 1);
  const uint64_t base = ip[0];
  bool rebase = base != 0;
  if (rebase)
    for (auto &x : ip) x -= base;
  CK(cudaMemcpyAsync(d_ip, rebase ? ip.data() : q_indptr, ((size_t)n_q + 1) * 8,
                     cudaMemcpyHostToDevice, s));
  if (nnz) {
    CK(cudaMemcpyAsync(d_ix, q_indices + base, nnz * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_v, q_values + base, nnz * 4, cudaMemcpyHostToDevice, s));
  }
  int st = sinn_search(ix, d_ip, d_ix, d_v, n_q, k, k_prime, d_oi, d_os, stream);
  if (st) return st;
  CK(cudaMemcpyAsync(out_ids, d_oi, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(out_scores, d_os, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, s));
  return sinn_sync(ix, stream);
}

// ------------------------------------------------ search without allocation
// Some callers cannot allocate device memory while they search: code running
// inside a memory budget that was fixed up front, or a host whose allocator
// must not be entered on its serving path (an allocation may synchronise the
// device or fail under fragmentation).  sinn_search_noalloc serves them: its
// scratch is this file-scope device array, which exists on every device that
// loads the library for as long as the library stays loaded, so the call
// itself never allocates.  All calls on one device share it.
constexpr size_t kNoAllocBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
// Last address found per device, read only while a stream is being captured.
std::atomic<void *> g_noalloc_ptr[kMaxDevices];

// The array's device address in the current context.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// the device current -- on every call, which keeps it right after a context
// is torn down and made again (cudaDeviceReset) in the same process; the
// lookup allocates nothing.  While the stream is being captured no lookup is
// made (it could load the module) and the address an earlier call found on
// this device is used: the first call on a device must come before any
// capture.  Concurrent first calls from several host threads each look the
// address up and store the same value.
int noalloc_scratch(int dev, cudaStream_t s, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return SINN_ECUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return SINN_ECUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) {
    void *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) return SINN_ECUDA;
    *out = p;
    return SINN_OK;
  }
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    (void)cudaGetLastError();
    return SINN_ECUDA;
  }
  g_noalloc_ptr[dev].store(p, std::memory_order_release);
  *out = p;
  return SINN_OK;
}
}  // namespace

extern "C" int sinn_search_noalloc(sinn_index *ix, const uint64_t *q_indptr,
                                   const uint32_t *q_indices, const float *q_values,
                                   uint32_t n_q, uint32_t k, uint32_t k_prime, uint32_t *out_ids,
                                   float *out_scores, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k == 0 || k > SINN_MAX_K || k_prime < k) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  FixedScratch fx;
  if ((st = noalloc_scratch(ix->device, (cudaStream_t)stream, &fx.base))) return st;
  fx.bytes = kNoAllocBytes;
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = k;
  r.kp = k_prime;
  r.kp_min = k;
  r.kp_max = k_prime;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.stage = Stage::kFull;
  // phase timing records events; keep this call free of any resource creation
  const bool tm = ix->tm_on;
  ix->tm_on = false;
  st = run_search(ix, r, (cudaStream_t)stream, &fx);
  ix->tm_on = tm;
  return st;
}

// ------------------------------------------------------- search contexts
// A context owns the scratch of one in-flight search, so several searches of
// the same index can run at once on different streams (the index itself is
// only read by a search).  Mutations must still be ordered against them.
struct sinn_ctx {
  sinn_index *ix = nullptr;
  void *scratch = nullptr;
  size_t bytes = 0;
  uint32_t seq = SINN_SEQ_LATEST;  // snapshot its searches see
};

extern "C" int sinn_ctx_set_snapshot(sinn_ctx *c, uint32_t seq) {
  if (!c || seq > SINN_SEQ_LATEST) return SINN_EINVAL;
  c->seq = seq;
  return SINN_OK;
}

extern "C" int sinn_ctx_create(sinn_index *ix, uint64_t scratch_bytes, sinn_ctx **out) {
  if (!ix || !out || scratch_bytes < (1u << 20)) return SINN_EINVAL;
  *out = nullptr;
  sinn_ctx *c = new (std::nothrow) sinn_ctx();
  if (!c) return SINN_ENOMEM;
  SinnDevice dev_guard_(ix->device);
  if (sinn_dev_malloc((void **)&c->scratch, scratch_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    delete c;
    return SINN_ENOMEM;
  }
  c->ix = ix;
  c->bytes = scratch_bytes;
  *out = c;
  return SINN_OK;
}

extern "C" int sinn_ctx_destroy(sinn_ctx *c) {
  if (!c) return SINN_OK;
  SinnDevice dev_guard_(c->ix->device);
  cudaDeviceSynchronize();
  cudaFree(c->scratch);
  delete c;
  return SINN_OK;
}

extern "C" uint64_t sinn_ctx_query_bytes(sinn_ctx *c, uint32_t k_prime_max) {
  if (!c || k_prime_max == 0) return 0;
  return layout_for(c->ix, 1, k_prime_max).total;
}

// sinn_search / sinn_search_kp on a context's scratch (k_prime may be NULL:
// fixed k' = k_prime_max).
extern "C" int sinn_search_ctx(sinn_ctx *c, const uint64_t *q_indptr, const uint32_t *q_indices,
                               const float *q_values, uint32_t n_q, uint32_t k,
                               const uint32_t *k_prime, uint32_t k_prime_max, uint32_t *out_ids,
                               float *out_scores, void *stream) {
  if (!c) return SINN_EINVAL;
  sinn_index *ix = c->ix;
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k == 0 || k > SINN_MAX_K || k_prime_max < k) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  FixedScratch fx{c->scratch, c->bytes};
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = k;
  r.kp = k_prime_max;
  r.kp_arr = k_prime;
  r.kp_min = k;
  r.kp_max = k_prime_max;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.stage = Stage::kFull;
  r.seq = c->seq;
  return run_search(ix, r, (cudaStream_t)stream, &fx);
}

// ------------------------------------------- per-query k' and Alg. 6 budget
// One search with a per-query k' (or k_prime_max for all) and a per-query
// anytime budget (or the index's), on a context's scratch or the index's own.
int sinn_search_ext(sinn_index *ix, sinn_ctx *c, const uint64_t *q_indptr,
                    const uint32_t *q_indices, const float *q_values, uint32_t n_q, uint32_t k,
                    const uint32_t *k_prime, uint32_t k_prime_max, const uint64_t *budget,
                    uint32_t *out_ids, float *out_scores, cudaStream_t s) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k == 0 || k > SINN_MAX_K || k_prime_max < k) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = k;
  r.kp = k_prime_max;
  r.kp_arr = k_prime;
  r.kp_min = k;
  r.kp_max = k_prime_max;
  r.budget_arr = budget;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.stage = Stage::kFull;
  if (!c) return run_search(ix, r, s);
  r.seq = c->seq;
  FixedScratch fx{c->scratch, c->bytes};
  return run_search(ix, r, s, &fx);
}

extern "C" int sinn_search_kpb(sinn_index *ix, const uint64_t *q_indptr,
                               const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                               uint32_t k, const uint32_t *k_prime, uint32_t k_prime_max,
                               const uint64_t *budget, uint32_t *out_ids, float *out_scores,
                               void *stream) {
  return sinn_search_ext(ix, nullptr, q_indptr, q_indices, q_values, n_q, k, k_prime,
                         k_prime_max, budget, out_ids, out_scores, (cudaStream_t)stream);
}

extern "C" int sinn_candidates_kpb(sinn_index *ix, const uint64_t *q_indptr,
                                   const uint32_t *q_indices, const float *q_values,
                                   uint32_t n_q, uint32_t k_prime, const uint64_t *budget,
                                   uint32_t *out_ids, float *out_scores, uint32_t *out_count,
                                   void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (k_prime == 0) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!out_ids || !out_scores || !out_count) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  SearchReq r{};
  r.q_indptr = q_indptr;
  r.q_idx = q_indices;
  r.q_val = q_values;
  r.n_q = n_q;
  r.k = 1;
  r.kp = k_prime;
  r.kp_min = 1;
  r.kp_max = k_prime;
  r.budget_arr = budget;
  r.out_ids = out_ids;
  r.out_scores = out_scores;
  r.out_count = out_count;
  r.stage = Stage::kCandidates;
  return run_search(ix, r, (cudaStream_t)stream);
}

namespace {
// P_q = sum over the query's non-zeros of |I[j]| (live postings): what Alg. 6
// visits with no budget.  One warp per query; a malformed row gives 0.
__global__ void k_query_postings(const uint64_t *__restrict__ ip, const uint32_t *__restrict__ idx,
                                 const float *__restrict__ val, uint32_t n_q, uint32_t n,
                                 const uint32_t *__restrict__ coord_len, uint64_t *out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= n_q) return;
  const uint64_t s = ip[q], e = ip[q + 1];
  uint64_t sum = 0;
  bool bad = e < s;
  for (uint64_t p = s + lane; !bad && p < e; p += 32) {
    const uint32_t j = idx[p];
    const float v = val[p];
    if (j >= n || !isfinite(v) || (p > s && idx[p - 1] >= j)) bad = true;
    else if (v != 0.0f) sum += coord_len[j];
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
  bad = __any_sync(0xFFFFFFFFu, bad);
  if (lane == 0) out[q] = bad ? 0ull : sum;
}
}  // namespace

extern "C" int sinn_query_postings(sinn_index *ix, const uint64_t *q_indptr,
                                   const uint32_t *q_indices, const float *q_values,
                                   uint32_t n_q, uint64_t *out, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (n_q == 0) return SINN_OK;
  if (!out) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  ix->launches++;
  k_query_postings<<<(unsigned)(((uint64_t)n_q * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      q_indptr, q_indices, q_values, n_q, ix->n, ix->d_coord_len, out);
  CK(cudaGetLastError());
  return SINN_OK;
}

// ------------------------------------------------------------------ tuning

static bool tuning_ok(const sinn_tuning &t) {
  return t.bound_every >= 1 && t.bound_every <= 64 && t.emit_min_batch >= 1 &&
         t.emit_min_batch <= 65535 && t.rerank_blocks <= 1024 &&
         t.dense_blocks_per_sm >= 1 && t.dense_blocks_per_sm <= 32 && t.tiles_per_block >= 1 &&
         t.tiles_per_block <= 64 && t.persistent_blocks_per_sm <= 4 && t.array_walk <= 1;
}

extern "C" int sinn_get_tuning(sinn_index *ix, sinn_tuning *out) {
  if (!ix || !out) return SINN_EINVAL;
  *out = ix->tune;
  return SINN_OK;
}

extern "C" int sinn_set_tuning(sinn_index *ix, const sinn_tuning *t) {
  if (!ix || !t || !tuning_ok(*t)) return SINN_EINVAL;
  ix->tune = *t;
  ix->shape_version++;
  return SINN_OK;
}

// Coordinate descent: each field in turn takes the candidate value with the
// shortest search time (a change must gain 1% to be kept).
extern "C" int sinn_autotune(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                             const float *q_values, uint32_t n_q, uint32_t k, uint32_t k_prime,
                             uint32_t reps, sinn_tuning *out, void *stream) {
  int st = check_query_args(ix, q_indptr, n_q);
  if (st) return st;
  if (n_q == 0 || reps == 0 || reps > 8 || k == 0 || k > SINN_MAX_K || k_prime < k)
    return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *ids = nullptr;
  float *sc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(sinn_dev_malloc((void **)&ids, (size_t)n_q * k * 4));
  CK(sinn_dev_malloc((void **)&sc, (size_t)n_q * k * 4));
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto run = [&](float *ms) -> int {
    float best = 3.4e38f;
    for (uint32_t r = 0; r < reps; ++r) {
      CK(cudaEventRecord(e0, s));
      int q = sinn_search(ix, q_indptr, q_indices, q_values, n_q, k, k_prime, ids, sc, stream);
      if (q) return q;
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float t = 0.0f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    *ms = best;
    return SINN_OK;
  };
  const sinn_tuning start = ix->tune;
  float best_ms = 0.0f;
  st = run(&best_ms);  // warm-up: scratch grows here
  if (!st) st = run(&best_ms);
  sinn_tuning best = ix->tune;
  struct Field {
    uint32_t sinn_tuning::*f;
    uint32_t n, vals[6];
  };
  const Field fields[] = {
      {&sinn_tuning::max_batch, 6, {0, 256, 512, 1024, 2048, 4096}},
      {&sinn_tuning::array_walk, 2, {0, 1}},
      {&sinn_tuning::tiles_per_block, 6, {1, 2, 4, 8, 16, 32}},
      {&sinn_tuning::persistent_blocks_per_sm, 3, {0, 2, 4}},
      {&sinn_tuning::bound_every, 6, {1, 2, 4, 8, 16, 32}},
      {&sinn_tuning::rerank_blocks, 6, {0, 4, 16, 64, 256, 1024}},
      {&sinn_tuning::dense_blocks_per_sm, 6, {1, 2, 4, 8, 16, 32}},
      {&sinn_tuning::emit_min_batch, 6, {4, 8, 16, 32, 64, 128}},
  };
  for (const Field &fd : fields) {
    if (st) break;
    for (uint32_t vi = 0; vi < fd.n; ++vi) {
      const uint32_t v = fd.vals[vi];
      if (v == best.*fd.f) continue;
      if (fd.f == &sinn_tuning::max_batch && v >= n_q) continue;  // same as unlimited
      ix->tune = best;
      ix->tune.*fd.f = v;
      float ms = 0.0f;
      if ((st = run(&ms))) break;
      if (ms < 0.99f * best_ms) {
        best_ms = ms;
        best = ix->tune;
      }
    }
  }
  ix->tune = st ? start : best;
  ix->shape_version++;
  if (out) *out = ix->tune;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(sc);
  return st;
}

// ------------------------------------------------------------------ anytime

extern "C" int sinn_set_budget(sinn_index *ix, uint64_t postings) {
  if (!ix) return SINN_EINVAL;
  if (ix->budget != postings) ix->shape_version++;  // recorded searches bake it in
  ix->budget = postings;
  return SINN_OK;
}

extern "C" uint64_t sinn_get_budget(sinn_index *ix) { return ix ? ix->budget : 0; }
