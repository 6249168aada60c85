// Index construction and maintenance on the GPU: Alg. 5 (indexing) and
// Sec. 4.3 (deletion) of SINNAMON, plus the C ABI calls that own the index.
//
// Layout (device):
//   d_pi        n*h uint32      pi_o(j) at [j*h + o]
//   d_U, d_L    m x cap fp32    row k holds bin k of every id slot (row-major,
//                               as the paper stores the sketch matrix)
//   d_live      cap bits        live ids
//   d_fwd*      vector store    (coordinate, value) pairs per id
//   d_tile_dir  2 x tiles x n   per tile t, copy v and coordinate j (at
//               uint2           (2t + v) n + j), the container of the
//                               postings of I[j] with ids in
//                               [t*T, (t+1)*T): {start, count} in 16-bit words
//                               of that copy's storage.  Searches read the
//                               copy d_tile_sel[t]; a rebuild writes the
//                               other one and then selects it.  count >= T/8:
//                               a bitmap of T bits (bit d = local id d; a
//                               deleted posting's bit is cleared); otherwise a
//                               sorted array of count 16-bit local ids (bit 15
//                               marks a deleted posting).  Arrays fill the
//                               storage from the front, bitmaps from the back
//                               (T/16-word aligned).  This is the array/bitmap
//                               split of the Roaring containers the paper
//                               uses for its lists, per tile of T ids; the
//                               threshold is set where scoring a bitmap by
//                               sweeping all T ids (4 ids per 16-byte load)
//                               costs no more per posting than walking an
//                               array.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "sinn_internal.cuh"

#define CK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return sinn_check_cuda(e_); \
  } while (0)

int sinn_check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SINN_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SINN_ENOMEM : SINN_ECUDA;
}

// Allocation fault injection: >= 0 counts down the allocations still to
// succeed before one fails (then it is off again); -1 is off.
static std::atomic<int64_t> g_fail_alloc{-1};

static bool alloc_should_fail() {
  int64_t v = g_fail_alloc.load();
  while (v >= 0) {
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

cudaError_t sinn_dev_malloc(void **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t sinn_dev_malloc_async(void **p, size_t bytes, cudaStream_t s) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, s);
}

cudaError_t sinn_host_malloc(void **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

extern "C" int sinn_debug_fail_alloc(int64_t after) {
  g_fail_alloc.store(after < 0 ? -1 : after);
  return SINN_OK;
}

// SplitMix64's output function (Steele, Lea, Flood, OOPSLA 2014).
static uint64_t lib_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// -------------------------------------------------------------- kernels

// Insert-batch validation: coordinates < n and strictly increasing per row,
// values finite.  One warp per row.
__global__ void k_validate_csr(const uint64_t *__restrict__ indptr,
                               const uint32_t *__restrict__ indices,
                               const float *__restrict__ values, uint32_t rows, uint32_t n,
                               uint32_t *err, uint32_t bit, int nonneg) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= rows) return;
  const uint64_t s = indptr[w], e = indptr[w + 1];
  bool bad = false;
  for (uint64_t p = s + lane; p < e; p += 32) {
    uint32_t c = indices[p];
    float v = values[p];
    if (c >= n || !isfinite(v) || (nonneg && v < 0.0f)) bad = true;
    if (p > s && indices[p - 1] >= c) bad = true;
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(err, bit);
}

// Copy each row into the vector store at its assigned offset.  One warp per row.
__global__ void k_fwd_write(const uint64_t *__restrict__ indptr,
                            const uint32_t *__restrict__ indices,
                            const float *__restrict__ values, uint32_t rows,
                            const uint32_t *__restrict__ ids, const uint64_t *__restrict__ offs,
                            uint2 *__restrict__ fwd, uint64_t *__restrict__ fwd_off,
                            uint32_t *__restrict__ fwd_nnz, uint32_t *__restrict__ coord_len,
                            uint64_t fwd_cap, uint64_t cap, uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= rows) return;
  const uint64_t s = indptr[w], e = indptr[w + 1], o = offs[w];
  if (!SINN_IN_BOUNDS(o + (e - s) <= fwd_cap && ids[w] < cap, err)) return;
  for (uint64_t p = s + lane; p < e; p += 32) {
    const float v = values[p];
    fwd[o + (p - s)] = make_uint2(indices[p], __float_as_uint(v));
    if (v != 0.0f) atomicAdd(&coord_len[indices[p]], 1u);  // |I[j]| grows
  }
  if (lane == 0) {
    fwd_off[ids[w]] = o;
    fwd_nnz[ids[w]] = (uint32_t)(e - s);
  }
}

// Alg. 5, sketch: u[k] = max and l[k] = min of x_i[j] over the non-zeros j
// with pi_o(j) = k for some o; empty bins -inf / +inf.  Max and min are taken
// on order-preserving integer keys, so the stored bins are the input floats
// bit for bit.  A block sketches G rows in shared memory, then writes the
// columns out row by row of the sketch (consecutive ids -> coalesced stores).
__global__ void k_sketch(const uint64_t *__restrict__ indptr, const uint32_t *__restrict__ indices,
                         const float *__restrict__ values, uint32_t rows,
                         const uint32_t *__restrict__ ids, const uint32_t *__restrict__ pi,
                         uint32_t m, uint32_t h, uint64_t cap, uint32_t G, void *__restrict__ U,
                         void *__restrict__ L, int bf16, uint32_t *err) {
  extern __shared__ uint32_t sk[];
  uint32_t *uk = sk;          // G*m
  uint32_t *lk = sk + G * m;  // G*m
  const uint32_t r0 = blockIdx.x * G;
  const uint32_t g_cnt = min(G, rows - r0);
  const uint32_t NEG_INF_KEY = 0x007FFFFFu;  // key of -inf
  const uint32_t POS_INF_KEY = 0xFF800000u;  // key of +inf
  for (uint32_t t = threadIdx.x; t < g_cnt * m; t += blockDim.x) {
    uk[t] = NEG_INF_KEY;
    lk[t] = POS_INF_KEY;
  }
  __syncthreads();
  for (uint32_t g = 0; g < g_cnt; ++g) {
    const uint64_t s = indptr[r0 + g], e = indptr[r0 + g + 1];
    for (uint64_t p = s + threadIdx.x; p < e; p += blockDim.x) {
      float v = values[p];
      if (v == 0.0f) continue;  // not a non-zero
      uint32_t key = sinn_f2key(v);
      uint32_t c = indices[p];
      for (uint32_t o = 0; o < h; ++o) {
        uint32_t k = pi[(uint64_t)c * h + o];
        if (!SINN_IN_BOUNDS(k < m, err)) continue;
        atomicMax(&uk[g * m + k], key);
        atomicMin(&lk[g * m + k], key);
      }
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < g_cnt * m; t += blockDim.x) {
    uint32_t k = t / g_cnt, g = t % g_cnt;
    uint64_t id = ids[r0 + g];
    if (!SINN_IN_BOUNDS(id < cap, err)) continue;
    const uint64_t at = (uint64_t)k * cap + id;
    const float u = sinn_key2f(uk[g * m + k]), l = sinn_key2f(lk[g * m + k]);
    if (bf16) {  // bounds stay bounds: U rounds up, L rounds down
      ((uint16_t *)U)[at] = sinn_bf16_dir(u, true);
      if (L) ((uint16_t *)L)[at] = sinn_bf16_dir(l, false);
    } else {
      ((float *)U)[at] = u;
      if (L) ((float *)L)[at] = l;  // no L plane: SINNAMON+
    }
  }
}

__global__ void k_set_live(const uint32_t *__restrict__ ids, uint32_t cnt, uint32_t *live,
                           int set) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  uint32_t id = ids[i];
  if (set) atomicOr(&live[id >> 5], 1u << (id & 31));
  else atomicAnd(&live[id >> 5], ~(1u << (id & 31)));
}

// Block-wide exclusive scan of one value per thread; *total receives the
// sum.  Every thread of the block must call it; part holds 33 words.
__device__ uint32_t block_scan_value(uint32_t x, uint32_t *part, uint32_t *total) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = x;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= (uint32_t)d) inc += y;
  }
  if (lane == 31) part[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t v = lane < nw ? part[lane] : 0u;
    uint32_t z = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, d);
      if (lane >= (uint32_t)d) z += y;
    }
    if (lane < nw) part[lane] = z - v;
    if (lane == 31) part[32] = z;
  }
  __syncthreads();
  const uint32_t r = part[wid] + inc - x;
  *total = part[32];
  __syncthreads();
  return r;
}

// Rebuild of the postings of a group of tiles into each tile's other copy,
// merging the copy searches read now with the batch's new vectors (Alg. 5:
// the new vectors' postings appended to their lists; Sec. 4.3: tombstones
// dropped).  Container (tile, j) of the new copy holds the current
// container's postings that are not tombstones plus the tile-local ids of
// the new vectors with a non-zero at j: a bitmap of T bits when that makes
// at least T >> SINN_BITMAP_SHIFT postings, else an array of 16-bit local
// ids in ascending order.  Only the new vectors are read from the store.
//   count_old  one warp per (tile, 32 coordinates): each lane counts the live
//              postings of its coordinate's array; the warp counts each
//              bitmap together
//   count_new  one warp per new vector: its postings per coordinate
//   plan       one block per tile: container kinds, array starts by a scan in
//              coordinate order, bitmap slots from the back of the storage in
//              the same order; the directory is written and the bitmaps zeroed
//   merge_old  as count_old: the live postings into the new containers, in
//              order (array to array or bitmap, bitmap to bitmap or array)
//   merge_new  one warp per new vector: bitmap bits, or array slots after the
//              old postings by atomic cursors; each array so extended is
//              listed once
//   sort       one warp per listed array: ascending order again
struct RebuildArgs {
  const uint32_t *tiles;      // tile per group entry (ascending)
  const uint32_t *ver;        // copy (0 or 1) of the tile the entry rebuilds into
  uint16_t *const *new_post;  // storage per group entry
  const uint64_t *post_cap;   // storage size per entry (16-bit words, multiple of T/16)
  uint32_t *cnt;              // n per entry: counts, then array cursors
  uint32_t *out_len;          // postings per entry
  const uint2 *dir;           // every tile's directories (copy v of tile t at (2t + v) n)
  uint16_t *const *post;      // every tile's storage (copy v of tile t at 2t + v)
  const uint32_t *new_ids;    // the new vectors of the group's tiles
  uint32_t *dirty;            // nb * n bits: arrays the new vectors extend
  uint32_t *dlist;            // those arrays, as entry * n + coordinate
  uint32_t *dcount;           // their number
  uint32_t dcap;              // room in dlist
  uint32_t n_new, nb, n, T, log2T;
  uint32_t *err;              // device error word (bounds-check builds)
};

// Group entry of tile t (entries are ascending), or -1.
__device__ __forceinline__ int rb_entry(const RebuildArgs &a, uint32_t t) {
  uint32_t lo = 0, hi = a.nb;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.tiles[mid] < t) lo = mid + 1;
    else hi = mid;
  }
  return (lo < a.nb && a.tiles[lo] == t) ? (int)lo : -1;
}

__global__ void __launch_bounds__(256) k_rb_count_old(RebuildArgs a) {
  const uint32_t lane = threadIdx.x & 31, BMIN = a.T >> SINN_BITMAP_SHIFT, W128 = a.T >> 7;
  const uint32_t nch = (a.n + 31) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
       w < (uint64_t)a.nb * nch; w += nwarps) {
    const uint32_t i = (uint32_t)(w / nch), c = (uint32_t)(w % nch) * 32 + lane;
    const uint32_t t = a.tiles[i], ov = 1u - a.ver[i];  // the copy searches read now
    const uint2 de = c < a.n ? a.dir[((uint64_t)t * 2 + ov) * a.n + c] : make_uint2(0u, 0u);
    const uint16_t *po = a.post[(uint64_t)t * 2 + ov];
    uint32_t live = 0;
    if (de.y > 0 && de.y < BMIN)
      for (uint32_t e = 0; e < de.y; ++e) live += (po[de.x + e] & SINN_TOMB) ? 0u : 1u;
    uint32_t bms = __ballot_sync(0xFFFFFFFFu, de.y >= BMIN);
    while (bms) {  // deletes clear bitmap bits: the live postings are the set bits
      const uint32_t src = __ffs(bms) - 1;
      bms &= bms - 1;
      const uint4 *wd = (const uint4 *)(po + __shfl_sync(0xFFFFFFFFu, de.x, src));
      uint32_t pc = 0;
      for (uint32_t k = lane; k < W128; k += 32) {
        const uint4 q = wd[k];
        pc += __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);
      }
      for (int o = 16; o > 0; o >>= 1) pc += __shfl_xor_sync(0xFFFFFFFFu, pc, o);
      if (lane == src) live = pc;
    }
    if (c < a.n) a.cnt[(uint64_t)i * a.n + c] = live;
  }
}

__global__ void __launch_bounds__(256)
    k_rb_count_new(RebuildArgs a, const uint64_t *__restrict__ fwd_off,
                   const uint32_t *__restrict__ fwd_nnz, const uint2 *__restrict__ fwd) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < a.n_new;
       w += nwarps) {
    const uint32_t id = a.new_ids[w];
    const int i = rb_entry(a, id >> a.log2T);
    if (!SINN_IN_BOUNDS(i >= 0, a.err)) continue;
    const uint64_t fo = fwd_off[id];
    const uint32_t nz = fwd_nnz[id];
    uint32_t *cnt = a.cnt + (uint64_t)i * a.n;
    for (uint32_t e = lane; e < nz; e += 32) {
      const uint2 pr = fwd[fo + e];
      if ((pr.y & 0x7FFFFFFFu) != 0u) atomicAdd(&cnt[pr.x], 1u);
    }
  }
}

__global__ void __launch_bounds__(1024)
    k_rb_plan(RebuildArgs a, uint2 *__restrict__ tile_dir, uint16_t **tile_post, uint32_t *err) {
  __shared__ uint32_t part[33];
  const uint32_t i = blockIdx.x, t = a.tiles[i], n = a.n, v = a.ver[i];
  const uint32_t W16 = a.T >> 4, BMIN = a.T >> SINN_BITMAP_SHIFT;
  uint16_t *post = a.new_post[i];
  const uint64_t cap16 = a.post_cap[i];
  uint32_t *cnt = a.cnt + (uint64_t)i * n;
  uint2 *dir = tile_dir + ((uint64_t)t * 2 + v) * n;
  // each thread owns a contiguous run of coordinates
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t c0 = min(n, threadIdx.x * per), c1 = min(n, c0 + per);
  uint32_t sa = 0, sb = 0, st = 0;
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t v = cnt[c];
    st += v;
    if (v >= BMIN) sb++;
    else sa += v;
  }
  uint32_t tot_a, tot_b, tot_t;
  uint32_t run_a = block_scan_value(sa, part, &tot_a);
  uint32_t run_b = block_scan_value(sb, part, &tot_b);
  (void)block_scan_value(st, part, &tot_t);
  if ((uint64_t)tot_a + (uint64_t)tot_b * W16 > cap16) {  // cannot happen if sized right
    if (threadIdx.x == 0) atomicOr(err, SINN_DERR_INTERNAL);
    return;
  }
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t v = cnt[c];
    if (v == 0) {
      dir[c] = make_uint2(0u, 0u);
    } else if (v >= BMIN) {
      dir[c] = make_uint2((uint32_t)(cap16 - (uint64_t)(run_b + 1) * W16), v);
      run_b++;
    } else {
      dir[c] = make_uint2(run_a, v);
      cnt[c] = run_a;
      run_a += v;
    }
  }
  uint32_t *z = (uint32_t *)(post + (cap16 - (uint64_t)tot_b * W16));
  const uint64_t words = (uint64_t)tot_b * (W16 / 2);
  for (uint64_t k = threadIdx.x; k < words; k += blockDim.x) z[k] = 0u;
  if (threadIdx.x == 0) {
    a.out_len[i] = tot_t;
    tile_post[(uint64_t)t * 2 + v] = post;
  }
}

__global__ void __launch_bounds__(256) k_rb_merge_old(RebuildArgs a) {
  const uint32_t lane = threadIdx.x & 31, BMIN = a.T >> SINN_BITMAP_SHIFT;
  const uint32_t W128 = a.T >> 7, W32 = a.T >> 5, wpl = W32 >> 5;
  const uint32_t nch = (a.n + 31) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
       w < (uint64_t)a.nb * nch; w += nwarps) {
    const uint32_t i = (uint32_t)(w / nch), c = (uint32_t)(w % nch) * 32 + lane;
    const uint32_t t = a.tiles[i], v = a.ver[i], ov = 1u - v;
    const bool in = c < a.n;
    const uint2 de = in ? a.dir[((uint64_t)t * 2 + ov) * a.n + c] : make_uint2(0u, 0u);
    const uint2 dn = in ? a.dir[((uint64_t)t * 2 + v) * a.n + c] : make_uint2(0u, 0u);
    const uint16_t *po = a.post[(uint64_t)t * 2 + ov];
    uint16_t *pn = a.new_post[i];
    const uint64_t pcap = a.post_cap[i];
    (void)pcap;  // read by the bounds checks only
    uint32_t *cur = a.cnt + (uint64_t)i * a.n + c;
    const bool old_bm = de.y >= BMIN, new_bm = dn.y >= BMIN;
    // an old array: its lane alone, in order
    if (de.y > 0 && !old_bm) {
      if (new_bm) {
        uint32_t *bm = (uint32_t *)(pn + dn.x);
        if (SINN_IN_BOUNDS((uint64_t)dn.x + a.T / 16 <= pcap, a.err))
          for (uint32_t e = 0; e < de.y; ++e) {
            const uint32_t x = po[de.x + e];
            if (!(x & SINN_TOMB)) bm[(x & 0x7FFFu) >> 5] |= 1u << (x & 31u);
          }
      } else {
        uint32_t at = *cur;
        for (uint32_t e = 0; e < de.y; ++e) {
          const uint32_t x = po[de.x + e];
          if (x & SINN_TOMB) continue;
          if (SINN_IN_BOUNDS(at < dn.x + dn.y && at < pcap, a.err)) pn[at] = (uint16_t)x;
          ++at;
        }
        *cur = at;
      }
    }
    // an old bitmap: the warp together (an array it turns into starts at
    // its coordinate's cursor)
    const uint32_t cur0 = (old_bm && dn.y > 0 && !new_bm) ? *cur : 0u;
    uint32_t bms = __ballot_sync(0xFFFFFFFFu, old_bm);
    while (bms) {
      const uint32_t src = __ffs(bms) - 1;
      bms &= bms - 1;
      const uint32_t ox = __shfl_sync(0xFFFFFFFFu, de.x, src);
      const uint32_t nx = __shfl_sync(0xFFFFFFFFu, dn.x, src);
      const uint32_t ny = __shfl_sync(0xFFFFFFFFu, dn.y, src);
      if (ny >= BMIN) {  // bitmap to bitmap: the words as they are
        if (!SINN_IN_BOUNDS((uint64_t)nx + a.T / 16 <= pcap, a.err)) continue;
        const uint4 *src4 = (const uint4 *)(po + ox);
        uint4 *dst4 = (uint4 *)(pn + nx);
        for (uint32_t k = lane; k < W128; k += 32) dst4[k] = src4[k];
      } else if (ny > 0) {  // bitmap to array (deletes took it below the threshold)
        const uint32_t *wd = (const uint32_t *)(po + ox);
        uint32_t mine = 0;
        for (uint32_t j = 0; j < wpl; ++j) mine += __popc(wd[lane * wpl + j]);
        uint32_t inc = mine;
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
          if (lane >= (uint32_t)d) inc += y;
        }
        const uint32_t base = __shfl_sync(0xFFFFFFFFu, cur0, src);
        uint32_t at = base + inc - mine;
        for (uint32_t j = 0; j < wpl; ++j) {
          uint32_t bits = wd[lane * wpl + j];
          while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (SINN_IN_BOUNDS(at < nx + ny && at < pcap, a.err))
              pn[at] = (uint16_t)(((lane * wpl + j) << 5) + b);
            ++at;
          }
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
        if (lane == src) *cur = base + total;
      }
    }
  }
}

__global__ void __launch_bounds__(256)
    k_rb_merge_new(RebuildArgs a, const uint64_t *__restrict__ fwd_off,
                   const uint32_t *__restrict__ fwd_nnz, const uint2 *__restrict__ fwd) {
  const uint32_t lane = threadIdx.x & 31, BMIN = a.T >> SINN_BITMAP_SHIFT;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < a.n_new;
       w += nwarps) {
    const uint32_t id = a.new_ids[w];
    const int i = rb_entry(a, id >> a.log2T);
    if (i < 0) continue;  // reported by the count
    const uint32_t t = a.tiles[i], d = id & (a.T - 1);
    const uint2 *dir = a.dir + ((uint64_t)t * 2 + a.ver[i]) * a.n;
    uint16_t *pn = a.new_post[i];
    uint32_t *cur = a.cnt + (uint64_t)i * a.n;
    const uint64_t fo = fwd_off[id];
    const uint32_t nz = fwd_nnz[id];
    for (uint32_t e = lane; e < nz; e += 32) {
      const uint2 pr = fwd[fo + e];
      if ((pr.y & 0x7FFFFFFFu) == 0u) continue;
      const uint2 dn = dir[pr.x];
      if (dn.y >= BMIN) {
        if (SINN_IN_BOUNDS((uint64_t)dn.x + a.T / 16 <= a.post_cap[i], a.err))
          atomicOr((uint32_t *)(pn + dn.x) + (d >> 5), 1u << (d & 31));
      } else {
        const uint32_t at = atomicAdd(&cur[pr.x], 1u);
        if (SINN_IN_BOUNDS(at < dn.x + dn.y && at < a.post_cap[i], a.err)) pn[at] = (uint16_t)d;
        // the array's order is restored by the sort (listed once)
        const uint32_t key = (uint32_t)i * a.n + pr.x, bit = 1u << (key & 31);
        if (!(atomicOr(&a.dirty[key >> 5], bit) & bit)) {
          const uint32_t p = atomicAdd(a.dcount, 1u);
          if (SINN_IN_BOUNDS(p < a.dcap, a.err)) a.dlist[p] = key;
        }
      }
    }
  }
}

// Sorts the listed array containers of the rebuilt tiles: up to 32 postings
// in registers (a bitonic network), more through a T-bit bitmap in shared
// memory.  Dynamic shared memory: T/32 words per warp.
__global__ void __launch_bounds__(256) k_rb_sort(RebuildArgs a) {
  extern __shared__ uint32_t sm[];
  const uint32_t lane = threadIdx.x & 31, words = a.T >> 5, wpl = words >> 5;
  uint32_t *bm = sm + (threadIdx.x >> 5) * words;
  const uint32_t nl = min(*a.dcount, a.dcap);
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < nl; w += nwarps) {
    const uint32_t key = a.dlist[w], i = key / a.n, c = key % a.n;
    const uint2 de = a.dir[((uint64_t)a.tiles[i] * 2 + a.ver[i]) * a.n + c];
    if (de.y < 2) continue;  // warp-uniform
    uint16_t *seg = a.new_post[i] + de.x;
    if (de.y <= 32) {
      // one posting per lane, sorted by a bitonic network over the warp
      // (empty lanes hold 0xFFFF, above every local id)
      uint32_t d = lane < de.y ? (seg[lane] & 0x7FFFu) : 0xFFFFu;
      for (uint32_t k = 2; k <= 32; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, d, j);
          const bool up = (lane & k) == 0, lower = (lane & j) == 0;
          d = (lower == up) ? min(d, o) : max(d, o);
        }
      }
      if (lane < de.y) seg[lane] = (uint16_t)d;
      continue;
    }
    for (uint32_t j = lane; j < words; j += 32) bm[j] = 0u;
    __syncwarp();
    for (uint32_t e = lane; e < de.y; e += 32) {
      const uint32_t d = seg[e] & 0x7FFFu;
      atomicOr(&bm[d >> 5], 1u << (d & 31));
    }
    __syncwarp();
    const uint32_t w0 = lane * wpl;
    uint32_t mine = 0;
    for (uint32_t j = 0; j < wpl; ++j) mine += __popc(bm[w0 + j]);
    uint32_t inc = mine;
    for (int s = 1; s < 32; s <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, s);
      if (lane >= (uint32_t)s) inc += y;
    }
    uint32_t pos = inc - mine;
    for (uint32_t j = 0; j < wpl; ++j) {
      uint32_t bits = bm[w0 + j];
      while (bits) {
        const uint32_t b = __ffs(bits) - 1;
        seg[pos++] = (uint16_t)(((w0 + j) << 5) + b);
        bits &= bits - 1;
      }
    }
    __syncwarp();
  }
}

// After a group's rebuild kernels: searches from now on read the copies just
// written (the copies they read before stay as they were).
__global__ void k_rb_flip(RebuildArgs a, uint32_t *tile_sel) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nb) tile_sel[a.tiles[i]] = a.ver[i];
}

// Sec. 4.3 deletion: for each deleted id, remove it from every list it is in
// -- clear its bit in a bitmap container, or set the tombstone bit of its
// posting in an array container (binary search: arrays are sorted) -- then
// clear its live bit.  One warp per id.
__global__ void k_tombstone(const uint32_t *__restrict__ ids, uint32_t cnt,
                            const uint64_t *__restrict__ fwd_off,
                            const uint32_t *__restrict__ fwd_nnz, const uint2 *__restrict__ fwd,
                            const uint2 *__restrict__ tile_dir, uint16_t *const *tile_post,
                            const uint32_t *__restrict__ tile_sel, uint32_t *live, uint32_t n,
                            uint32_t log2T, uint32_t *tomb_count,
                            uint32_t *coord_len, uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= cnt) return;
  const uint32_t id = ids[w];
  const uint32_t t = id >> log2T;
  const uint32_t BMIN = (1u << log2T) >> SINN_BITMAP_SHIFT;
  const uint32_t d = id & ((1u << log2T) - 1u);
  const uint32_t v = tile_sel[t];  // the copy searches read
  const uint2 *dir = tile_dir + ((uint64_t)t * 2 + v) * n;
  uint16_t *post = tile_post[(uint64_t)t * 2 + v];
  const uint64_t fo = fwd_off[id];
  const uint32_t nz = fwd_nnz[id];
  uint32_t marked = 0;
  for (uint32_t e = lane; e < nz; e += 32) {
    const uint2 pr = fwd[fo + e];
    if ((pr.y & 0x7FFFFFFFu) == 0u) continue;
    const uint2 de = dir[pr.x];
    bool ok = false;
    if (de.y >= BMIN) {
      uint32_t *bm = (uint32_t *)(post + de.x);
      const uint32_t bit = 1u << (d & 31);
      ok = (atomicAnd(bm + (d >> 5), ~bit) & bit) != 0u;
    } else {
      uint32_t lo = de.x, hi = de.x + de.y;
      while (lo < hi) {  // first position with local id >= d
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint32_t)(post[mid] & 0x7FFFu) < d) lo = mid + 1;
        else hi = mid;
      }
      if (lo < de.x + de.y && (uint32_t)(post[lo] & 0x7FFFu) == d && !(post[lo] & SINN_TOMB)) {
        post[lo] = (uint16_t)(post[lo] | SINN_TOMB);
        ok = true;
      }
    }
    if (ok) {
      marked++;
      atomicSub(&coord_len[pr.x], 1u);  // |I[j]| shrinks
    }
    else atomicOr(err, SINN_DERR_INTERNAL);
  }
  for (int s = 16; s > 0; s >>= 1) marked += __shfl_xor_sync(0xFFFFFFFFu, marked, s);
  if (lane == 0) {
    atomicAnd(&live[id >> 5], ~(1u << (id & 31)));
    tomb_count[w] = marked;
  }
}

__global__ void k_gather_columns(const uint32_t *__restrict__ ids, uint32_t cnt,
                                 const void *__restrict__ U, const void *__restrict__ L,
                                 uint32_t m, uint64_t cap, int bf16, float *u_out,
                                 float *l_out) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= (uint64_t)cnt * m) return;
  uint32_t r = (uint32_t)(i / m), k = (uint32_t)(i % m);
  uint64_t id = ids[r];
  if (id >= cap) {  // no storage for this id: report NaN
    u_out[i] = __int_as_float(0x7FC00000);
    if (l_out) l_out[i] = __int_as_float(0x7FC00000);
    return;
  }
  const uint64_t at = (uint64_t)k * cap + id;
  u_out[i] = bf16 ? sinn_bf16_f(((const uint16_t *)U)[at]) : ((const float *)U)[at];
  if (l_out) l_out[i] = bf16 ? sinn_bf16_f(((const uint16_t *)L)[at]) : ((const float *)L)[at];
}

__global__ void k_store_u64(uint64_t *dst, uint64_t v) { *dst = v; }

// arr[ids[i]] = v for i < cnt (birth and death sequence numbers).
__global__ void k_fill_ids(const uint32_t *__restrict__ ids, uint32_t cnt, uint32_t *arr,
                           uint32_t v) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) arr[ids[i]] = v;
}

// ------------------------------------------------------------- host side

static cudaEvent_t tm_event(sinn_index *ix) {
  if (!ix->tm_pool.empty()) {
    cudaEvent_t e = ix->tm_pool.back();
    ix->tm_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Inside a stream capture an event must be recorded as an external event to
// become a node that records at every replay.
static void tm_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

// Phases as NVTX ranges, so that a profiler's timeline shows them by name.
static const char *const kPhaseNames[SINN_PHASES] = {"sinn query prep", "sinn score",
                                                     "sinn select", "sinn rerank",
                                                     "sinn insert", "sinn delete"};

SinnPhase::SinnPhase(sinn_index *ix_, cudaStream_t s_, int ph) : ix(ix_), s(s_), phase(ph) {
  nvtxRangePushA(ph >= 0 && ph < SINN_PHASES ? kPhaseNames[ph] : "sinn");
  if (ix->tm_on) {
    a = tm_event(ix);
    tm_record(a, s);
  }
}

SinnPhase::~SinnPhase() {
  if (a) {
    cudaEvent_t b = tm_event(ix);
    tm_record(b, s);
    ix->tm_spans.push_back({phase, a, b});
  }
  nvtxRangePop();
}

extern "C" int sinn_timing_start(sinn_index *ix) {
  if (!ix) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  for (auto &sp : ix->tm_spans) {
    ix->tm_pool.push_back(sp.a);
    ix->tm_pool.push_back(sp.b);
  }
  ix->tm_spans.clear();
  for (int p = 0; p < SINN_PHASES; ++p) {
    ix->tm_acc_ms[p] = 0.0;
    ix->tm_acc_spans[p] = 0;
  }
  ix->launches = 0;
  ix->tm_on = true;
  return SINN_OK;
}

extern "C" int sinn_timing_stop(sinn_index *ix, sinn_timing_t *out) {
  if (!ix || !out) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  memset(out, 0, sizeof(*out));
  ix->tm_on = false;
  for (auto &sp : ix->tm_spans) {
    CK(cudaEventSynchronize(sp.b));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, sp.a, sp.b));
    if (sp.phase >= 0 && sp.phase < SINN_PHASES) {
      out->ms[sp.phase] += ms;
      out->spans[sp.phase] += 1;
    }
    ix->tm_pool.push_back(sp.a);
    ix->tm_pool.push_back(sp.b);
  }
  ix->tm_spans.clear();
  for (int p = 0; p < SINN_PHASES; ++p) {
    out->ms[p] += ix->tm_acc_ms[p];
    out->spans[p] += ix->tm_acc_spans[p];
  }
  out->launches = ix->launches;
  return SINN_OK;
}

static void release(sinn_index *ix) {
  if (!ix) return;
  SinnDevice dev_guard_(ix->device);
  cudaDeviceSynchronize();
  for (uint16_t *p : ix->tile_post)
    if (p) cudaFree(p);
  for (auto &sp : ix->tm_spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (cudaEvent_t e : ix->tm_pool) cudaEventDestroy(e);
  cudaFree(ix->d_pi);
  cudaFree(ix->d_U);
  cudaFree(ix->d_L);
  cudaFree(ix->d_live);
  cudaFree(ix->d_fwd_off);
  cudaFree(ix->d_fwd_nnz);
  cudaFree(ix->d_fwd);
  cudaFree(ix->d_tile_dir);
  cudaFree(ix->d_tile_post);
  cudaFree(ix->d_tile_sel);
  cudaFree(ix->d_born);
  cudaFree(ix->d_died);
  cudaFree(ix->d_recent);
  cudaFree(ix->d_err);
  cudaFree(ix->d_live_count);
  cudaFree(ix->d_coord_len);
  cudaFree(ix->scratch);
  cudaFree(ix->iscratch);
  cudaFree(ix->hstage);
  if (ix->pinned) cudaFreeHost(ix->pinned);
  delete ix;
}

int sinn_ensure_scratch(sinn_index *ix, size_t bytes) {
  if (bytes <= ix->scratch_size) return SINN_OK;
  if (ix->scratch) {
    CK(cudaDeviceSynchronize());
    CK(cudaFree(ix->scratch));
    ix->scratch = nullptr;
    ix->scratch_size = 0;
  }
  CK(sinn_dev_malloc((void **)&ix->scratch, bytes));
  ix->scratch_size = bytes;
  return SINN_OK;
}

static int ensure_iscratch(sinn_index *ix, size_t bytes) {
  if (bytes <= ix->iscratch_size) return SINN_OK;
  if (ix->iscratch) {
    CK(cudaDeviceSynchronize());
    CK(cudaFree(ix->iscratch));
    ix->iscratch = nullptr;
    ix->iscratch_size = 0;
  }
  size_t b = std::max(bytes, ix->iscratch_size * 3 / 2);
  CK(sinn_dev_malloc((void **)&ix->iscratch, b));
  ix->iscratch_size = b;
  return SINN_OK;
}

int sinn_ensure_pinned(sinn_index *ix, size_t bytes) {
  if (bytes <= ix->pinned_size) return SINN_OK;
  if (ix->pinned) {
    CK(cudaDeviceSynchronize());
    CK(cudaFreeHost(ix->pinned));
    ix->pinned = nullptr;
    ix->pinned_size = 0;
  }
  size_t b = std::max(bytes, ix->pinned_size * 3 / 2);
  CK(sinn_host_malloc((void **)&ix->pinned, b));
  ix->pinned_size = b;
  return SINN_OK;
}

template <typename T>
static int realloc_copy(T **p, uint64_t old_elems, uint64_t new_elems, bool zero_rest) {
  T *q = nullptr;
  CK(sinn_dev_malloc((void **)&q, new_elems * sizeof(T)));
  if (zero_rest) CK(cudaMemset(q, 0, new_elems * sizeof(T)));
  if (*p && old_elems) CK(cudaMemcpy(q, *p, old_elems * sizeof(T), cudaMemcpyDeviceToDevice));
  if (*p) CK(cudaFree(*p));
  *p = q;
  return SINN_OK;
}

// Grow id capacity to hold ids < need (rounded up to whole tiles).  Every new
// array is allocated before any is filled: if one allocation fails, the
// others are freed and the index is left as it was (SINN_ENOMEM).
static int grow_capacity(sinn_index *ix, uint64_t need) {
  if (need <= ix->cap) return SINN_OK;
  uint64_t nc = std::max<uint64_t>(ix->cap * 2, need);
  nc = (nc + ix->T - 1) / ix->T * ix->T;
  const uint64_t max_cap = 65535ull * ix->T;  // tiles index the second grid dimension
  if (need > max_cap) return SINN_ENOMEM;
  nc = std::min(nc, max_cap);
  const uint64_t ot = ix->cap / ix->T, nt = nc / ix->T;
  const size_t e = ix->sk_elem;
  const int planes = (ix->flags & SINN_FLAG_NONNEG) ? 1 : 2;  // SINNAMON+: U only
  struct Grow {
    void **dst;       // the index's pointer
    size_t elem;      // bytes per element
    uint64_t o, n;    // old and new elements (rows of the sketch planes: per row)
    bool plane;       // a sketch plane: m rows, re-strided
    void *q;
  };
  constexpr int NG = 11;
  Grow g[NG] = {
      {&ix->d_U, e, ix->cap, nc, true, nullptr},
      {&ix->d_L, e, ix->cap, nc, true, nullptr},
      {(void **)&ix->d_live, 4, ix->cap / 32, nc / 32, false, nullptr},
      {(void **)&ix->d_fwd_off, 8, ix->cap, nc, false, nullptr},
      {(void **)&ix->d_fwd_nnz, 4, ix->cap, nc, false, nullptr},
      {(void **)&ix->d_tile_dir, sizeof(uint2), 2 * ot * ix->n, 2 * nt * ix->n, false, nullptr},
      {(void **)&ix->d_tile_post, sizeof(uint16_t *), 2 * ot, 2 * nt, false, nullptr},
      {(void **)&ix->d_tile_sel, 4, ot, nt, false, nullptr},
      {(void **)&ix->d_born, 4, ix->cap, nc, false, nullptr},
      {(void **)&ix->d_died, 4, ix->cap, nc, false, nullptr},
      {(void **)&ix->d_recent, 4, ix->cap / 32, nc / 32, false, nullptr},
  };
  CK(cudaDeviceSynchronize());
  for (int i = 0; i < NG; ++i) {
    if (i == 1 && planes == 1) continue;
    const size_t bytes = g[i].elem * g[i].n * (g[i].plane ? ix->m : 1);
    const cudaError_t err = sinn_dev_malloc(&g[i].q, bytes);
    if (err != cudaSuccess) {
      for (int k = 0; k < i; ++k)
        if (g[k].q) cudaFree(g[k].q);
      return sinn_check_cuda(err);
    }
  }
  for (int i = 0; i < NG; ++i) {
    if (!g[i].q) continue;
    void *old = *g[i].dst;
    if (g[i].plane) {  // copy the m rows into the wider layout
      if (old && g[i].o)
        CK(cudaMemcpy2D(g[i].q, g[i].n * e, old, g[i].o * e, g[i].o * e, ix->m,
                        cudaMemcpyDeviceToDevice));
    } else {
      CK(cudaMemset(g[i].q, 0, g[i].elem * g[i].n));
      if (old && g[i].o) CK(cudaMemcpy(g[i].q, old, g[i].elem * g[i].o, cudaMemcpyDeviceToDevice));
    }
    if (old) CK(cudaFree(old));
    *g[i].dst = g[i].q;
  }
  ix->cap = nc;
  ix->shape_version++;
  ix->live.resize(nc, 0);
  ix->nnz.resize(nc, 0);
  ix->recent.resize(nc, 0);
  ix->tile_post.resize(2 * nt, nullptr);
  ix->tile_post_cap.resize(2 * nt, 0);
  ix->tile_sel.resize(nt, 0);
  ix->tile_flip_seq.resize(nt, 0);
  ix->tile_post_len.resize(nt, 0);
  ix->tile_nnz.resize(nt, 0);
  ix->tile_tombs.resize(nt, 0);
  return SINN_OK;
}

static int grow_store(sinn_index *ix, uint64_t need) {
  if (need <= ix->fwd_cap) return SINN_OK;
  uint64_t nc = std::max<uint64_t>(need, ix->fwd_cap * 2);
  nc = std::max<uint64_t>(nc, 1 << 16);
  CK(cudaDeviceSynchronize());
  int st = realloc_copy(&ix->d_fwd, ix->fwd_used, nc, false);
  if (st) return st;
  ix->fwd_cap = nc;
  ix->shape_version++;
  return SINN_OK;
}

extern "C" int sinn_create_ex(const sinn_config *cfg, sinn_index **out) {
  if (!cfg || !out) return SINN_EINVAL;
  *out = nullptr;
  const uint32_t n = cfg->n, m = cfg->m, h = cfg->h;
  if (n == 0 || m == 0 || h == 0 || h > m || h > SINN_MAX_H || m > 4096) return SINN_EINVAL;
  uint32_t T = cfg->tile_docs ? cfg->tile_docs : 4096;
  if (T < 1024 || T > 16384 || (T & (T - 1))) return SINN_EINVAL;
  if (cfg->flags & ~(SINN_FLAG_NONNEG | SINN_FLAG_BF16_SKETCH)) return SINN_EINVAL;
  if (cfg->table)
    for (uint64_t t = 0; t < (uint64_t)n * h; ++t)
      if (cfg->table[t] >= m) return SINN_EINVAL;
  sinn_index *ix = new (std::nothrow) sinn_index();
  if (!ix) return SINN_ENOMEM;
  cudaGetDevice(&ix->device);
  ix->n = n;
  ix->m = m;
  ix->h = h;
  ix->T = T;
  ix->log2T = 0;
  while ((1u << ix->log2T) < T) ix->log2T++;
  ix->seed = cfg->seed ? cfg->seed : 0x5151ULL;
  ix->flags = cfg->flags;
  ix->sk_elem = (cfg->flags & SINN_FLAG_BF16_SKETCH) ? 2 : 4;
  ix->max_qnnz = cfg->max_query_nnz ? cfg->max_query_nnz : 1024;
  ix->scratch_budget = cfg->scratch_bytes ? cfg->scratch_bytes : (4ULL << 30);
  std::vector<uint32_t> tab((uint64_t)n * h);
  for (uint32_t j = 0; j < n; ++j)
    for (uint32_t o = 0; o < h; ++o) {
      uint64_t t = (uint64_t)j * h + o;
      if (cfg->table) {
        tab[t] = cfg->table[t];
      } else {
        uint64_t x = ix->seed ^ ((uint64_t)(o + 1) * 0x9E3779B97F4A7C15ULL) ^ (uint64_t)j;
        tab[t] = (uint32_t)(lib_mix64(x) % m);
      }
    }
  int st = SINN_OK;
  auto fail = [&](int s) {
    release(ix);
    return s;
  };
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&ix->d_pi, tab.size() * sizeof(uint32_t)))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemcpy(ix->d_pi, tab.data(), tab.size() * sizeof(uint32_t),
                                       cudaMemcpyHostToDevice))))
    return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&ix->d_err, sizeof(uint32_t) * 4))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(ix->d_err, 0, sizeof(uint32_t) * 4)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&ix->d_live_count, sizeof(uint64_t)))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(ix->d_live_count, 0, sizeof(uint64_t))))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&ix->d_coord_len, (size_t)n * 4))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(ix->d_coord_len, 0, (size_t)n * 4)))) return fail(st);
  uint64_t hint = std::max<uint64_t>(cfg->capacity_hint, T);
  if ((st = grow_capacity(ix, hint))) return fail(st);
  *out = ix;
  return SINN_OK;
}

extern "C" int sinn_create(uint32_t n, uint32_t m, uint32_t h, sinn_index **out) {
  sinn_config c;
  memset(&c, 0, sizeof(c));
  c.n = n;
  c.m = m;
  c.h = h;
  return sinn_create_ex(&c, out);
}

extern "C" int sinn_destroy(sinn_index *ix) {
  release(ix);
  return SINN_OK;
}

extern "C" const char *sinn_strerror(int code) {
  switch (code) {
    case SINN_OK: return "ok";
    case SINN_EINVAL: return "invalid argument";
    case SINN_ENOTFOUND: return "id not live";
    case SINN_ENOMEM: return "out of memory";
    case SINN_ECUDA: return "CUDA runtime error";
    case SINN_EDEVICE: return "device-side error";
    case SINN_ESCRATCH: return "request needs more than the fixed no-allocation scratch";
    case SINN_EIO: return "file could not be read or written, or is not a saved index";
    default: return "unknown error";
  }
}

static int read_and_clear_err(sinn_index *ix, cudaStream_t s, uint32_t *bits) {
  CK(cudaMemcpyAsync(bits, ix->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*bits) CK(cudaMemsetAsync(ix->d_err, 0, sizeof(uint32_t), s));
  return SINN_OK;
}

extern "C" int sinn_sync(sinn_index *ix, void *stream) {
  if (!ix) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t bits = 0;
  int st = read_and_clear_err(ix, s, &bits);
  if (st) return st;
  CK(cudaStreamSynchronize(s));
  if (bits & SINN_DERR_DEVICE) return SINN_EDEVICE;
  if (bits) return SINN_EINVAL;
  return SINN_OK;
}

// Storage a tile's rebuild writes into: a new buffer of `cap` 16-bit words,
// or (p == nullptr) the tile's own buffer, rebuilt in place.
struct TileAlloc {
  uint16_t *p;
  uint64_t cap;
};

// Words a tile of `nnz` stored entries needs: containers never need more words
// than postings; bitmaps sit on T/16-word boundaries counted from the end.
static uint64_t tile_words(const sinn_index *ix, uint64_t nnz) {
  const uint64_t W16 = ix->T / 16;
  return std::max<uint64_t>((nnz + W16 - 1) / W16 * W16, W16);
}

// Storage for the rebuild of tile t once it holds `nnz` entries.  A rebuild
// writes the tile's other copy (the one searches do not read): into that
// copy's storage if it is large enough and not over twice too large, else
// into a new buffer with a quarter of room to grow.  Allocation failures
// return SINN_ENOMEM.
static int tile_alloc(sinn_index *ix, uint32_t t, uint64_t nnz, cudaStream_t s, TileAlloc *out) {
  const uint64_t W16 = ix->T / 16, need = tile_words(ix, nnz);
  const uint64_t slot = (uint64_t)t * 2 + (1u - ix->tile_sel[t]);
  if (ix->tile_post[slot] && ix->tile_post_cap[slot] >= need &&
      ix->tile_post_cap[slot] <= 2 * need) {
    *out = {nullptr, ix->tile_post_cap[slot]};  // no search reads that copy
    return SINN_OK;
  }
  const uint64_t cap = need + need / 4 / W16 * W16;
  out->cap = cap;
  out->p = nullptr;
  CK(sinn_dev_malloc_async((void **)&out->p, cap * sizeof(uint16_t), s));
  return SINN_OK;
}

// Device scratch of a rebuild of nb tiles with up to n_new new vectors:
// counts, tiles, target copies, storage pointers, storage sizes, lengths,
// the extended-array marks, their list (room for `dcap`) and count, the new
// vectors' ids.
struct RebuildLayout {
  size_t o_cn, o_tl, o_vr, o_pt, o_pc, o_ln, o_dm, o_dc, o_dl, o_id, bytes;
  uint32_t dcap;
};
static RebuildLayout rebuild_layout(const sinn_index *ix, uint32_t nb, uint64_t n_new,
                                    uint64_t new_entries) {
  RebuildLayout L;
  const uint64_t pairs = (uint64_t)nb * ix->n;
  L.dcap = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(pairs, new_entries));
  L.o_cn = 0;
  L.o_tl = L.o_cn + (size_t)pairs * 4;
  L.o_vr = L.o_tl + (size_t)nb * 4;
  L.o_pt = (L.o_vr + (size_t)nb * 4 + 15) / 16 * 16;
  L.o_pc = L.o_pt + (size_t)nb * 8;
  L.o_ln = L.o_pc + (size_t)nb * 8;
  L.o_dm = (L.o_ln + (size_t)nb * 4 + 15) / 16 * 16;
  L.o_dc = L.o_dm + (size_t)(pairs + 31) / 32 * 4;
  L.o_dl = (L.o_dc + 4 + 15) / 16 * 16;
  L.o_id = L.o_dl + (size_t)L.dcap * 4;
  L.bytes = L.o_id + (size_t)std::max<uint64_t>(n_new, 1) * 4;
  return L;
}

// Tiles rebuilt per group: their per-coordinate counts fit 1 GiB of scratch.
static uint32_t rebuild_group_tiles(const sinn_index *ix, size_t tiles) {
  const uint64_t per = (uint64_t)ix->n * 4;
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (1ull << 30) / per));
}

// Rebuild the postings of a group of tiles (sorted, unique) into each tile's
// other copy -- the current copy's live postings and those of the new
// vectors `new_ids` (host, n_new ids in these tiles, new_entries store
// entries between them) -- with the storage `pre` gives per tile (allocated
// here if pre is null), then make those copies the ones searches read.  A
// search already reading a tile keeps its copy intact; flip_seq is the
// sequence number recorded for the switch.
static int rebuild_group(sinn_index *ix, const uint32_t *tiles, uint32_t nb, cudaStream_t s,
                         const TileAlloc *pre, uint32_t flip_seq, const uint32_t *new_ids,
                         uint32_t n_new, uint64_t new_entries) {
  const RebuildLayout RL = rebuild_layout(ix, nb, n_new, new_entries);
  int st = ensure_iscratch(ix, RL.bytes);
  if (st) return st;
  std::vector<uint16_t *> newp(nb);
  std::vector<uint64_t> pcap(nb);
  std::vector<uint32_t> ver(nb);
  for (uint32_t i = 0; i < nb; ++i) {
    const uint32_t t = tiles[i];
    ver[i] = 1u - ix->tile_sel[t];
    const uint64_t slot = (uint64_t)t * 2 + ver[i];
    TileAlloc ta;
    if (pre) {
      ta = pre[i];
    } else if ((st = tile_alloc(ix, t, ix->tile_nnz[t], s, &ta))) {
      for (uint32_t k = 0; k < i; ++k)
        if (newp[k] != ix->tile_post[(uint64_t)tiles[k] * 2 + ver[k]]) cudaFreeAsync(newp[k], s);
      return st;
    }
    newp[i] = ta.p ? ta.p : ix->tile_post[slot];
    pcap[i] = ta.cap;
  }
  const size_t hb = (size_t)nb * (4 + 4 + 8 + 8) + (size_t)n_new * 4;
  CK(cudaStreamSynchronize(s));  // earlier copies may still read the staging buffer
  if ((st = sinn_ensure_pinned(ix, hb))) return st;
  char *hp = (char *)ix->pinned;
  memcpy(hp, tiles, (size_t)nb * 4);
  memcpy(hp + (size_t)nb * 4, ver.data(), (size_t)nb * 4);
  memcpy(hp + (size_t)nb * 8, newp.data(), (size_t)nb * 8);
  memcpy(hp + (size_t)nb * 16, pcap.data(), (size_t)nb * 8);
  if (n_new) memcpy(hp + (size_t)nb * 24, new_ids, (size_t)n_new * 4);
  char *sp = (char *)ix->iscratch;
  CK(cudaMemcpyAsync(sp + RL.o_tl, hp, (size_t)nb * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sp + RL.o_vr, hp + (size_t)nb * 4, (size_t)nb * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sp + RL.o_pt, hp + (size_t)nb * 8, (size_t)nb * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sp + RL.o_pc, hp + (size_t)nb * 16, (size_t)nb * 8, cudaMemcpyHostToDevice,
                     s));
  if (n_new)
    CK(cudaMemcpyAsync(sp + RL.o_id, hp + (size_t)nb * 24, (size_t)n_new * 4,
                       cudaMemcpyHostToDevice, s));
  // the marks and the list count start at zero (the counts are written whole)
  CK(cudaMemsetAsync(sp + RL.o_dm, 0, RL.o_dl - RL.o_dm, s));
  RebuildArgs a;
  a.tiles = (const uint32_t *)(sp + RL.o_tl);
  a.ver = (const uint32_t *)(sp + RL.o_vr);
  a.new_post = (uint16_t *const *)(sp + RL.o_pt);
  a.post_cap = (const uint64_t *)(sp + RL.o_pc);
  a.cnt = (uint32_t *)(sp + RL.o_cn);
  a.out_len = (uint32_t *)(sp + RL.o_ln);
  a.dir = ix->d_tile_dir;
  a.post = ix->d_tile_post;
  a.new_ids = (const uint32_t *)(sp + RL.o_id);
  a.dirty = (uint32_t *)(sp + RL.o_dm);
  a.dcount = (uint32_t *)(sp + RL.o_dc);
  a.dlist = (uint32_t *)(sp + RL.o_dl);
  a.dcap = RL.dcap;
  a.n_new = n_new;
  a.nb = nb;
  a.n = ix->n;
  a.T = ix->T;
  a.log2T = ix->log2T;
  a.err = ix->d_err;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  // grids: a warp per (tile, 32 coordinates), per new vector, per listed
  // array, each at most 32 blocks per SM
  const uint64_t cap_blocks = (uint64_t)std::max(1, sms) * 32;
  const uint64_t chunk_blocks =
      std::min<uint64_t>(((uint64_t)nb * ((ix->n + 31) / 32) + 7) / 8, cap_blocks);
  const uint64_t new_blocks = std::min<uint64_t>(((uint64_t)n_new + 7) / 8, cap_blocks);
  const uint64_t sort_blocks = std::min<uint64_t>(((uint64_t)RL.dcap + 7) / 8, cap_blocks);
  ix->launches += 5 + (n_new ? 3 : 0);
  k_rb_count_old<<<(unsigned)chunk_blocks, 256, 0, s>>>(a);
  if (n_new)
    k_rb_count_new<<<(unsigned)new_blocks, 256, 0, s>>>(a, ix->d_fwd_off, ix->d_fwd_nnz,
                                                        ix->d_fwd);
  k_rb_plan<<<nb, 1024, 0, s>>>(a, ix->d_tile_dir, ix->d_tile_post, ix->d_err);
  k_rb_merge_old<<<(unsigned)chunk_blocks, 256, 0, s>>>(a);
  if (n_new) {
    k_rb_merge_new<<<(unsigned)new_blocks, 256, 0, s>>>(a, ix->d_fwd_off, ix->d_fwd_nnz,
                                                        ix->d_fwd);
    k_rb_sort<<<(unsigned)sort_blocks, 256, (size_t)8 * (ix->T / 32) * 4, s>>>(a);
  }
  k_rb_flip<<<(nb + 255) / 256, 256, 0, s>>>(a, ix->d_tile_sel);
  CK(cudaGetLastError());
  for (uint32_t i = 0; i < nb; ++i) {
    const uint32_t t = tiles[i];
    const uint64_t slot = (uint64_t)t * 2 + ver[i];
    // the copy's previous storage (replaced by a larger or smaller buffer)
    // is read by no search: searches read the other copy until the flip
    if (ix->tile_post[slot] && ix->tile_post[slot] != newp[i])
      CK(cudaFreeAsync(ix->tile_post[slot], s));
    ix->tile_post[slot] = newp[i];
    ix->tile_post_cap[slot] = pcap[i];
    ix->tile_sel[t] = (uint8_t)ver[i];
    ix->tile_flip_seq[t] = flip_seq;
  }
  std::vector<uint32_t> lens(nb);
  CK(cudaMemcpyAsync(hp, sp + RL.o_ln, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  memcpy(lens.data(), hp, (size_t)nb * 4);
  for (uint32_t i = 0; i < nb; ++i) {
    const uint32_t t = tiles[i];
    ix->tile_post_len[t] = lens[i];
    ix->tombstones -= ix->tile_tombs[t];  // a rebuild compacts tombstones away
    ix->tile_tombs[t] = 0;
  }
  return SINN_OK;
}

// Rebuild the postings of the given tiles (sorted, unique) with the new
// vectors `new_ids` (each in one of them; new_entries store entries in
// all), in groups whose per-coordinate counts fit 1 GiB of scratch, into
// the storage `pre` gives per tile (or allocated as they go if pre is null).
static int rebuild_tiles(sinn_index *ix, const std::vector<uint32_t> &tiles, cudaStream_t s,
                         const std::vector<TileAlloc> *pre, uint32_t flip_seq,
                         const std::vector<uint32_t> &new_ids, uint64_t new_entries) {
  if (tiles.empty()) return SINN_OK;
  const uint32_t g = rebuild_group_tiles(ix, tiles.size());
  std::vector<uint32_t> ids(new_ids);
  std::sort(ids.begin(), ids.end());  // by tile: each group's ids are one run
  size_t k = 0;
  for (size_t g0 = 0; g0 < tiles.size(); g0 += g) {
    const uint32_t nb = (uint32_t)std::min<size_t>(g, tiles.size() - g0);
    const uint32_t last = tiles[g0 + nb - 1];
    const size_t k0 = k;
    while (k < ids.size() && (ids[k] >> ix->log2T) <= last) ++k;
    int st = rebuild_group(ix, tiles.data() + g0, nb, s, pre ? pre->data() + g0 : nullptr,
                           flip_seq, ids.data() + k0, (uint32_t)(k - k0), new_entries);
    if (st) return st;
  }
  return SINN_OK;
}

// From the first sequence-numbered mutation on, searches check the snapshot
// words (recorded searches are made again to pass them).
static void mark_snapshots(sinn_index *ix) {
  if (!ix->snapshots) {
    ix->snapshots = true;
    ix->shape_version++;
  }
}

// Alg. 5 for a batch (sinn_insert; with `at`, sinn_insert_at: the new ids
// are born at sequence number seq, and a tile may only be rebuilt once no
// search older than its last rebuild can still read its other copy).
static int insert_impl(sinn_index *ix, const uint64_t *indptr, const uint32_t *indices,
                       const float *values, uint32_t n_docs, uint32_t *out_ids, void *stream,
                       bool at, uint32_t seq) {
  if (!ix) return SINN_EINVAL;
  if (n_docs == 0) return SINN_OK;
  if (!indptr || !out_ids) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  // host copy of the row pointers (sizes drive allocation)
  const size_t ipb = ((size_t)n_docs + 1) * 8;
  if ((st = sinn_ensure_pinned(ix, ipb + (size_t)n_docs * 12 + 64))) return st;
  uint64_t *hip = (uint64_t *)ix->pinned;
  CK(cudaMemcpyAsync(hip, indptr, ipb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<uint64_t> ip(hip, hip + n_docs + 1);
  for (uint32_t r = 0; r < n_docs; ++r)
    if (ip[r + 1] < ip[r]) return SINN_EINVAL;
  const uint64_t total = ip[n_docs] - ip[0];
  if (total && (!indices || !values)) return SINN_EINVAL;
  for (uint32_t r = 0; r < n_docs; ++r)
    if (ip[r + 1] - ip[r] > 0xFFFFFFFFull) return SINN_EINVAL;
  SinnPhase phase(ix, s, 4);
  // validation before any change
  if (total) {
    ix->launches++;
    uint32_t bits = 0;
    k_validate_csr<<<(n_docs + 7) / 8, 256, 0, s>>>(indptr, indices, values, n_docs, ix->n,
                                                    ix->d_err, SINN_DERR_INSERT,
                                                    (ix->flags & SINN_FLAG_NONNEG) ? 1 : 0);
    CK(cudaGetLastError());
    if ((st = read_and_clear_err(ix, s, &bits))) return st;
    if (bits & SINN_DERR_INSERT) return SINN_EINVAL;
  }
  // ids: smallest free first, then fresh
  std::vector<uint32_t> ids(n_docs);
  std::vector<uint32_t> tiles;      // tiles the batch lands in (sorted)
  std::vector<uint64_t> tile_add;   // entries the batch adds to each
  std::vector<TileAlloc> pre;       // their rebuilds' storage
  const uint64_t n_free = ix->free_ids.size();
  if (ix->next_id + (n_docs > n_free ? n_docs - n_free : 0) > 0xFFFFFFFEull) return SINN_ENOMEM;
  uint64_t max_id = 0;
  bool reuse_recent = false;  // a reused id still carries snapshot words
  {
    auto fq = ix->free_ids;  // commit only after allocations succeed
    uint64_t nid = ix->next_id;
    for (uint32_t r = 0; r < n_docs; ++r) {
      if (!fq.empty()) {
        ids[r] = fq.top();
        fq.pop();
        reuse_recent = reuse_recent || ix->recent[ids[r]];
      } else {
        ids[r] = (uint32_t)nid++;
      }
      max_id = std::max<uint64_t>(max_id, ids[r]);
    }
    std::vector<std::pair<uint32_t, uint64_t>> te(n_docs);  // (tile, entries)
    for (uint32_t r = 0; r < n_docs; ++r) te[r] = {ids[r] >> ix->log2T, ip[r + 1] - ip[r]};
    std::sort(te.begin(), te.end());
    for (const auto &x : te) {
      if (tiles.empty() || tiles.back() != x.first) {
        tiles.push_back(x.first);
        tile_add.push_back(0);
      }
      tile_add.back() += x.second;
    }
    // a sequence-numbered insert rebuilds a tile into the copy searches do
    // not read; a search older than the tile's last rebuild may still read
    // it, unless every such search has been reclaimed
    if (at)
      for (uint32_t t : tiles)
        if (t < ix->tile_flip_seq.size() && ix->tile_flip_seq[t] > ix->reclaimed)
          return SINN_EBUSY;
    if ((st = grow_capacity(ix, max_id + 1))) return st;
    if ((st = grow_store(ix, ix->fwd_used + total))) return st;
    // the rest of the insert's allocations, made before anything changes: on
    // SINN_ENOMEM the index is as it was
    const uint32_t gmax = std::min<uint32_t>(rebuild_group_tiles(ix, tiles.size()),
                                             (uint32_t)tiles.size());
    const size_t o_off0 = ((size_t)n_docs * 4 + 15) / 16 * 16;
    if ((st = ensure_iscratch(ix, std::max(o_off0 + (size_t)n_docs * 8,
                                           rebuild_layout(ix, gmax, n_docs, total).bytes))))
      return st;
    if ((st = sinn_ensure_pinned(ix, std::max(ipb + (size_t)n_docs * 12 + 64,
                                              (size_t)gmax * 24 + (size_t)n_docs * 4))))
      return st;
    pre.resize(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) {
      if ((st = tile_alloc(ix, tiles[i], ix->tile_nnz[tiles[i]] + tile_add[i], s, &pre[i]))) {
        for (size_t k = 0; k < i; ++k)
          if (pre[k].p) cudaFreeAsync(pre[k].p, s);
        cudaStreamSynchronize(s);
        return st;
      }
    }
    ix->free_ids = fq;
    if ((nid + ix->T - 1) / ix->T != (ix->next_id + ix->T - 1) / ix->T) ix->shape_version++;
    ix->next_id = nid;
  }
  // offsets in the store, staged with the ids
  uint32_t *hids = (uint32_t *)((char *)ix->pinned + ipb);
  uint64_t *hoff = (uint64_t *)((char *)ix->pinned + ipb + (((size_t)n_docs * 4 + 7) / 8 * 8));
  for (uint32_t r = 0; r < n_docs; ++r) {
    hids[r] = ids[r];
    hoff[r] = ix->fwd_used + (ip[r] - ip[0]);
  }
  ix->fwd_used += total;
  const size_t o_off = ((size_t)n_docs * 4 + 15) / 16 * 16;
  if ((st = ensure_iscratch(ix, o_off + (size_t)n_docs * 8))) return st;
  uint32_t *d_ids = (uint32_t *)ix->iscratch;
  uint64_t *d_off = (uint64_t *)((char *)ix->iscratch + o_off);
  CK(cudaMemcpyAsync(d_ids, hids, (size_t)n_docs * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_off, hoff, (size_t)n_docs * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(out_ids, d_ids, (size_t)n_docs * 4, cudaMemcpyDeviceToDevice, s));
  ix->launches += 3;  // store, sketch, live bits (the tile rebuild counts itself)
  if (at || reuse_recent) {
    // visibility before the live bits: a search older than seq that sees an
    // id live also sees it was born after its snapshot (a plain insert is
    // visible to every snapshot)
    ix->launches += at ? 3 : 2;
    const unsigned g = (n_docs + 255) / 256;
    k_fill_ids<<<g, 256, 0, s>>>(d_ids, n_docs, ix->d_born, at ? seq : 0u);
    k_fill_ids<<<g, 256, 0, s>>>(d_ids, n_docs, ix->d_died, SINN_SEQ_NEVER);
    if (at) k_set_live<<<g, 256, 0, s>>>(d_ids, n_docs, ix->d_recent, 1);
    CK(cudaGetLastError());
  }
  k_fwd_write<<<(n_docs + 7) / 8, 256, 0, s>>>(indptr, indices, values, n_docs, d_ids, d_off,
                                              ix->d_fwd, ix->d_fwd_off, ix->d_fwd_nnz,
                                              ix->d_coord_len, ix->fwd_cap, ix->cap, ix->d_err);
  CK(cudaGetLastError());
  uint32_t G = std::max<uint32_t>(1, std::min<uint32_t>(32, 6144 / ix->m));
  k_sketch<<<(n_docs + G - 1) / G, 256, (size_t)2 * G * ix->m * 4, s>>>(
      indptr, indices, values, n_docs, d_ids, ix->d_pi, ix->m, ix->h, ix->cap, G, ix->d_U,
      ix->d_L, ix->sk_elem == 2 ? 1 : 0, ix->d_err);
  CK(cudaGetLastError());
  k_set_live<<<(n_docs + 255) / 256, 256, 0, s>>>(d_ids, n_docs, ix->d_live, 1);
  CK(cudaGetLastError());
  for (uint32_t r = 0; r < n_docs; ++r) {
    uint32_t id = ids[r];
    ix->live[id] = 1;
    ix->nnz[id] = (uint32_t)(ip[r + 1] - ip[r]);
    ix->tile_nnz[id >> ix->log2T] += ix->nnz[id];
    ix->live_count++;
    if (at) {
      ix->recent[id] = 1;
      ix->recent_ins.push_back({seq, id});
    }
  }
  ix->launches++;
  k_store_u64<<<1, 1, 0, s>>>(ix->d_live_count, ix->live_count);
  CK(cudaGetLastError());
  if ((st = rebuild_tiles(ix, tiles, s, &pre, at ? seq : 0u, ids, total))) return st;
  uint32_t bits = 0;
  if ((st = read_and_clear_err(ix, s, &bits))) return st;
  return bits ? SINN_EDEVICE : SINN_OK;
}

extern "C" int sinn_insert(sinn_index *ix, const uint64_t *indptr, const uint32_t *indices,
                           const float *values, uint32_t n_docs, uint32_t *out_ids,
                           void *stream) {
  return insert_impl(ix, indptr, indices, values, n_docs, out_ids, stream, false, 0);
}

extern "C" int sinn_insert_at(sinn_index *ix, const uint64_t *indptr, const uint32_t *indices,
                              const float *values, uint32_t n_docs, uint32_t *out_ids,
                              uint32_t seq, void *stream) {
  if (!ix || seq > SINN_SEQ_LATEST) return SINN_EINVAL;
  mark_snapshots(ix);
  return insert_impl(ix, indptr, indices, values, n_docs, out_ids, stream, true, seq);
}

// Sec. 4.3 deletion of n_ids live ids (host list v, device copy d_src):
// postings tombstoned in the copy searches read, live bits cleared, ids
// freed for reuse.
static int delete_physical(sinn_index *ix, const uint32_t *d_src, const std::vector<uint32_t> &v,
                           cudaStream_t s) {
  const uint32_t n_ids = (uint32_t)v.size();
  int st;
  const size_t o_cnt = ((size_t)n_ids * 4 + 15) / 16 * 16;
  if ((st = ensure_iscratch(ix, o_cnt + (size_t)n_ids * 4))) return st;
  if ((st = sinn_ensure_pinned(ix, (size_t)n_ids * 4 + 64))) return st;
  uint32_t *d_ids = (uint32_t *)ix->iscratch;
  uint32_t *d_cnt = (uint32_t *)((char *)ix->iscratch + o_cnt);
  if (d_src) {
    CK(cudaMemcpyAsync(d_ids, d_src, (size_t)n_ids * 4, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaStreamSynchronize(s));  // the staging buffer is free
    memcpy(ix->pinned, v.data(), (size_t)n_ids * 4);
    CK(cudaMemcpyAsync(d_ids, ix->pinned, (size_t)n_ids * 4, cudaMemcpyHostToDevice, s));
  }
  SinnPhase phase(ix, s, 5);
  ix->launches++;
  k_tombstone<<<(n_ids + 7) / 8, 256, 0, s>>>(d_ids, n_ids, ix->d_fwd_off, ix->d_fwd_nnz,
                                              ix->d_fwd, ix->d_tile_dir, ix->d_tile_post,
                                              ix->d_tile_sel, ix->d_live, ix->n, ix->log2T, d_cnt,
                                              ix->d_coord_len, ix->d_err);
  CK(cudaGetLastError());
  uint32_t *hc = (uint32_t *)ix->pinned;
  CK(cudaMemcpyAsync(hc, d_cnt, (size_t)n_ids * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (uint32_t i = 0; i < n_ids; ++i) {
    ix->tile_tombs[v[i] >> ix->log2T] += hc[i];
    ix->tombstones += hc[i];
  }
  for (uint32_t id : v) {
    ix->live[id] = 0;
    ix->tile_nnz[id >> ix->log2T] -= ix->nnz[id];
    ix->nnz[id] = 0;
    ix->live_count--;
    ix->free_ids.push(id);
  }
  ix->launches++;
  k_store_u64<<<1, 1, 0, s>>>(ix->d_live_count, ix->live_count);
  CK(cudaGetLastError());
  uint32_t bits = 0;
  if ((st = read_and_clear_err(ix, s, &bits))) return st;
  return bits ? SINN_EDEVICE : SINN_OK;
}

// The ids of a delete call on the host, checked: each live (and not already
// deleted at a sequence number), none repeated.
static int delete_ids(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, cudaStream_t s,
                      std::vector<uint32_t> *out) {
  int st;
  if ((st = sinn_ensure_pinned(ix, (size_t)n_ids * 4 + 64))) return st;
  uint32_t *h = (uint32_t *)ix->pinned;
  CK(cudaMemcpyAsync(h, ids, (size_t)n_ids * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out->assign(h, h + n_ids);
  for (uint32_t id : *out)
    if (id >= ix->next_id || ix->live[id] != 1) return SINN_ENOTFOUND;
  std::vector<uint32_t> srt(*out);
  std::sort(srt.begin(), srt.end());
  if (std::adjacent_find(srt.begin(), srt.end()) != srt.end()) return SINN_EINVAL;
  return SINN_OK;
}

extern "C" int sinn_delete(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, void *stream) {
  if (!ix) return SINN_EINVAL;
  if (n_ids == 0) return SINN_OK;
  if (!ids) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> v;
  int st = delete_ids(ix, ids, n_ids, s, &v);
  if (st) return st;
  return delete_physical(ix, ids, v, s);
}

extern "C" int sinn_delete_at(sinn_index *ix, const uint32_t *ids, uint32_t n_ids, uint32_t seq,
                              void *stream) {
  if (!ix || seq > SINN_SEQ_LATEST) return SINN_EINVAL;
  if (n_ids == 0) return SINN_OK;
  if (!ids) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> v;
  int st = delete_ids(ix, ids, n_ids, s, &v);
  if (st) return st;
  mark_snapshots(ix);
  // searches at seq or later no longer count the ids; their postings stay
  // for the older ones until sinn_reclaim removes them
  SinnPhase phase(ix, s, 5);
  ix->launches += 2;
  const unsigned g = (n_ids + 255) / 256;
  k_fill_ids<<<g, 256, 0, s>>>(ids, n_ids, ix->d_died, seq);
  k_set_live<<<g, 256, 0, s>>>(ids, n_ids, ix->d_recent, 1);
  CK(cudaGetLastError());
  for (uint32_t id : v) {
    ix->live[id] = 2;
    ix->recent[id] = 1;
    ix->pending_del.push_back({seq, id});
  }
  CK(cudaStreamSynchronize(s));
  return SINN_OK;
}

extern "C" int sinn_reclaim(sinn_index *ix, uint32_t horizon, void *stream) {
  if (!ix || horizon > SINN_SEQ_LATEST + 1) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  ix->reclaimed = std::max(ix->reclaimed, horizon);
  // deleted ids no search still counts: postings removed, ids freed (their
  // death words stay, so a search that still sees them live drops them)
  std::vector<uint32_t> dead;
  std::vector<std::pair<uint32_t, uint32_t>> keep;
  for (const auto &p : ix->pending_del) {
    if (p.first <= ix->reclaimed) dead.push_back(p.second);
    else keep.push_back(p);
  }
  int st = SINN_OK;
  if (!dead.empty()) {
    for (uint32_t id : dead) ix->live[id] = 1;  // physically live until removed
    st = delete_physical(ix, nullptr, dead, s);
    if (st) {
      for (uint32_t id : dead) ix->live[id] = 2;
      return st;
    }
    ix->pending_del.swap(keep);
  }
  // inserted ids every search in flight counts: no snapshot check needed
  std::vector<uint32_t> settled;
  std::vector<std::pair<uint32_t, uint32_t>> young;
  for (const auto &p : ix->recent_ins) {
    if (p.first > ix->reclaimed) young.push_back(p);
    else if (ix->live[p.second] == 1) settled.push_back(p.second);
  }
  ix->recent_ins.swap(young);
  if (!settled.empty()) {
    const size_t o = 0;
    if ((st = ensure_iscratch(ix, o + settled.size() * 4))) return st;
    if ((st = sinn_ensure_pinned(ix, settled.size() * 4 + 64))) return st;
    CK(cudaStreamSynchronize(s));
    memcpy(ix->pinned, settled.data(), settled.size() * 4);
    CK(cudaMemcpyAsync(ix->iscratch, ix->pinned, settled.size() * 4, cudaMemcpyHostToDevice, s));
    ix->launches++;
    k_set_live<<<(unsigned)((settled.size() + 255) / 256), 256, 0, s>>>(
        (const uint32_t *)ix->iscratch, (uint32_t)settled.size(), ix->d_recent, 0);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    for (uint32_t id : settled) ix->recent[id] = 0;
  }
  return SINN_OK;
}

extern "C" int sinn_reserve(sinn_index *ix, uint64_t more_ids, uint64_t more_entries) {
  if (!ix) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  if (more_ids > 0xFFFFFFFEull || more_entries > (1ull << 40)) return SINN_ENOMEM;
  int st = grow_capacity(ix, ix->next_id + more_ids);
  if (st) return st;
  return grow_store(ix, ix->fwd_used + more_entries);
}

extern "C" int sinn_stats(sinn_index *ix, sinn_stats_t *out) {
  if (!ix || !out) return SINN_EINVAL;
  memset(out, 0, sizeof(*out));
  out->live = ix->live_count - ix->pending_del.size();
  out->capacity = ix->cap;
  out->next_id = ix->next_id;
  uint64_t post = 0, pbytes = 0;
  for (size_t t = 0; t < ix->tile_post_len.size(); ++t) post += ix->tile_post_len[t];
  for (size_t i = 0; i < ix->tile_post_cap.size(); ++i) pbytes += ix->tile_post_cap[i] * 2;
  out->postings = post;
  out->tombstones = ix->tombstones;
  out->bytes_lists = pbytes + 2 * (ix->cap / ix->T) * (uint64_t)ix->n * 8;
  out->pending_deletes = (uint32_t)ix->pending_del.size();
  out->bytes_sketch = (ix->d_L ? 2ull : 1ull) * ix->m * ix->cap * ix->sk_elem;
  out->bytes_store = ix->fwd_cap * 8 + ix->cap * 12;
  out->bytes_scratch = ix->scratch_size + ix->iscratch_size;
  out->n = ix->n;
  out->m = ix->m;
  out->h = ix->h;
  out->tile_docs = ix->T;
  out->flags = ix->flags;
  return SINN_OK;
}

extern "C" int sinn_hash_table(sinn_index *ix, uint32_t *table) {
  if (!ix || !table) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  CK(cudaMemcpy(table, ix->d_pi, (size_t)ix->n * ix->h * 4, cudaMemcpyDeviceToHost));
  return SINN_OK;
}

extern "C" int sinn_sketch_columns(sinn_index *ix, const uint32_t *ids, uint32_t n_ids,
                                   float *u_out, float *l_out, void *stream) {
  if (!ix || (n_ids && (!ids || !u_out)) || (l_out && !ix->d_L)) return SINN_EINVAL;
  if (n_ids == 0) return SINN_OK;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t tot = (uint64_t)n_ids * ix->m;
  k_gather_columns<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ids, n_ids, ix->d_U, ix->d_L,
                                                                  ix->m, ix->cap,
                                                                  ix->sk_elem == 2 ? 1 : 0,
                                                                  u_out, l_out);
  CK(cudaGetLastError());
  return SINN_OK;
}

extern "C" int sinn_inverted_list(sinn_index *ix, uint32_t coord, uint32_t *out, uint64_t cap,
                                  uint64_t *len) {
  if (!ix || coord >= ix->n || !len || (cap && !out)) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  CK(cudaDeviceSynchronize());
  const uint64_t nt = ix->cap / ix->T;
  const uint32_t W16 = ix->T / 16;
  // the coordinate's entry in both copies of every tile; the current one counts
  std::vector<uint2> dd(2 * nt);
  CK(cudaMemcpy2D(dd.data(), sizeof(uint2), ix->d_tile_dir + coord, (size_t)ix->n * sizeof(uint2),
                  sizeof(uint2), 2 * nt, cudaMemcpyDeviceToHost));
  uint64_t cnt = 0;
  std::vector<uint16_t> buf;
  for (uint64_t t = 0; t < nt; ++t) {
    const uint64_t slot = 2 * t + ix->tile_sel[t];
    const uint2 de = dd[slot];
    if (de.y == 0 || !ix->tile_post[slot]) continue;
    const bool bitmap = de.y >= (ix->T >> SINN_BITMAP_SHIFT);
    buf.resize(bitmap ? W16 : de.y);
    CK(cudaMemcpy(buf.data(), ix->tile_post[slot] + de.x, buf.size() * 2, cudaMemcpyDeviceToHost));
    auto emit = [&](uint32_t d) {
      if (cnt < cap) out[cnt] = (uint32_t)((t << ix->log2T) + d);
      cnt++;
    };
    if (bitmap) {
      for (uint32_t w = 0; w < W16; ++w)
        for (uint32_t b = 0; b < 16; ++b)
          if ((buf[w] >> b) & 1u) emit(w * 16 + b);
    } else {
      for (uint16_t d : buf)
        if (!(d & SINN_TOMB)) emit(d);
    }
  }
  *len = cnt;
  return SINN_OK;
}

// ------------------------------------------------------------ save / load
// A saved index is the index's whole state, device arrays copied through a
// host buffer: a header (magic, version, parameters, counters, tuning), then
// the mapping table, the sketch planes, the live bits, the store offsets,
// counts and entries, the tile directory, the per-coordinate live counts, the
// host mirror (live flags, counts, free ids, per-tile sizes) and each tile's
// container storage.  Every array is preceded by its byte count, checked on
// load.  Little-endian hosts only (x86-64 and aarch64 both are).
namespace {

constexpr char kMagic[8] = {'S', 'I', 'N', 'N', 'I', 'D', 'X', '1'};
constexpr uint32_t kVersion = 1;

struct SaveHeader {
  char magic[8];
  uint32_t version, n, m, h, T, flags, max_qnnz, sk_elem;
  uint64_t seed, cap, next_id, live_count, fwd_used, fwd_cap, budget, scratch_budget, tombstones;
  sinn_tuning tune;
};

constexpr size_t kChunk = 64ull << 20;  // host staging per copy

struct File {
  FILE *f = nullptr;
  std::vector<char> buf;
  ~File() {
    if (f) fclose(f);
  }
  bool put(const void *p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
  bool get(void *p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }
};

// One array: its byte count, then the bytes (from the device if dev).
int put_array(File &F, const void *src, uint64_t bytes, bool dev) {
  if (!F.put(&bytes, 8)) return SINN_EIO;
  if (!dev) return F.put(src, bytes) ? SINN_OK : SINN_EIO;
  for (uint64_t o = 0; o < bytes; o += kChunk) {
    const size_t n = (size_t)std::min<uint64_t>(kChunk, bytes - o);
    CK(cudaMemcpy(F.buf.data(), (const char *)src + o, n, cudaMemcpyDeviceToHost));
    if (!F.put(F.buf.data(), n)) return SINN_EIO;
  }
  return SINN_OK;
}

// One array of exactly `bytes` bytes into dst (on the device if dev).
int get_array(File &F, void *dst, uint64_t bytes, bool dev) {
  uint64_t have = 0;
  if (!F.get(&have, 8) || have != bytes) return SINN_EIO;
  if (!dev) return F.get(dst, bytes) ? SINN_OK : SINN_EIO;
  for (uint64_t o = 0; o < bytes; o += kChunk) {
    const size_t n = (size_t)std::min<uint64_t>(kChunk, bytes - o);
    if (!F.get(F.buf.data(), n)) return SINN_EIO;
    CK(cudaMemcpy((char *)dst + o, F.buf.data(), n, cudaMemcpyHostToDevice));
  }
  return SINN_OK;
}

// Everything sinn_save writes after opening the file.
int save_body(sinn_index *ix, File &F) {
  F.buf.resize(kChunk);
  SaveHeader hd{};
  memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.n = ix->n;
  hd.m = ix->m;
  hd.h = ix->h;
  hd.T = ix->T;
  hd.flags = ix->flags;
  hd.max_qnnz = ix->max_qnnz;
  hd.sk_elem = ix->sk_elem;
  hd.seed = ix->seed;
  hd.cap = ix->cap;
  hd.next_id = ix->next_id;
  hd.live_count = ix->live_count;
  hd.fwd_used = ix->fwd_used;
  hd.fwd_cap = ix->fwd_cap;
  hd.budget = ix->budget;
  hd.scratch_budget = ix->scratch_budget;
  hd.tombstones = ix->tombstones;
  hd.tune = ix->tune;
  if (!F.put(&hd, sizeof hd)) return SINN_EIO;
  const uint64_t cap = ix->cap, tiles = cap / ix->T, plane = (uint64_t)ix->m * cap * ix->sk_elem;
  int st;
  if ((st = put_array(F, ix->d_pi, (uint64_t)ix->n * ix->h * 4, true))) return st;
  if ((st = put_array(F, ix->d_U, plane, true))) return st;
  if ((st = put_array(F, ix->d_L, ix->d_L ? plane : 0, true))) return st;
  if ((st = put_array(F, ix->d_live, cap / 32 * 4, true))) return st;
  if ((st = put_array(F, ix->d_fwd_off, cap * 8, true))) return st;
  if ((st = put_array(F, ix->d_fwd_nnz, cap * 4, true))) return st;
  if ((st = put_array(F, ix->d_fwd, ix->fwd_used * 8, true))) return st;
  {  // the directory of each tile's current copy
    const uint64_t bytes = tiles * ix->n * 8;
    if (!F.put(&bytes, 8)) return SINN_EIO;
    for (uint64_t t = 0; t < tiles; ++t) {
      CK(cudaMemcpy(F.buf.data(), ix->d_tile_dir + (2 * t + ix->tile_sel[t]) * ix->n,
                    (size_t)ix->n * 8, cudaMemcpyDeviceToHost));
      if (!F.put(F.buf.data(), (size_t)ix->n * 8)) return SINN_EIO;
    }
  }
  if ((st = put_array(F, ix->d_coord_len, (uint64_t)ix->n * 4, true))) return st;
  if ((st = put_array(F, ix->live.data(), cap, false))) return st;
  if ((st = put_array(F, ix->nnz.data(), cap * 4, false))) return st;
  std::vector<uint32_t> free_ids;
  for (auto q = ix->free_ids; !q.empty(); q.pop()) free_ids.push_back(q.top());
  if ((st = put_array(F, free_ids.data(), free_ids.size() * 4, false))) return st;
  std::vector<uint64_t> cur_cap(tiles);
  for (uint64_t t = 0; t < tiles; ++t) cur_cap[t] = ix->tile_post_cap[2 * t + ix->tile_sel[t]];
  if ((st = put_array(F, ix->tile_post_len.data(), tiles * 8, false))) return st;
  if ((st = put_array(F, cur_cap.data(), tiles * 8, false))) return st;
  if ((st = put_array(F, ix->tile_nnz.data(), tiles * 8, false))) return st;
  if ((st = put_array(F, ix->tile_tombs.data(), tiles * 8, false))) return st;
  for (uint64_t t = 0; t < tiles; ++t) {
    const uint64_t slot = 2 * t + ix->tile_sel[t];
    if ((st = put_array(F, ix->tile_post[slot],
                        ix->tile_post[slot] ? ix->tile_post_cap[slot] * 2 : 0, true)))
      return st;
  }
  return SINN_OK;
}

}  // namespace

extern "C" int sinn_save(sinn_index *ix, const char *path) {
  if (!ix || !path) return SINN_EINVAL;
  // deletions not yet reclaimed have no place in the file
  if (!ix->pending_del.empty()) return SINN_EBUSY;
  SinnDevice dev_guard_(ix->device);
  CK(cudaDeviceSynchronize());
  // written to a temporary file beside the target and renamed over it only
  // when every byte is on disk: an error part-way leaves the previous
  // checkpoint as it was
  const std::string tmp = std::string(path) + ".tmp";
  File F;
  F.f = fopen(tmp.c_str(), "wb");
  if (!F.f) return SINN_EIO;
  const int st = save_body(ix, F);
  const bool flushed = st == SINN_OK && fflush(F.f) == 0;
  const bool closed = fclose(F.f) == 0;
  F.f = nullptr;
  if (st != SINN_OK || !flushed || !closed || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return st != SINN_OK ? st : SINN_EIO;
  }
  return SINN_OK;
}

namespace {

// What sinn_load's first pass keeps: the header, every array the kernels
// index through (checked), and where the value-only arrays sit in the file.
struct LoadPlan {
  SaveHeader hd{};
  std::vector<uint32_t> table, live_bits, fwd_nnz, coord_len, nnz, free_ids;
  std::vector<uint64_t> fwd_off, post_len, post_cap, tile_nnz, tile_tombs;
  std::vector<uint8_t> live;
  std::vector<uint2> dir;
  off_t at_U = 0, at_L = 0, at_fwd = 0;  // file offsets of those arrays' bytes
  std::vector<off_t> at_post;            // per tile (0: no storage)
};

// The byte count of the next array, which must be `bytes`; then skip it and
// note where its bytes begin.
bool skip_array(File &F, uint64_t bytes, off_t *at) {
  uint64_t have = 0;
  if (!F.get(&have, 8) || have != bytes) return false;
  *at = ftello(F.f);
  return *at >= 0 && fseeko(F.f, (off_t)bytes, SEEK_CUR) == 0;
}

// First pass, on the host only: read the file and check it against the
// invariants every saved index satisfies.  The sketch planes hold values
// (never used as indices) and are only located.  Everything the kernels
// index through -- live bits, store offsets, counts and coordinates, the tile
// directory and the tile containers -- is checked here, so that a damaged or
// foreign file is SINN_EIO before the device is touched rather than an
// out-of-range access on the GPU.
int load_check(File &F, LoadPlan &L) {
  SaveHeader &hd = L.hd;
  if (!F.get(&hd, sizeof hd) || memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kVersion)
    return SINN_EIO;
  // parameters as sinn_create_ex accepts them, and counters that fit them
  if (hd.n == 0 || hd.m == 0 || hd.h == 0 || hd.h > hd.m || hd.h > SINN_MAX_H || hd.m > 4096 ||
      hd.T < 1024 || hd.T > 16384 || (hd.T & (hd.T - 1)) || hd.cap % hd.T || hd.cap == 0 ||
      hd.cap > 65535ull * hd.T || hd.next_id > hd.cap || hd.live_count > hd.next_id ||
      hd.fwd_used > hd.fwd_cap || hd.sk_elem != ((hd.flags & SINN_FLAG_BF16_SKETCH) ? 2u : 4u) ||
      (hd.flags & ~(SINN_FLAG_NONNEG | SINN_FLAG_BF16_SKETCH)))
    return SINN_EIO;
  F.buf.resize(kChunk);
  const uint64_t cap = hd.cap, tiles = cap / hd.T, n = hd.n;
  const uint64_t plane = (uint64_t)hd.m * cap * hd.sk_elem;
  const bool has_L = !(hd.flags & SINN_FLAG_NONNEG);
  L.table.resize(n * hd.h);
  int st = get_array(F, L.table.data(), L.table.size() * 4, false);
  if (st) return st;
  for (uint32_t b : L.table)
    if (b >= hd.m) return SINN_EIO;
  if (!skip_array(F, plane, &L.at_U) || !skip_array(F, has_L ? plane : 0, &L.at_L))
    return SINN_EIO;
  L.live_bits.resize(cap / 32);
  L.fwd_off.resize(cap);
  L.fwd_nnz.resize(cap);
  if ((st = get_array(F, L.live_bits.data(), cap / 32 * 4, false))) return st;
  if ((st = get_array(F, L.fwd_off.data(), cap * 8, false))) return st;
  if ((st = get_array(F, L.fwd_nnz.data(), cap * 4, false))) return st;
  {  // the store's entries: every coordinate < n (each came from a validated insert)
    uint64_t have = 0;
    const uint64_t bytes = hd.fwd_used * 8;
    if (!F.get(&have, 8) || have != bytes) return SINN_EIO;
    L.at_fwd = ftello(F.f);
    for (uint64_t o = 0; o < bytes; o += kChunk) {
      const size_t nb = (size_t)std::min<uint64_t>(kChunk, bytes - o);
      if (!F.get(F.buf.data(), nb)) return SINN_EIO;
      const uint2 *e = (const uint2 *)F.buf.data();
      for (size_t i = 0; i < nb / 8; ++i)
        if (e[i].x >= n) return SINN_EIO;
    }
  }
  L.dir.resize(tiles * n);
  L.coord_len.resize(n);
  L.live.resize(cap);
  L.nnz.resize(cap);
  if ((st = get_array(F, L.dir.data(), tiles * n * 8, false))) return st;
  if ((st = get_array(F, L.coord_len.data(), n * 4, false))) return st;
  if ((st = get_array(F, L.live.data(), cap, false))) return st;
  if ((st = get_array(F, L.nnz.data(), cap * 4, false))) return st;
  uint64_t nfree = 0;
  if (!F.get(&nfree, 8) || nfree % 4 || nfree / 4 > hd.next_id) return SINN_EIO;
  L.free_ids.resize(nfree / 4);
  if (!F.get(L.free_ids.data(), nfree)) return SINN_EIO;
  L.post_len.resize(tiles);
  L.post_cap.resize(tiles);
  L.tile_nnz.resize(tiles);
  L.tile_tombs.resize(tiles);
  if ((st = get_array(F, L.post_len.data(), tiles * 8, false))) return st;
  if ((st = get_array(F, L.post_cap.data(), tiles * 8, false))) return st;
  if ((st = get_array(F, L.tile_nnz.data(), tiles * 8, false))) return st;
  if ((st = get_array(F, L.tile_tombs.data(), tiles * 8, false))) return st;
  // live ids: host flags equal the device bits, only below next_id, as many
  // as the header says; each live vector's entries lie inside the used store
  // and its count is the host's; per tile, the entries of its live vectors
  // are the host's running sum (it sizes the tile's storage on a rebuild)
  uint64_t nlive = 0;
  std::vector<uint64_t> tile_sum(tiles, 0);
  for (uint64_t i = 0; i < cap; ++i) {
    const uint8_t l = L.live[i];
    const bool bit = (L.live_bits[i >> 5] >> (i & 31)) & 1u;
    if (l > 1 || bit != (l == 1)) return SINN_EIO;
    if (!l) continue;
    if (i >= hd.next_id || L.fwd_nnz[i] != L.nnz[i] || L.fwd_off[i] > hd.fwd_used ||
        L.fwd_nnz[i] > hd.fwd_used - L.fwd_off[i])
      return SINN_EIO;
    ++nlive;
    tile_sum[i / hd.T] += L.fwd_nnz[i];
  }
  if (nlive != hd.live_count) return SINN_EIO;
  for (uint64_t t = 0; t < tiles; ++t)
    if (tile_sum[t] != L.tile_nnz[t]) return SINN_EIO;
  // free ids: distinct, below next_id, not live; with the live ids they are
  // every id handed out
  {
    std::vector<uint8_t> seen(hd.next_id, 0);
    for (uint32_t id : L.free_ids) {
      if (id >= hd.next_id || L.live[id] || seen[id]) return SINN_EIO;
      seen[id] = 1;
    }
    if (L.free_ids.size() + hd.live_count != hd.next_id) return SINN_EIO;
  }
  // containers inside their tile's storage (arrays from the front, bitmaps
  // on T/16-word boundaries from the back, read as 32-bit words); array
  // entries are local ids < T
  const uint32_t BMIN = hd.T >> SINN_BITMAP_SHIFT, W16 = hd.T / 16;
  std::vector<uint16_t> words;
  L.at_post.assign(tiles, 0);
  for (uint64_t t = 0; t < tiles; ++t) {
    uint64_t bytes = 0;
    if (!F.get(&bytes, 8)) return SINN_EIO;
    const uint2 *de = L.dir.data() + t * n;
    if (bytes == 0) {  // a tile without storage holds no container
      for (uint64_t j = 0; j < n; ++j)
        if (de[j].y) return SINN_EIO;
      if (L.post_len[t]) return SINN_EIO;
      L.post_cap[t] = 0;
      continue;
    }
    if (bytes != L.post_cap[t] * 2) return SINN_EIO;
    L.at_post[t] = ftello(F.f);
    words.resize(bytes / 2);
    if (!F.get(words.data(), bytes)) return SINN_EIO;
    const uint64_t wcap = L.post_cap[t];
    for (uint64_t j = 0; j < n; ++j) {
      const uint64_t start = de[j].x, cnt = de[j].y;
      if (cnt == 0) continue;
      if (cnt > hd.T) return SINN_EIO;
      const uint64_t w = cnt >= BMIN ? W16 : cnt;
      if (start > wcap || w > wcap - start) return SINN_EIO;
      if (cnt >= BMIN && start % W16) return SINN_EIO;
      if (cnt < BMIN)
        for (uint64_t q = start; q < start + cnt; ++q)
          if ((words[q] & 0x7FFFu) >= hd.T) return SINN_EIO;
    }
  }
  return SINN_OK;
}

// One value-only array of `bytes` bytes at file offset `at`, to the device.
int upload_from(File &F, off_t at, void *dst, uint64_t bytes) {
  if (!bytes) return SINN_OK;
  if (fseeko(F.f, at, SEEK_SET) != 0) return SINN_EIO;
  for (uint64_t o = 0; o < bytes; o += kChunk) {
    const size_t nb = (size_t)std::min<uint64_t>(kChunk, bytes - o);
    if (!F.get(F.buf.data(), nb)) return SINN_EIO;
    CK(cudaMemcpy((char *)dst + o, F.buf.data(), nb, cudaMemcpyHostToDevice));
  }
  return SINN_OK;
}

}  // namespace

extern "C" int sinn_load(const char *path, sinn_index **out) {
  if (!path || !out) return SINN_EINVAL;
  *out = nullptr;
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return SINN_EIO;
  LoadPlan L;
  int st = load_check(F, L);
  if (st) return st;
  const SaveHeader &hd = L.hd;
  // second pass: an index of the same parameters, filled from the checked
  // arrays and the value-only ones re-read from the file
  sinn_config cfg{};
  cfg.n = hd.n;
  cfg.m = hd.m;
  cfg.h = hd.h;
  cfg.tile_docs = hd.T;
  cfg.seed = hd.seed;
  cfg.capacity_hint = hd.cap;
  cfg.table = L.table.data();
  cfg.max_query_nnz = hd.max_qnnz;
  cfg.flags = hd.flags;
  cfg.scratch_bytes = hd.scratch_budget;
  sinn_index *ix = nullptr;
  if ((st = sinn_create_ex(&cfg, &ix))) return st;
  SinnDevice dev_guard_(ix->device);
  auto fail = [&](int e) {
    release(ix);
    return e;
  };
  auto up = [&](void *dst, const void *src, uint64_t bytes) {
    return bytes ? sinn_check_cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice)) : SINN_OK;
  };
  if (ix->cap != hd.cap) return fail(SINN_EIO);
  if ((st = grow_store(ix, std::max<uint64_t>(hd.fwd_cap, 1)))) return fail(st);
  const uint64_t cap = hd.cap, tiles = cap / hd.T, plane = (uint64_t)hd.m * cap * hd.sk_elem;
  if ((st = upload_from(F, L.at_U, ix->d_U, plane))) return fail(st);
  if ((st = upload_from(F, L.at_L, ix->d_L, ix->d_L ? plane : 0))) return fail(st);
  if ((st = upload_from(F, L.at_fwd, ix->d_fwd, hd.fwd_used * 8))) return fail(st);
  for (uint64_t t = 0; t < tiles; ++t) {  // every tile's copy 0 is current
    if (!L.post_cap[t]) continue;
    uint16_t *p = nullptr;
    if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&p, L.post_cap[t] * 2)))) return fail(st);
    ix->tile_post[2 * t] = p;
    ix->tile_post_cap[2 * t] = L.post_cap[t];
    if ((st = upload_from(F, L.at_post[t], p, L.post_cap[t] * 2))) return fail(st);
  }
  if ((st = up(ix->d_live, L.live_bits.data(), cap / 32 * 4))) return fail(st);
  if ((st = up(ix->d_fwd_off, L.fwd_off.data(), cap * 8))) return fail(st);
  if ((st = up(ix->d_fwd_nnz, L.fwd_nnz.data(), cap * 4))) return fail(st);
  if (tiles &&
      (st = sinn_check_cuda(cudaMemcpy2D(ix->d_tile_dir, (size_t)2 * hd.n * 8, L.dir.data(),
                                         (size_t)hd.n * 8, (size_t)hd.n * 8, tiles,
                                         cudaMemcpyHostToDevice))))
    return fail(st);
  if ((st = up(ix->d_coord_len, L.coord_len.data(), (uint64_t)hd.n * 4))) return fail(st);
  if ((st = up(ix->d_tile_post, ix->tile_post.data(), 2 * tiles * sizeof(uint16_t *))))
    return fail(st);
  if ((st = up(ix->d_live_count, &hd.live_count, 8))) return fail(st);
  ix->live = L.live;
  ix->nnz = L.nnz;
  for (uint32_t id : L.free_ids) ix->free_ids.push(id);
  ix->tile_post_len = L.post_len;
  ix->tile_nnz = L.tile_nnz;
  ix->tile_tombs = L.tile_tombs;
  ix->next_id = hd.next_id;
  ix->live_count = hd.live_count;
  ix->fwd_used = hd.fwd_used;
  ix->budget = hd.budget;
  ix->tombstones = hd.tombstones;
  if (sinn_set_tuning(ix, &hd.tune) != SINN_OK) return fail(SINN_EIO);
  ix->shape_version++;
  *out = ix;
  return SINN_OK;
}
