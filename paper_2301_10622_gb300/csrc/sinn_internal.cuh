// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <queue>
#include <vector>

#include "../../include/sinnamon.h"

// ---------------------------------------------------------------- constants
#define SINN_MAX_H 8
#define SINN_MAX_K 1024
#define SINN_TOMB 0x8000u   // tombstone bit of a 16-bit local posting id
#define SINN_HIST0_BITS 12  // first select level: key bits [31:20]
#define SINN_HIST1_BITS 12  // second level: key bits [19:8]
#define SINN_HIST2_BITS 8   // third level: key bits [7:0]
// A tile's container of one coordinate is a bitmap of T bits once it holds
// at least T >> SINN_BITMAP_SHIFT postings (an eighth of the tile), else a
// sorted array of 16-bit local ids.  Scoring a bitmap reads the term's
// sketch row for every id of the tile: up to 8x its postings, but coalesced
// and without atomics or index loads; at T/8 and above that is the cheaper
// of the two (measured against T/4 and T/16), and the bitmap (T/16 words)
// is never larger than the array.
#define SINN_BITMAP_SHIFT 3

// device error bits (sticky flag)
#define SINN_DERR_QUERY 1u     // malformed query
#define SINN_DERR_INTERNAL 2u  // an internal capacity check failed
#define SINN_DERR_INSERT 4u    // malformed insert batch (validation kernel)
#define SINN_DERR_TIMEOUT 8u   // a bounded wait in a kernel ran out
#define SINN_DERR_BOUNDS 16u   // a checked index was out of range (bounds-check builds)
// bits that mean a kernel went wrong (SINN_EDEVICE), not a malformed input
#define SINN_DERR_DEVICE (SINN_DERR_INTERNAL | SINN_DERR_TIMEOUT | SINN_DERR_BOUNDS)

// never deleted (died of a live id)
#define SINN_SEQ_NEVER 0xFFFFFFFFu

// Index checks compiled in with -DSINN_BOUNDS_CHECK (the library's stand-in
// for a memory checker): a failed check sets SINN_DERR_BOUNDS in the error
// word `err` and the caller skips the access.  Compiled out, the condition is
// not evaluated and the check is true.
#ifdef SINN_BOUNDS_CHECK
#define SINN_IN_BOUNDS(cond, err) ((cond) ? true : (atomicOr((err), SINN_DERR_BOUNDS), false))
#else
#define SINN_IN_BOUNDS(cond, err) true
#endif

// ------------------------------------------------------------ index object
struct sinn_index {
  uint32_t n = 0, m = 0, h = 0;
  uint32_t T = 0, log2T = 0;  // ids per tile
  uint64_t seed = 0;
  uint32_t max_qnnz = 0;
  uint64_t scratch_budget = 0;
  int device = 0;
  uint32_t flags = 0;        // SINN_FLAG_NONNEG: no L plane (SINNAMON+)
  uint64_t budget = 0;       // Alg. 6 anytime budget in postings, 0 = none
  // Search launch parameters.  Defaults: refresh the running bound every 4
  // tiles; launches of fewer than 32 queries score densely (their tiles run
  // at about the same time, so the bound could not prune); batches as large
  // as the scratch allows; re-rank blocks per query sized to k' (about 64
  // candidates each); 8 dense blocks (of 256 threads) per SM; 4 tiles per
  // block of the batched scoring kernel, one block per item; array postings
  // in per-term chunks.
  sinn_tuning tune{4, 32, 0, 0, 8, 4, 0, 0};

  // ---- device state
  uint32_t *d_pi = nullptr;        // n*h mappings
  void *d_U = nullptr;             // m x cap, row-major (row k contiguous over ids):
  void *d_L = nullptr;             //   fp32, or bfloat16 bits with SINN_FLAG_BF16_SKETCH
  uint32_t sk_elem = 4;            // bytes per sketch bin
  uint32_t *d_live = nullptr;      // cap/32 bitmap words
  uint64_t *d_fwd_off = nullptr;   // cap: offset of each vector in d_fwd
  uint32_t *d_fwd_nnz = nullptr;   // cap: entries stored (zeros included)
  uint2 *d_fwd = nullptr;          // vector store pool: (coordinate, value bits)
  uint64_t fwd_cap = 0, fwd_used = 0;
  // Each tile has two copies of its containers (directory and storage), so
  // that a rebuild can write one while searches read the other; d_tile_sel
  // names the copy searches use.  Copy v of tile t: directory entries at
  // d_tile_dir + (2t + v) n (per coordinate {start, count}; count >= T/8: a
  // bitmap of T bits, else a sorted array), storage d_tile_post[2t + v].
  uint2 *d_tile_dir = nullptr;     // 2 x tiles_cap x n
  uint16_t **d_tile_post = nullptr;  // 2 x tiles_cap device pointers
  uint32_t *d_tile_sel = nullptr;  // tiles_cap: the copy searches read
  // Snapshot visibility: a search at sequence number s counts id i only if
  // born[i] <= s < died[i]; consulted only for ids whose recent bit is set
  // (every other live id is visible to every search).
  uint32_t *d_born = nullptr;      // cap
  uint32_t *d_died = nullptr;      // cap
  uint32_t *d_recent = nullptr;    // cap/32 bitmap words
  uint32_t *d_err = nullptr;       // sticky device error bits
  uint64_t *d_live_count = nullptr;  // live_count, kept on the device for the searches
  uint32_t *d_coord_len = nullptr;   // n: live postings per coordinate, |I[j]|
  uint64_t cap = 0;                // id capacity = tiles_cap * T

  // ---- host mirror
  std::vector<uint8_t> live;        // per id: 1 live, 2 deleted at a sequence number
                                    // but its postings kept (sinn_delete_at), 0 free
  std::vector<uint32_t> nnz;        // per id: stored entries of the live vector
  std::vector<uint8_t> recent;      // per id: its recent bit is set on the device
  std::priority_queue<uint32_t, std::vector<uint32_t>, std::greater<uint32_t>> free_ids;
  uint64_t next_id = 0, live_count = 0;  // live_count: ids with postings (live != 0)
  std::vector<uint16_t *> tile_post;     // 2 per tile: each copy's storage (device)
  std::vector<uint64_t> tile_post_cap;   // 2 per tile: storage words of each copy
  std::vector<uint8_t> tile_sel;         // per tile: the copy searches read
  std::vector<uint32_t> tile_flip_seq;   // per tile: sequence number of the insert that
                                         // made that copy current (0: stream-ordered)
  std::vector<uint64_t> tile_post_len;   // per tile: postings of the current copy
                                         // (tombstones included)
  std::vector<uint64_t> tile_nnz;        // sum of nnz over live vectors of the tile
  std::vector<uint64_t> tile_tombs;      // tombstoned postings per tile
  uint64_t tombstones = 0;
  // sequence-numbered mutations (sinn_insert_at, sinn_delete_at, sinn_reclaim)
  bool snapshots = false;   // a sequence-numbered mutation was made: searches check
                            // the snapshot words (set once, never cleared)
  uint32_t reclaimed = 0;   // every search at a smaller sequence number has finished
  std::vector<std::pair<uint32_t, uint32_t>> pending_del;  // (died, id), postings kept
  std::vector<std::pair<uint32_t, uint32_t>> recent_ins;   // (born, id), recent bit set
  // Bumped whenever a recorded search (sinn_plan) would go stale: device
  // arrays reallocated, the tiles in use or the tuning changed.
  uint64_t shape_version = 0;

  // ---- scratch (search and insert), grow-only
  void *scratch = nullptr;
  size_t scratch_size = 0;
  void *iscratch = nullptr;
  size_t iscratch_size = 0;
  // pinned host staging
  void *pinned = nullptr;
  size_t pinned_size = 0;
  // device staging for sinn_search_host
  void *hstage = nullptr;
  size_t hstage_size = 0;

  // ---- timing (sinn_timing_start/stop)
  bool tm_on = false;
  struct Span {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Span> tm_spans;
  std::vector<cudaEvent_t> tm_pool;
  double tm_acc_ms[SINN_PHASES] = {};      // phases timed inside replayed graphs
  uint64_t tm_acc_spans[SINN_PHASES] = {};
  uint64_t launches = 0;
};

// Brackets one phase with CUDA events when timing is on.
struct SinnPhase {
  sinn_index *ix;
  cudaStream_t s;
  int phase;
  cudaEvent_t a = nullptr;
  SinnPhase(sinn_index *ix_, cudaStream_t s_, int ph);
  ~SinnPhase();
};

// Makes `dev` the calling thread's current device for the scope of an ABI
// call and restores the caller's device on the way out (every return path),
// so a host thread that drives several GPUs keeps its own current device.
struct SinnDevice {
  int prev = -1;
  explicit SinnDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~SinnDevice() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  SinnDevice(const SinnDevice &) = delete;
  SinnDevice &operator=(const SinnDevice &) = delete;
};

// host helpers shared across translation units
// Every device and pinned-host allocation of the library goes through these,
// so that a test can make the n-th next one fail (sinn_debug_fail_alloc).
cudaError_t sinn_dev_malloc(void **p, size_t bytes);
cudaError_t sinn_dev_malloc_async(void **p, size_t bytes, cudaStream_t s);
cudaError_t sinn_host_malloc(void **p, size_t bytes);
int sinn_ensure_scratch(sinn_index *ix, size_t bytes);
int sinn_ensure_pinned(sinn_index *ix, size_t bytes);
int sinn_check_cuda(cudaError_t e);

struct sinn_ctx;
// sinn_search with a per-query k' (k_prime null: k_prime_max for every query)
// and a per-query Alg. 6 budget in postings (budget null: the index's), on a
// context's scratch (c) or, c null, the index's own (search.cu).
int sinn_search_ext(sinn_index *ix, sinn_ctx *c, const uint64_t *q_indptr,
                    const uint32_t *q_indices, const float *q_values, uint32_t n_q, uint32_t k,
                    const uint32_t *k_prime, uint32_t k_prime_max, const uint64_t *budget,
                    uint32_t *out_ids, float *out_scores, cudaStream_t s);

// ---------------------------------------------------------- device helpers
// Order-preserving map from float to uint32 (for all non-NaN values: a < b as
// floats iff key(a) < key(b) as unsigned integers).
__device__ __forceinline__ uint32_t sinn_f2key(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float sinn_key2f(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}

// bfloat16 bins: the floats whose 16 low bits are zero.  An upper bin takes
// the least bfloat16 at or above x, a lower bin the greatest at or below it
// (toward zero is up for a negative x and down for a positive one).
__device__ __forceinline__ uint16_t sinn_bf16_dir(float x, bool up) {
  const uint32_t b = __float_as_uint(x);
  uint32_t t = b >> 16;
  if (b & 0xFFFFu) {
    const bool toward_zero_ok = (b >> 31) ? up : !up;
    if (!toward_zero_ok) t += 1u;  // one bfloat16 step away from zero
  }
  return (uint16_t)t;
}

__device__ __forceinline__ float sinn_bf16_f(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }
__device__ __forceinline__ bool sinn_is_live(const uint32_t *live, uint64_t id) {
  return (__ldg(live + (id >> 5)) >> (id & 31)) & 1u;
}

// A load from L2 that the compiler neither caches nor moves ahead of the
// code that decides to make it: the snapshot words are written by mutations
// that may run while a search does.  Taken only after the id's live bit was
// seen set, it sees the visibility words that the mutation wrote before it
// set that bit (they were written by an earlier kernel of its stream).
__device__ __forceinline__ uint32_t sinn_ld_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Whether a search at sequence number seq counts a live id whose recent bit
// (bit of rwv, the id's recent-bitmap word) is set: only when
// born <= seq < died.  Ids whose recent bit is clear count for every search.
__device__ __forceinline__ bool sinn_visible_recent(const uint32_t *born, const uint32_t *died,
                                                    uint32_t seq, uint64_t id) {
  return sinn_ld_gpu(born + id) <= seq && seq < sinn_ld_gpu(died + id);
}
