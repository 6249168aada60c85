// Learned per-query k' (the paper's Sec. 5.3 / Sec. 7 suggestion that k' be
// chosen per query from the expected approximation error): query features,
// a 2-hidden-layer MLP with BF16 tensor-core GEMMs (FP32 accumulation), its
// training step (pinball loss, Adam) and a search that uses its prediction.
//
// GEMMs run on the 5th-generation tensor cores (tcgen05.mma, bf16 inputs,
// fp32 accumulators in tensor memory) on 128x128 tiles staged through shared
// memory; operands are read through arbitrary (row, column) strides, so the
// same kernel computes X W^T, dY W and dY^T X.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/sinnamon_kprime.h"
#include "sinn_internal.cuh"

#define CK(x)                                          \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) return sinn_check_cuda(e_); \
  } while (0)

namespace {


struct GemmArgs {
  // C[m][n] = alpha * sum_k A(m,k) B(n,k) (+ bias[n]) (ReLU) ; A, B bf16
  const __nv_bfloat16 *A;
  int64_t sam, sak;
  const __nv_bfloat16 *B;
  int64_t sbn, sbk;
  int M, N, K;
  float alpha;
  const float *bias;        // nullable, per n
  int relu;                 // 1: max(0, .)
  float *C;                 // nullable fp32 out, row stride ldc
  int64_t ldc;
  __nv_bfloat16 *Cb;        // nullable bf16 out, row stride ldcb
  int64_t ldcb;
  const float *mask;        // nullable: multiply by (mask[m*ldm+n] > 0)
  int64_t ldm;
  uint32_t *err;            // device error word: SINN_DERR_TIMEOUT if a wait ran out
};

// ---------------------------------------------------------------- GEMM
// C = alpha * A B^T on the 5th-generation tensor cores: one 128x128 output
// tile per CTA of 128 threads.  For each 64-wide slice of K the threads stage
// A (128 x 64) and B (128 x 64) in shared memory in the canonical K-major
// layout without swizzle -- core matrices of 8 rows x 16 bytes, 128 bytes
// apart along K and 1024 bytes apart along M (N) -- and one thread issues four
// tcgen05.mma (M = 128, N = 128, K = 16, bf16 in, fp32 accumulate) into a
// 128-column tensor-memory accumulator, committing to an mbarrier that the
// CTA waits on before it overwrites the operands.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes = rows 32w..32w+31).
// Every wait is bounded: on a timeout the CTA sets SINN_DERR_TIMEOUT in the
// caller's error word, still waits (bounded) for its MMAs and frees its
// tensor memory.
constexpr int TC_M = 128, TC_N = 128, TC_K = 64;
constexpr uint32_t kTcSpin = 1u << 24;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of a rows x 64 K-major tile.
__device__ __forceinline__ uint32_t tc_off(uint32_t r, uint32_t k) {
  return ((r >> 3) * (TC_K / 8) + (k >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// Shared-memory matrix descriptor (no swizzle): start, leading byte offset
// (between core matrices along K), stride byte offset (along M / N), the
// descriptor version 1 in bits 46-47.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = (TC_K / 8) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((lbo >> 4) & 0x3FFFu) << 16 |
         ((sbo >> 4) & 0x3FFFu) << 32 | (uint64_t)1 << 46;
}

// Instruction descriptor, kind::f16: fp32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          uint32_t spins = kTcSpin) {
  for (uint32_t it = 0; it < spins; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g) {
  __shared__ __align__(1024) uint8_t As[TC_M * TC_K * 2];
  __shared__ __align__(1024) uint8_t Bs[TC_N * TC_K * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem, s_fail;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {  // tensor memory: 128 fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"((uint32_t)TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = s_tmem;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  uint32_t phase = 0, issued = 0;
  for (int k0 = 0; k0 < g.K; k0 += TC_K) {
    // stage the slice (zeros beyond M, N, K)
    for (int e = tid; e < TC_M * TC_K; e += 128) {
      const int r = e / TC_K, c = e % TC_K;
      const int m = m0 + r, n = n0 + r, k = k0 + c;
      *(__nv_bfloat16 *)(As + tc_off(r, c)) =
          (m < g.M && k < g.K) ? g.A[m * g.sam + k * g.sak] : zero;
      *(__nv_bfloat16 *)(Bs + tc_off(r, c)) =
          (n < g.N && k < g.K) ? g.B[n * g.sbn + k * g.sbk] : zero;
    }
    // generic-proxy writes become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int s = 0; s < TC_K / 16; ++s) {
        const uint64_t da = tc_desc(smem_u32(As) + s * 256);  // 2 core matrices along K
        const uint64_t db = tc_desc(smem_u32(Bs) + s * 256);
        const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              mb)
          : "memory");
    }
    issued++;
    // the MMAs have read the operands before they are overwritten
    if (!mbar_wait(mb, phase)) {
      if (tid == 0) atomicOr(g.err, SINN_DERR_TIMEOUT);
      s_fail = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (s_fail) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!s_fail && issued > 0) {
    // warp w reads rows 32w + lane, 32 columns at a time
    const uint32_t row = warp * 32 + (tid & 31);
    const int m = m0 + (int)row;
    for (int c0 = 0; c0 < TC_N; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c0 + j;
          if (n >= g.N) continue;
          float x = g.alpha * __uint_as_float(v[j]);
          if (g.bias) x += g.bias[n];
          if (g.mask && !(g.mask[m * g.ldm + n] > 0.0f)) x = 0.0f;
          if (g.relu) x = fmaxf(x, 0.0f);
          if (g.C) g.C[m * g.ldc + n] = x;
          if (g.Cb) g.Cb[m * g.ldcb + n] = __float2bfloat16(x);
        }
      }
    }
  } else if (s_fail && tid == 0) {
    // wait (bounded) for the MMAs still in flight before the memory goes
    (void)mbar_wait(mb, phase ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)TC_N)
                 : "memory");
}

// A bounded wait on an mbarrier that nothing completes (arrive = 0) or that
// the block completes itself first (arrive = 1): the GEMM's timeout path,
// run alone.  A wait that runs out sets SINN_DERR_TIMEOUT in *err.
__global__ void k_wait_probe(uint32_t spins, int arrive, uint32_t *err) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t mb = smem_u32(&bar);
  if (threadIdx.x == 0)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mb)
                 : "memory");
  __syncthreads();
  if (!mbar_wait(mb, 0u, spins) && threadIdx.x == 0) atomicOr(err, SINN_DERR_TIMEOUT);
}

void gemm(const GemmArgs &g, cudaStream_t s) {
  dim3 grid((g.N + TC_N - 1) / TC_N, (g.M + TC_M - 1) / TC_M);
  k_gemm_tc<<<grid, 128, 0, s>>>(g);
}

// Features -> normalised bf16 inputs (padded to K columns with zeros).
__global__ void k_normalise(const float *X, uint32_t B, uint32_t nin, uint32_t kpad,
                            const float *mean, const float *inv_std, __nv_bfloat16 *Xb) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= (uint64_t)B * kpad) return;
  const uint32_t r = (uint32_t)(i / kpad), c = (uint32_t)(i % kpad);
  const float v = c < nin ? (X[(uint64_t)r * nin + c] - mean[c]) * inv_std[c] : 0.0f;
  Xb[i] = __float2bfloat16(v);
}

// y[r] = sum_c H[r][c] w[c] + b (one warp per row), fp32.
__global__ void k_head(const float *H, uint32_t B, uint32_t hdim, const float *w, const float *b,
                       float *y) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (r >= B) return;
  float s = 0.0f;
  for (uint32_t c = lane; c < hdim; c += 32) s = fmaf(H[r * hdim + c], w[c], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) y[r] = s + b[0];
}

// Pinball loss at quantile tau: dL/dy = (1[t < y] - tau) / B; also the loss.
__global__ void k_pinball(const float *y, const float *t, uint32_t B, float tau, float *dy,
                          float *loss) {
  __shared__ float part[32];
  float l = 0.0f;
  for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) {
    const float u = t[i] - y[i];
    l += u >= 0.0f ? tau * u : (tau - 1.0f) * u;
    dy[i] = ((u < 0.0f ? 1.0f : 0.0f) - tau) / (float)B;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) s += part[w];
    if (loss) *loss = s / (float)B;
  }
}

// dH2[r][c] = dy[r] w3[c] masked by Z2 > 0 (as fp32 and bf16); dw3[c] and
// db3 are reduced by k_colsum.
__global__ void k_head_back(const float *dy, const float *w3, const float *H2, uint32_t B,
                            uint32_t hdim, float *dZ2, __nv_bfloat16 *dZ2b) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= (uint64_t)B * hdim) return;
  const uint32_t r = (uint32_t)(i / hdim), c = (uint32_t)(i % hdim);
  const float v = H2[i] > 0.0f ? dy[r] * w3[c] : 0.0f;
  dZ2[i] = v;
  dZ2b[i] = __float2bfloat16(v);
}

// out[c] = sum_r X[r][c] * (s ? s[r] : 1) over rows (column sums), fp32.
__global__ void k_colsum(const float *X, const float *s, uint32_t B, uint32_t cols, float *out) {
  const uint32_t c = blockIdx.x * blockDim.y + threadIdx.y;
  if (c >= cols) return;
  float a = 0.0f;
  for (uint32_t r = threadIdx.x; r < B; r += 32) a += X[(uint64_t)r * cols + c] * (s ? s[r] : 1.0f);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
  if (threadIdx.x == 0) out[c] = a;
}

__global__ void k_sum(const float *x, uint32_t n, float *out) {
  __shared__ float part[32];
  float a = 0.0f;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) a += x[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) s += part[w];
    *out = s;
  }
}

// Adam on all parameters (flat), then refresh the bf16 copies.
__global__ void k_adam(float *p, const float *g, float *m1, float *m2, uint64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// bf16 copies of W1 (hid x kpad, zero-padded columns), W2 (hid x hid) and
// W2^T (for dH1 = dZ2 W2 as a row-major-by-row operand).
__global__ void k_weights_bf16(const float *W1, const float *W2, uint32_t nin, uint32_t kpad,
                               uint32_t hid, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b,
                               __nv_bfloat16 *W2tb) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < (uint64_t)hid * kpad) {
    const uint32_t r = (uint32_t)(i / kpad), c = (uint32_t)(i % kpad);
    W1b[i] = __float2bfloat16(c < nin ? W1[(uint64_t)r * nin + c] : 0.0f);
  }
  if (i < (uint64_t)hid * hid) {
    const uint32_t r = (uint32_t)(i / hid), c = (uint32_t)(i % hid);
    W2b[i] = __float2bfloat16(W2[i]);
    W2tb[(uint64_t)c * hid + r] = __float2bfloat16(W2[i]);
  }
}

// Per-query features: nnz, L1, L2 of the non-zeros, then log2(1 + |I[j]|)
// for the 16 terms of largest |q_j| (ties by j), 0 where fewer.  |I[j]| is
// summed over the tiles' containers (tombstones included).
__global__ void k_features(const uint64_t *__restrict__ ip, const uint32_t *__restrict__ idx,
                           const float *__restrict__ val, uint32_t n, const uint2 *tile_dir,
                           const uint32_t *tile_sel, uint32_t tiles, float *out) {
  const uint32_t q = blockIdx.x, tid = threadIdx.x;
  __shared__ uint32_t sj[SINN_KP_TOP];
  __shared__ float red[3][32];
  __shared__ uint32_t s_top;
  const uint64_t s = ip[q], e = ip[q + 1];
  float c0 = 0.0f, l1 = 0.0f, l2 = 0.0f;
  for (uint64_t p = s + tid; p < e; p += blockDim.x) {
    const float v = val[p];
    if (v == 0.0f || !isfinite(v) || idx[p] >= n) continue;
    c0 += 1.0f;
    l1 += fabsf(v);
    l2 += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, o);
    l1 += __shfl_xor_sync(0xFFFFFFFFu, l1, o);
    l2 += __shfl_xor_sync(0xFFFFFFFFu, l2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = c0;
    red[1][tid >> 5] = l1;
    red[2][tid >> 5] = l2;
  }
  if (tid == 0) s_top = 0;
  __syncthreads();
  // top terms by rank counting (|v| desc, j asc)
  for (uint64_t p = s + tid; p < e; p += blockDim.x) {
    const float v = val[p];
    const uint32_t j = idx[p];
    if (v == 0.0f || !isfinite(v) || j >= n) continue;
    uint32_t r = 0;
    for (uint64_t t = s; t < e && r < SINN_KP_TOP; ++t) {
      const float w = val[t];
      if (w == 0.0f || !isfinite(w) || idx[t] >= n) continue;
      r += (fabsf(w) > fabsf(v)) || (fabsf(w) == fabsf(v) && idx[t] < j);
    }
    if (r < SINN_KP_TOP) {
      sj[r] = j;
      atomicMax(&s_top, r + 1);
    }
  }
  __syncthreads();
  float *o = out + (uint64_t)q * SINN_KP_FEATURES;
  if (tid == 0) {
    float a = 0.0f, b = 0.0f, c = 0.0f;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
    }
    o[0] = log2f(1.0f + a);
    o[1] = b;
    o[2] = sqrtf(c);
  }
  // list lengths: warp w sums term w over tiles
  const uint32_t lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (uint32_t r = wid; r < SINN_KP_TOP; r += nw) {
    float f = 0.0f;
    if (r < s_top) {
      uint64_t cnt = 0;
      for (uint32_t t = lane; t < tiles; t += 32)  // each tile's current copy
        cnt += tile_dir[((uint64_t)t * 2 + __ldcg(tile_sel + t)) * n + sj[r]].y;
      for (int s2 = 16; s2 > 0; s2 >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, s2);
      f = log2f(1.0f + (float)cnt);
    }
    if (lane == 0) o[3 + r] = f;
  }
}

// k'[q] = clamp(ceil(2^y[q]), lo, hi)
__global__ void k_kprime(const float *y, uint32_t B, uint32_t lo, uint32_t hi, uint32_t *kp) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float v = exp2f(fminf(fmaxf(y[i], 0.0f), 31.0f));
  kp[i] = min(max((uint32_t)ceilf(v), lo), hi);
}

// Network inputs of the budget levels: row q*L + l is query q's features
// followed by the level's input, -shift[l] (log2 of its budget fraction).
__global__ void k_level_rows(const float *F, uint32_t n_q, uint32_t L, sinn_kp_policy pol,
                             float *X) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  constexpr uint32_t NI = SINN_KP_FEATURES + 1;
  if (i >= (uint64_t)n_q * L * NI) return;
  const uint64_t row = i / NI;
  const uint32_t c = (uint32_t)(i % NI);
  const uint64_t q = row / L;
  const uint32_t l = (uint32_t)(row % L);
  X[i] = c < SINN_KP_FEATURES ? F[q * SINN_KP_FEATURES + c] : -(float)pol.shift[l];
}

// The policy's choice per query (one thread each).  Level l scores the terms
// of Alg. 6 until ceil(P_q / 2^shift[l]) postings are reached and needs
// k'_l = ceil(2^(y[q*L+l] + margin)) (at least lo); it is feasible when
// k'_l <= hi.  The feasible level of least cost posting_cost * postings +
// k'_l wins (ties: the earlier level, the larger budget); with none
// feasible, level 0 (the whole query) at k' = hi.  Budget 0 means the whole
// query (no break).
__global__ void k_policy(const float *y, const uint64_t *P, uint32_t n_q, sinn_kp_policy pol,
                         uint32_t lo, uint32_t hi, uint32_t *kp, uint64_t *budget) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_q) return;
  const uint64_t pq = P[q];
  int best = -1;
  float best_cost = 0.0f;
  uint32_t best_kp = hi;
  for (uint32_t l = 0; l < pol.n_levels; ++l) {
    const float v = fminf(fmaxf(y[(uint64_t)q * pol.n_levels + l] + pol.margin, 0.0f), 31.0f);
    const float need = ceilf(exp2f(v));
    if (need > (float)hi) continue;
    const uint32_t k_l = max((uint32_t)need, lo);
    const uint32_t sh = pol.shift[l];
    const uint64_t b = sh ? (pq + (1ull << sh) - 1) >> sh : pq;
    const float cost = fmaf(pol.posting_cost, (float)b, (float)k_l);
    if (best < 0 || cost < best_cost) {
      best = (int)l;
      best_cost = cost;
      best_kp = k_l;
    }
  }
  const uint32_t sh = best < 0 ? 0u : pol.shift[best];
  kp[q] = best_kp;
  budget[q] = sh ? (pq + (1ull << sh) - 1) >> sh : 0ull;
}

}  // namespace

// ------------------------------------------------------------------ model
struct sinn_mlp {
  uint32_t nin = 0, hid = 0, kpad = 0;
  int device = 0;
  uint64_t nparams = 0;
  float *d_p = nullptr;   // flat params: W1 (hid x nin), b1, W2 (hid x hid), b2, w3, b3
  float *d_g = nullptr;   // gradients, same layout
  float *d_m1 = nullptr, *d_m2 = nullptr;
  float *d_mean = nullptr, *d_istd = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr;
  uint32_t *d_err = nullptr;  // device error bits of sinn_mlp_forward / _grad / _train_step
  uint64_t steps = 0;
  // activations (grow-only)
  uint32_t cap = 0;
  void *act = nullptr;
  bool bf16_fresh = false;
  // budget levels (n_levels = 0: none; the network then predicts k' alone)
  sinn_kp_policy policy{};
  uint64_t version = 0;  // bumped when the policy changes (recorded searches)
};

namespace {

struct Views {
  float *W1, *b1, *W2, *b2, *w3, *b3;
};

Views views(sinn_mlp *m, float *base) {
  Views v;
  v.W1 = base;
  v.b1 = v.W1 + (uint64_t)m->hid * m->nin;
  v.W2 = v.b1 + m->hid;
  v.b2 = v.W2 + (uint64_t)m->hid * m->hid;
  v.w3 = v.b2 + m->hid;
  v.b3 = v.w3 + m->hid;
  return v;
}

struct Acts {
  __nv_bfloat16 *Xb, *H1b, *dZ2b, *dZ1b;
  float *Z1, *H2, *y, *dy, *dZ2, *dH1, *loss;
};

// Carve activation buffers for up to cap rows from base (see acts_bytes).
size_t acts_bytes(const sinn_mlp *m, size_t c) {
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  return r(c * m->kpad * 2) + 3 * r(c * m->hid * 2) + 4 * r(c * m->hid * 4) + 2 * r(c * 4) +
         r(64);
}

void carve_acts(const sinn_mlp *m, void *base, size_t c, Acts *a) {
  char *p = (char *)base;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  a->Xb = (__nv_bfloat16 *)take(c * m->kpad * 2);
  a->H1b = (__nv_bfloat16 *)take(c * m->hid * 2);
  a->dZ2b = (__nv_bfloat16 *)take(c * m->hid * 2);
  a->dZ1b = (__nv_bfloat16 *)take(c * m->hid * 2);
  a->Z1 = (float *)take(c * m->hid * 4);
  a->H2 = (float *)take(c * m->hid * 4);
  a->dZ2 = (float *)take(c * m->hid * 4);
  a->dH1 = (float *)take(c * m->hid * 4);
  a->y = (float *)take(c * 4);
  a->dy = (float *)take(c * 4);
  a->loss = (float *)take(64);
}

int ensure_acts(sinn_mlp *m, uint32_t B, Acts *a) {
  if (B > m->cap) {
    if (m->act) {
      CK(cudaDeviceSynchronize());
      CK(cudaFree(m->act));
      m->act = nullptr;
    }
    const uint32_t c = std::max<uint32_t>(B, 1024);
    CK(sinn_dev_malloc((void **)&m->act, acts_bytes(m, c)));
    m->cap = c;
  }
  carve_acts(m, m->act, m->cap, a);
  return SINN_OK;
}

int refresh_bf16(sinn_mlp *m, cudaStream_t s) {
  if (m->bf16_fresh) return SINN_OK;
  Views v = views(m, m->d_p);
  const uint64_t n = std::max<uint64_t>((uint64_t)m->hid * m->kpad, (uint64_t)m->hid * m->hid);
  k_weights_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v.W1, v.W2, m->nin, m->kpad, m->hid,
                                                            m->W1b, m->W2b, m->W2tb);
  CK(cudaGetLastError());
  m->bf16_fresh = true;
  return SINN_OK;
}

// Forward through the network for B rows of raw features X; leaves the
// activations in a (needed by the backward pass).
int forward(sinn_mlp *m, const float *X, uint32_t B, Acts &a, cudaStream_t s, uint32_t *err) {
  int st = refresh_bf16(m, s);
  if (st) return st;
  Views v = views(m, m->d_p);
  const uint64_t nx = (uint64_t)B * m->kpad;
  k_normalise<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(X, B, m->nin, m->kpad, m->d_mean,
                                                          m->d_istd, a.Xb);
  GemmArgs g{};
  // Z1 = X W1^T + b1 ; H1 = relu(Z1)
  g.A = a.Xb; g.sam = m->kpad; g.sak = 1;
  g.B = m->W1b; g.sbn = m->kpad; g.sbk = 1;
  g.M = (int)B; g.N = (int)m->hid; g.K = (int)m->kpad; g.alpha = 1.0f;
  g.bias = v.b1; g.relu = 0; g.C = a.Z1; g.ldc = m->hid; g.Cb = nullptr; g.err = err;
  gemm(g, s);
  GemmArgs r = g;  // H1 (bf16) = relu(Z1)
  r.relu = 1; r.C = nullptr; r.Cb = a.H1b; r.ldcb = m->hid;
  gemm(r, s);
  // H2 = relu(H1 W2^T + b2)
  GemmArgs g2{};
  g2.A = a.H1b; g2.sam = m->hid; g2.sak = 1;
  g2.B = m->W2b; g2.sbn = m->hid; g2.sbk = 1;
  g2.M = (int)B; g2.N = (int)m->hid; g2.K = (int)m->hid; g2.alpha = 1.0f;
  g2.bias = v.b2; g2.relu = 1; g2.C = a.H2; g2.ldc = m->hid; g2.err = err;
  gemm(g2, s);
  k_head<<<(B + 7) / 8, 256, 0, s>>>(a.H2, B, m->hid, v.w3, v.b3, a.y);
  CK(cudaGetLastError());
  return SINN_OK;
}

// Gradients of the mean pinball loss into m->d_g.
int backward(sinn_mlp *m, const float *t, uint32_t B, float tau, Acts &a, cudaStream_t s,
             uint32_t *err) {
  Views v = views(m, m->d_p);
  Views gv = views(m, m->d_g);
  k_pinball<<<1, 1024, 0, s>>>(a.y, t, B, tau, a.dy, a.loss);
  // head: dw3 = H2^T dy ; db3 = sum dy ; dZ2 = dy w3 * 1[H2 > 0]
  k_colsum<<<(m->hid + 7) / 8, dim3(32, 8), 0, s>>>(a.H2, a.dy, B, m->hid, gv.w3);
  k_sum<<<1, 1024, 0, s>>>(a.dy, B, gv.b3);
  const uint64_t nh = (uint64_t)B * m->hid;
  k_head_back<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(a.dy, v.w3, a.H2, B, m->hid, a.dZ2,
                                                          a.dZ2b);
  // dW2 = dZ2^T H1 (hid x hid, reduction over rows) ; db2 = colsum dZ2
  GemmArgs g{};
  g.A = a.dZ2b; g.sam = 1; g.sak = m->hid;       // A(n_out, r) = dZ2[r][n_out]
  g.B = a.H1b; g.sbn = 1; g.sbk = m->hid;        // B(n_in, r) = H1[r][n_in]
  g.M = (int)m->hid; g.N = (int)m->hid; g.K = (int)B; g.alpha = 1.0f;
  g.C = gv.W2; g.ldc = m->hid; g.err = err;
  gemm(g, s);
  k_colsum<<<(m->hid + 7) / 8, dim3(32, 8), 0, s>>>(a.dZ2, nullptr, B, m->hid, gv.b2);
  // dH1 = dZ2 W2 (B x hid) masked by Z1 > 0 -> dZ1 ; B(n, k) = W2[k][n] = W2t[n][k]
  GemmArgs h{};
  h.A = a.dZ2b; h.sam = m->hid; h.sak = 1;
  h.B = m->W2tb; h.sbn = m->hid; h.sbk = 1;
  h.M = (int)B; h.N = (int)m->hid; h.K = (int)m->hid; h.alpha = 1.0f;
  h.mask = a.Z1; h.ldm = m->hid;
  h.C = a.dH1; h.ldc = m->hid; h.Cb = a.dZ1b; h.ldcb = m->hid; h.err = err;
  gemm(h, s);
  // dW1 = dZ1^T X (hid x nin) ; db1 = colsum dZ1
  GemmArgs w{};
  w.A = a.dZ1b; w.sam = 1; w.sak = m->hid;
  w.B = a.Xb; w.sbn = 1; w.sbk = m->kpad;
  w.M = (int)m->hid; w.N = (int)m->nin; w.K = (int)B; w.alpha = 1.0f;
  w.C = gv.W1; w.ldc = m->nin; w.err = err;
  gemm(w, s);
  k_colsum<<<(m->hid + 7) / 8, dim3(32, 8), 0, s>>>(a.dH1, nullptr, B, m->hid, gv.b1);
  CK(cudaGetLastError());
  return SINN_OK;
}

uint64_t splitmix_next(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

// The network's bf16 weight copies made current (no work when they are);
// used by recorded searches, which replay a graph without this check.
int sinn_mlp_refresh(sinn_mlp *m, cudaStream_t s) { return refresh_bf16(m, s); }

extern "C" int sinn_mlp_create(uint32_t n_in, uint32_t hidden, uint64_t seed, sinn_mlp **out) {
  if (!out) return SINN_EINVAL;
  *out = nullptr;
  if (n_in == 0 || hidden == 0 || hidden > 4096 || n_in > 1024) return SINN_EINVAL;
  sinn_mlp *m = new (std::nothrow) sinn_mlp();
  if (!m) return SINN_ENOMEM;
  cudaGetDevice(&m->device);
  m->nin = n_in;
  m->hid = hidden;
  m->kpad = (n_in + 15) / 16 * 16;
  m->nparams = (uint64_t)hidden * n_in + hidden + (uint64_t)hidden * hidden + hidden + hidden + 1;
  std::vector<float> p(m->nparams, 0.0f), ones(n_in, 1.0f), zeros(n_in, 0.0f);
  uint64_t s = seed ? seed : 0x5151;
  auto uni = [&](float bound) {  // uniform in [-bound, bound]
    const double u = (double)(splitmix_next(s) >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * bound);
  };
  Views v = views(m, p.data());
  for (uint64_t i = 0; i < (uint64_t)hidden * n_in; ++i) v.W1[i] = uni(sqrtf(6.0f / n_in));
  for (uint64_t i = 0; i < (uint64_t)hidden * hidden; ++i) v.W2[i] = uni(sqrtf(6.0f / hidden));
  for (uint32_t i = 0; i < hidden; ++i) v.w3[i] = uni(sqrtf(3.0f / hidden));
  int st = SINN_OK;
  auto fail = [&](int e) {
    sinn_mlp_destroy(m);
    return e;
  };
  const size_t pb = m->nparams * 4;
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_p, pb)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_g, pb)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_m1, pb)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_m2, pb)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_mean, n_in * 4)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_istd, n_in * 4)))) return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->W1b, (size_t)hidden * m->kpad * 2))))
    return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->W2b, (size_t)hidden * hidden * 2))))
    return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->W2tb, (size_t)hidden * hidden * 2))))
    return fail(st);
  if ((st = sinn_check_cuda(sinn_dev_malloc((void **)&m->d_err, 4)))) return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(m->d_err, 0, 4)))) return fail(st);
  if ((st = sinn_check_cuda(cudaMemcpy(m->d_p, p.data(), pb, cudaMemcpyHostToDevice))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(m->d_g, 0, pb)))) return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(m->d_m1, 0, pb)))) return fail(st);
  if ((st = sinn_check_cuda(cudaMemset(m->d_m2, 0, pb)))) return fail(st);
  if ((st = sinn_check_cuda(cudaMemcpy(m->d_mean, zeros.data(), n_in * 4, cudaMemcpyHostToDevice))))
    return fail(st);
  if ((st = sinn_check_cuda(cudaMemcpy(m->d_istd, ones.data(), n_in * 4, cudaMemcpyHostToDevice))))
    return fail(st);
  *out = m;
  return SINN_OK;
}

extern "C" int sinn_mlp_destroy(sinn_mlp *m) {
  if (!m) return SINN_OK;
  SinnDevice dev_guard_(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->d_p);
  cudaFree(m->d_g);
  cudaFree(m->d_m1);
  cudaFree(m->d_m2);
  cudaFree(m->d_mean);
  cudaFree(m->d_istd);
  cudaFree(m->W1b);
  cudaFree(m->W2b);
  cudaFree(m->W2tb);
  cudaFree(m->act);
  cudaFree(m->d_err);
  delete m;
  return SINN_OK;
}

extern "C" uint64_t sinn_mlp_num_params(sinn_mlp *m) { return m ? m->nparams : 0; }

extern "C" int sinn_mlp_sync(sinn_mlp *m, void *stream) {
  if (!m) return SINN_EINVAL;
  SinnDevice dev_guard_(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t bits = 0;
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(&bits, m->d_err, 4, cudaMemcpyDeviceToHost));
  if (bits) CK(cudaMemset(m->d_err, 0, 4));
  return bits ? SINN_EDEVICE : SINN_OK;
}

extern "C" int sinn_debug_wait_probe(uint32_t spins, int arrive, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *d = nullptr, bits = 0;
  CK(sinn_dev_malloc((void **)&d, 4));
  int st = sinn_check_cuda(cudaMemsetAsync(d, 0, 4, s));
  if (!st) {
    k_wait_probe<<<1, 32, 0, s>>>(spins, arrive ? 1 : 0, d);
    st = sinn_check_cuda(cudaGetLastError());
  }
  if (!st) st = sinn_check_cuda(cudaMemcpyAsync(&bits, d, 4, cudaMemcpyDeviceToHost, s));
  if (!st) st = sinn_check_cuda(cudaStreamSynchronize(s));
  cudaFree(d);
  if (st) return st;
  return (bits & SINN_DERR_TIMEOUT) ? SINN_EDEVICE : SINN_OK;
}

extern "C" int sinn_mlp_params(sinn_mlp *m, float *host_out, int which) {
  if (!m || !host_out) return SINN_EINVAL;
  SinnDevice dev_guard_(m->device);
  const float *src = which == 0 ? m->d_p : m->d_g;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(host_out, src, m->nparams * 4, cudaMemcpyDeviceToHost));
  return SINN_OK;
}

extern "C" int sinn_mlp_set_params(sinn_mlp *m, const float *host_in) {
  if (!m || !host_in) return SINN_EINVAL;
  SinnDevice dev_guard_(m->device);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(m->d_p, host_in, m->nparams * 4, cudaMemcpyHostToDevice));
  m->bf16_fresh = false;
  return SINN_OK;
}

extern "C" int sinn_mlp_set_normalizer(sinn_mlp *m, const float *mean, const float *stdev) {
  if (!m || !mean || !stdev) return SINN_EINVAL;
  std::vector<float> is(m->nin);
  for (uint32_t i = 0; i < m->nin; ++i) is[i] = stdev[i] > 0.0f ? 1.0f / stdev[i] : 1.0f;
  SinnDevice dev_guard_(m->device);
  CK(cudaMemcpy(m->d_mean, mean, m->nin * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->d_istd, is.data(), m->nin * 4, cudaMemcpyHostToDevice));
  return SINN_OK;
}

extern "C" int sinn_mlp_forward(sinn_mlp *m, const float *X, uint32_t B, float *y, void *stream) {
  if (!m || (B && (!X || !y))) return SINN_EINVAL;
  if (B == 0) return SINN_OK;
  SinnDevice dev_guard_(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Acts a;
  int st = ensure_acts(m, B, &a);
  if (st) return st;
  if ((st = forward(m, X, B, a, s, m->d_err))) return st;
  CK(cudaMemcpyAsync(y, a.y, (size_t)B * 4, cudaMemcpyDeviceToDevice, s));
  return SINN_OK;
}

extern "C" int sinn_mlp_grad(sinn_mlp *m, const float *X, const float *t, uint32_t B, float tau,
                             float *grad_out, float *loss_out, void *stream) {
  if (!m || B == 0 || !X || !t || tau <= 0.0f || tau >= 1.0f) return SINN_EINVAL;
  SinnDevice dev_guard_(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Acts a;
  int st = ensure_acts(m, B, &a);
  if (st) return st;
  if ((st = forward(m, X, B, a, s, m->d_err))) return st;
  if ((st = backward(m, t, B, tau, a, s, m->d_err))) return st;
  if (grad_out) CK(cudaMemcpyAsync(grad_out, m->d_g, m->nparams * 4, cudaMemcpyDeviceToDevice, s));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, a.loss, 4, cudaMemcpyDeviceToDevice, s));
  return SINN_OK;
}

extern "C" int sinn_mlp_train_step(sinn_mlp *m, const float *X, const float *t, uint32_t B,
                                   float tau, float lr, float *loss_out, void *stream) {
  int st = sinn_mlp_grad(m, X, t, B, tau, nullptr, loss_out, stream);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  m->steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->steps), c2 = 1.0f - powf(b2, (float)m->steps);
  k_adam<<<(unsigned)((m->nparams + 255) / 256), 256, 0, s>>>(m->d_p, m->d_g, m->d_m1, m->d_m2,
                                                            m->nparams, lr, b1, b2, 1e-8f, c1, c2);
  CK(cudaGetLastError());
  m->bf16_fresh = false;
  return SINN_OK;
}

extern "C" int sinn_kp_features(sinn_index *ix, const uint64_t *q_indptr, const uint32_t *q_indices,
                                const float *q_values, uint32_t n_q, float *out, void *stream) {
  if (!ix || (n_q && (!q_indptr || !out))) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  SinnDevice dev_guard_(ix->device);
  k_features<<<n_q, 256, 0, (cudaStream_t)stream>>>(q_indptr, q_indices, q_values, ix->n,
                                                    ix->d_tile_dir, ix->d_tile_sel,
                                                    (uint32_t)(ix->cap / ix->T), out);
  CK(cudaGetLastError());
  return SINN_OK;
}

namespace {

// Rows of the network per query: one per budget level, or one.
uint32_t level_rows(const sinn_mlp *m) { return m->policy.n_levels ? m->policy.n_levels : 1u; }

// Bytes of the activations of n_q queries (their level rows) plus the tail
// the choice uses: features, postings, k' and budgets per query, and the
// expanded network inputs.
size_t learned_bytes(const sinn_mlp *m, uint32_t n_q) {
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t R = (size_t)n_q * level_rows(m);
  return acts_bytes(m, R) + r((size_t)n_q * SINN_KP_FEATURES * 4) + r((size_t)n_q * 8) +
         r((size_t)n_q * 4) + r((size_t)n_q * 8) + r(R * (SINN_KP_FEATURES + 1) * 4);
}

struct Choice {
  uint32_t *kp;
  uint64_t *budget;  // null without a policy
};

// Features, the network and the choice of k' (and with a policy the Alg. 6
// budget) of n_q queries, on activations carved from `base` for their rows.
int choose(sinn_index *ix, sinn_mlp *m, void *base, const uint64_t *q_indptr,
           const uint32_t *q_indices, const float *q_values, uint32_t n_q, uint32_t kp_min,
           uint32_t kp_max, cudaStream_t s, Choice *out) {
  const uint32_t L = level_rows(m);
  const size_t R = (size_t)n_q * L;
  Acts a;
  carve_acts(m, base, R, &a);
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  char *t = (char *)base + acts_bytes(m, R);
  float *feat = (float *)t;
  t += r((size_t)n_q * SINN_KP_FEATURES * 4);
  uint64_t *P = (uint64_t *)t;
  t += r((size_t)n_q * 8);
  out->kp = (uint32_t *)t;
  t += r((size_t)n_q * 4);
  out->budget = m->policy.n_levels ? (uint64_t *)t : nullptr;
  t += r((size_t)n_q * 8);
  float *X = (float *)t;
  int st = sinn_kp_features(ix, q_indptr, q_indices, q_values, n_q, feat, s);
  if (st) return st;
  if ((st = refresh_bf16(m, s))) return st;
  if (!m->policy.n_levels) {
    if ((st = forward(m, feat, n_q, a, s, ix->d_err))) return st;
    k_kprime<<<(n_q + 255) / 256, 256, 0, s>>>(a.y, n_q, kp_min, kp_max, out->kp);
    CK(cudaGetLastError());
    ix->launches += 8;
    return SINN_OK;
  }
  if ((st = sinn_query_postings(ix, q_indptr, q_indices, q_values, n_q, P, s))) return st;
  const uint64_t nx = R * (SINN_KP_FEATURES + 1);
  k_level_rows<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(feat, n_q, L, m->policy, X);
  if ((st = forward(m, X, (uint32_t)R, a, s, ix->d_err))) return st;
  k_policy<<<(n_q + 255) / 256, 256, 0, s>>>(a.y, P, n_q, m->policy, kp_min, kp_max, out->kp,
                                             out->budget);
  CK(cudaGetLastError());
  ix->launches += 9;
  return SINN_OK;
}

// The network's own activation buffer holds learned_bytes(n_q): rows enough
// for the queries' level rows and, past them, the tail (under one row's bytes
// per query).
int ensure_learned(sinn_mlp *m, uint32_t n_q) {
  const uint64_t need = learned_bytes(m, n_q);
  if (m->act && acts_bytes(m, m->cap) >= need) return SINN_OK;
  const uint64_t rows = (uint64_t)n_q * level_rows(m) + n_q + 64;
  if (rows > 0xFFFFFFFFull) return SINN_EINVAL;
  Acts a;
  int st = ensure_acts(m, (uint32_t)rows, &a);
  if (st) return st;
  return acts_bytes(m, m->cap) >= need ? SINN_OK : SINN_ENOMEM;
}

bool learned_args_ok(sinn_index *ix, sinn_mlp *m, uint32_t k, uint32_t kp_min, uint32_t kp_max) {
  if (!ix || !m) return false;
  if (m->nin != SINN_KP_FEATURES + (m->policy.n_levels ? 1u : 0u)) return false;
  if (m->hid < SINN_KP_FEATURES + 1) return false;
  return k > 0 && kp_min >= k && kp_max >= kp_min;
}

}  // namespace

extern "C" int sinn_mlp_set_policy(sinn_mlp *m, const sinn_kp_policy *p) {
  if (!m) return SINN_EINVAL;
  if (!p) {
    m->policy = sinn_kp_policy{};
    m->version++;
    return SINN_OK;
  }
  if (p->n_levels == 0 || p->n_levels > SINN_KP_MAX_LEVELS || p->shift[0] != 0 ||
      !(p->posting_cost >= 0.0f) || !std::isfinite(p->posting_cost) || !std::isfinite(p->margin))
    return SINN_EINVAL;
  for (uint32_t l = 1; l < p->n_levels; ++l)
    if (p->shift[l] <= p->shift[l - 1] || p->shift[l] > 31) return SINN_EINVAL;
  if (m->nin != SINN_KP_FEATURES + 1) return SINN_EINVAL;
  m->policy = *p;
  for (uint32_t l = p->n_levels; l < SINN_KP_MAX_LEVELS; ++l) m->policy.shift[l] = 0;
  m->version++;
  return SINN_OK;
}

extern "C" int sinn_mlp_get_policy(sinn_mlp *m, sinn_kp_policy *out) {
  if (!m || !out) return SINN_EINVAL;
  *out = m->policy;
  return SINN_OK;
}

extern "C" int sinn_kp_choose(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                              const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                              uint32_t k_prime_min, uint32_t k_prime_max, uint32_t *out_kprime,
                              uint64_t *out_budget, void *stream) {
  if (!learned_args_ok(ix, m, 1, k_prime_min, k_prime_max) || k_prime_min == 0)
    return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!q_indptr || !out_kprime) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_learned(m, n_q);
  if (st) return st;
  Choice c;
  if ((st = choose(ix, m, m->act, q_indptr, q_indices, q_values, n_q, k_prime_min, k_prime_max,
                   s, &c)))
    return st;
  CK(cudaMemcpyAsync(out_kprime, c.kp, (size_t)n_q * 4, cudaMemcpyDeviceToDevice, s));
  if (out_budget) {
    if (c.budget) CK(cudaMemcpyAsync(out_budget, c.budget, (size_t)n_q * 8, cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemsetAsync(out_budget, 0, (size_t)n_q * 8, s));
  }
  return SINN_OK;
}

extern "C" int sinn_search_learned(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                                   const uint32_t *q_indices, const float *q_values, uint32_t n_q,
                                   uint32_t k, uint32_t k_prime_min, uint32_t k_prime_max,
                                   uint32_t *out_ids, float *out_scores, uint32_t *out_kprime,
                                   void *stream) {
  if (!learned_args_ok(ix, m, k, k_prime_min, k_prime_max)) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!q_indptr) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_learned(m, n_q);
  if (st) return st;
  Choice c;
  if ((st = choose(ix, m, m->act, q_indptr, q_indices, q_values, n_q, k_prime_min, k_prime_max,
                   s, &c)))
    return st;
  if (out_kprime) CK(cudaMemcpyAsync(out_kprime, c.kp, (size_t)n_q * 4, cudaMemcpyDeviceToDevice, s));
  return sinn_search_ext(ix, nullptr, q_indptr, q_indices, q_values, n_q, k, c.kp, k_prime_max,
                         c.budget, out_ids, out_scores, s);
}

// sinn_search_learned over host buffers: queries copied to the index's
// device staging buffer, searched, results copied back, then a wait.
extern "C" int sinn_search_learned_host(sinn_index *ix, sinn_mlp *m, const uint64_t *q_indptr,
                                        const uint32_t *q_indices, const float *q_values,
                                        uint32_t n_q, uint32_t k, uint32_t k_prime_min,
                                        uint32_t k_prime_max, uint32_t *out_ids,
                                        float *out_scores, uint32_t *out_kprime, void *stream) {
  if (!learned_args_ok(ix, m, k, k_prime_min, k_prime_max) || k > SINN_MAX_K) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!q_indptr || !out_ids || !out_scores) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (q_indptr[n_q] < q_indptr[0]) return SINN_EINVAL;
  const uint64_t nnz = q_indptr[n_q] - q_indptr[0];
  if (nnz && (!q_indices || !q_values)) return SINN_EINVAL;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_ip = al(((size_t)n_q + 1) * 8), b_ix = al(nnz * 4), b_v = al(nnz * 4),
               b_oi = al((size_t)n_q * k * 4), b_os = al((size_t)n_q * k * 4),
               b_kp = al((size_t)n_q * 4);
  const size_t need = b_ip + b_ix + b_v + b_oi + b_os + b_kp;
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
  uint32_t *d_kp = (uint32_t *)(p + b_ip + b_ix + b_v + b_oi + b_os);
  // row pointers rebased to zero on the device side
  std::vector<uint64_t> ip(q_indptr, q_indptr + n_q + 1);
  const uint64_t base = ip[0];
  for (auto &x : ip) x -= base;
  CK(cudaMemcpyAsync(d_ip, ip.data(), ((size_t)n_q + 1) * 8, cudaMemcpyHostToDevice, s));
  if (nnz) {
    CK(cudaMemcpyAsync(d_ix, q_indices + base, nnz * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_v, q_values + base, nnz * 4, cudaMemcpyHostToDevice, s));
  }
  int st = sinn_search_learned(ix, m, d_ip, d_ix, d_v, n_q, k, k_prime_min, k_prime_max, d_oi,
                               d_os, d_kp, stream);
  if (st) {
    cudaStreamSynchronize(s);  // the staged copies must not outlive the host vector
    return st;
  }
  CK(cudaMemcpyAsync(out_ids, d_oi, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(out_scores, d_os, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, s));
  if (out_kprime) CK(cudaMemcpyAsync(out_kprime, d_kp, (size_t)n_q * 4, cudaMemcpyDeviceToHost, s));
  return sinn_sync(ix, stream);
}

// sinn_search_learned on a context: the network's activations come from a
// caller buffer (act, act_bytes) so concurrent contexts share one model.
extern "C" uint64_t sinn_mlp_act_bytes(sinn_mlp *m, uint32_t rows) {
  return m ? learned_bytes(m, rows) + 512 : 0;
}

extern "C" int sinn_search_learned_ctx(sinn_ctx *c, sinn_index *ix, sinn_mlp *m, void *act,
                                       uint64_t act_bytes, const uint64_t *q_indptr,
                                       const uint32_t *q_indices, const float *q_values,
                                       uint32_t n_q, uint32_t k, uint32_t k_prime_min,
                                       uint32_t k_prime_max, uint32_t *out_ids, float *out_scores,
                                       uint32_t *out_kprime, void *stream) {
  if (!c || !act || !learned_args_ok(ix, m, k, k_prime_min, k_prime_max)) return SINN_EINVAL;
  if (n_q == 0) return SINN_OK;
  if (!q_indptr) return SINN_EINVAL;
  if (act_bytes < sinn_mlp_act_bytes(m, n_q)) return SINN_EINVAL;
  SinnDevice dev_guard_(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  Choice ch;
  int st = choose(ix, m, act, q_indptr, q_indices, q_values, n_q, k_prime_min, k_prime_max, s,
                  &ch);
  if (st) return st;
  if (out_kprime) CK(cudaMemcpyAsync(out_kprime, ch.kp, (size_t)n_q * 4, cudaMemcpyDeviceToDevice, s));
  return sinn_search_ext(ix, c, q_indptr, q_indices, q_values, n_q, k, ch.kp, k_prime_max,
                         ch.budget, out_ids, out_scores, s);
}

// The network's version (bumped by a policy change), for recorded searches.
uint64_t sinn_mlp_version(sinn_mlp *m) { return m ? m->version : 0; }
