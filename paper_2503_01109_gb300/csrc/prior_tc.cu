// prior_tc.cu -- inference of the learned seeding prior (an extension of eq11,
// not in the paper) on the fifth-generation tensor cores: tcgen05.mma with the
// operands in shared memory and the FP32 accumulators in tensor memory (TMEM).
//
// One CTA of 16 warps per SM walks tiles of 128 feature rows; the next tile's rows
// stream into shared memory (cp.async) while the current tile's second and third
// layers and epilogues run.  The three layers are three chains of
// tcgen05.mma.cta_group::1.kind::f16 instructions (M = 128 rows, BF16 operands,
// FP32 accumulation in 128 TMEM columns):
//   layer 1: X [128 x 272] W1^T -> 17 MMAs of K = 16, N = 128;
//   layer 2: H1 [128 x 128] W2^T -> 8 MMAs, N = 128;
//   layer 3: H2 [128 x 128] W3^T -> 8 MMAs, N = 16 (W3's 4 output rows padded).
// One thread issues the MMAs and commits them to an mbarrier; every warp then
// reads 32 columns of its 32 TMEM lanes (rows) with tcgen05.ld, adds the bias,
// applies GELU, rounds to BF16 and writes the next layer's operand into shared
// memory (four warps per lane quadrant, so the epilogue runs 16 warps wide).  The
// arithmetic is the one of the mma.sync training kernel (BF16 products, FP32
// sums, BF16 activations), so the outputs agree with it to FP32 summation order.
//
// Operands use the no-swizzle K-major canonical layout: 8x8 "core matrices" of
// BF16 (8 rows of 16 bytes, 128 contiguous bytes), adjacent along K at 128 bytes
// (leading byte offset) and along M / N at (K / 8) * 128 bytes (stride byte
// offset).  A K = 16 step of an MMA covers two core matrices along K.
//
// Every wait is bounded: thread 0 alone polls the mbarrier (the others wait at the
// next __syncthreads); a phase that has not completed after one second sets
// FGS_DEV_TIMEOUT in the status word, and the CTA waits once more (bounded) for
// the chain still in flight, releases its TMEM and returns.
#include <cmath>

#include "common.cuh"

namespace fgs {

namespace tc {

constexpr int kIn = FGS_PRIOR_IN;    // 272
constexpr int kHid = FGS_PRIOR_HID;  // 128
constexpr int kOut = FGS_PRIOR_OUT;  // 4
constexpr int kN3 = 16;              // layer 3's N: the 4 outputs padded to an MMA width
constexpr int kRows = 128;           // M of every MMA: rows per tile
constexpr int kThreads = 512;        // 16 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
                                     // rows) and accumulator columns 32 (w / 4) .. + 31
constexpr int kTmemCols = 128;

// shared-memory carve-up (bytes)
constexpr int kW1Bytes = kHid * kIn * 2;     // 69,632
constexpr int kW2Bytes = kHid * kHid * 2;    // 32,768
constexpr int kW3Bytes = kN3 * kHid * 2;     //  4,096
constexpr int kXBytes = kRows * kIn * 2;     // 69,632 (X)
constexpr int kHBytes = kRows * kHid * 2;    // 32,768 (H1, then H2)
constexpr int kOffW1 = 0;
constexpr int kOffW2 = kOffW1 + kW1Bytes;
constexpr int kOffW3 = kOffW2 + kW2Bytes;
constexpr int kOffX = kOffW3 + kW3Bytes;
constexpr int kOffH = kOffX + kXBytes;
constexpr int kOffBias = kOffH + kHBytes;              // b1 [128], b2 [128], b3 [16] floats
constexpr int kOffBar = kOffBias + (2 * kHid + kN3) * 4;  // mbarrier (8 B) + TMEM address (4 B)
constexpr int kSmemBytes = kOffBar + 16;
static_assert(kSmemBytes <= 227 * 1024, "prior tile must fit in shared memory");
static_assert(kOffX % 1024 == 0 && kOffH % 1024 == 0 && kOffW2 % 1024 == 0, "operand alignment");

constexpr uint64_t kWaitNs = 1000000000ull;  // one second

// Byte offset of element (r, k) of an [R][K] BF16 operand in the canonical layout.
__device__ __forceinline__ uint32_t canon(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset (K
// direction), stride byte offset (M / N direction), the fixed version bits 46-48
// = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (non-blocking polls) for the mbarrier phase with the given parity;
// false when it has not completed after kWaitNs.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// Starts asynchronous copies (cp.async, 16 bytes each) of a row-major [R][K] BF16
// matrix (rows 16-byte aligned, R a multiple of 8) into the canonical layout at
// dst; rows at or past rows_valid are zero-filled.  Eight consecutive threads
// fill one 128-byte core matrix (8 rows x 16 bytes), so a warp's shared-memory
// writes are contiguous and its global reads are 16-byte pieces of 8 rows.  The
// caller commits the group and completes it with cp_async_wait().
__device__ __forceinline__ void stage_async(char *dst, const uint16_t *src, int R, int K, int64_t rows_valid) {
  const int chunks = K >> 3;
  const uint32_t d0 = smem_addr(dst);
  for (int e = threadIdx.x; e < R * chunks; e += kThreads) {
    const int rest = e >> 3;
    const int kc = rest % chunks, r = ((rest / chunks) << 3) + (e & 7);
    const bool ok = r < rows_valid;
    const uint16_t *g = ok ? src + (int64_t)r * K + kc * 8 : src;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d0 + canon(r, kc * 8, K)), "l"(g),
                 "r"(ok ? 16 : 0)
                 : "memory");
  }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Feature rows [r0, r0 + 128) of [n][kIn] (rows from `live` on zero) into X.
__device__ __forceinline__ void stage_rows_async(char *sX, const uint16_t *feat, int64_t r0, int64_t live) {
  stage_async(sX, feat + r0 * kIn, kRows, kIn, live - r0);
  cp_async_commit();
}

// Issues the MMA chain D[128 x N] = A[128 x K] B[N x K]^T (fresh accumulation).
__device__ __forceinline__ void mma_chain(uint32_t d_tmem, const char *a, const char *b, int K, int N) {
  const uint32_t a0 = smem_addr(a), b0 = smem_addr(b);
  const uint32_t sbo = (uint32_t)(K >> 3) << 7;
  const uint32_t idesc = instr_desc(kRows, N);
  for (int s = 0; s < K / 16; ++s)
    mma_bf16(d_tmem, smem_desc(a0 + 256u * s, 128u, sbo), smem_desc(b0 + 256u * s, 128u, sbo), idesc, s > 0);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_infer_tc(fgs_mlp m, const uint16_t *__restrict__ feat, int64_t n, const int64_t *d_count,
               float *__restrict__ out, int32_t *d_status) {
  extern __shared__ __align__(1024) char smem[];
  char *sW1 = smem + kOffW1, *sW2 = smem + kOffW2, *sW3 = smem + kOffW3, *sX = smem + kOffX, *sH = smem + kOffH;
  float *sb1 = reinterpret_cast<float *>(smem + kOffBias), *sb2 = sb1 + kHid, *sb3 = sb2 + kHid;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kOffBar + 8);
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t live = d_count ? min(*d_count, n) : n;

  // weights and biases once per CTA, with the first feature tile in the same group
  stage_async(sW1, m.w1, kHid, kIn, kHid);
  stage_async(sW2, m.w2, kHid, kHid, kHid);
  stage_async(sW3, m.w3, kN3, kHid, 8);  // w3 holds 8 padded rows; rows 8..15 zero
  const int64_t step = (int64_t)gridDim.x * kRows;
  int64_t r0 = (int64_t)blockIdx.x * kRows;
  if (r0 < live) stage_async(sX, feat + r0 * kIn, kRows, kIn, live - r0);
  cp_async_commit();
  for (int e = threadIdx.x; e < kHid; e += kThreads) {
    sb1[e] = m.b1[e];
    sb2[e] = m.b2[e];
  }
  if (threadIdx.x < kN3) sb3[threadIdx.x] = threadIdx.x < 8 ? m.b3[threadIdx.x] : 0.f;
  if (threadIdx.x == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const int quad = warp & 3, cgrp = warp >> 2;                         // lane quadrant, column group
  const uint32_t my_lane = tmem + ((uint32_t)(quad * 32) << 16);         // this warp's 32 TMEM lanes
  const uint32_t bar_a = smem_addr(bar);
  uint32_t phase = 0;  // mbarrier parity, tracked by thread 0 only
  const int row = quad * 32 + lane;  // this thread's row of the tile (its TMEM lane)

  for (; r0 < live; r0 += step) {
    const int valid = (int)(live - r0 < kRows ? live - r0 : kRows);
    cp_async_wait();
    fence_async_smem();  // operands written through the generic proxy, read by the tensor cores
    tc_fence_before();
    __syncthreads();
    // three layers: issue, wait, epilogue into the next operand
    for (int layer = 0; layer < 3; ++layer) {
      tc_fence_after();
      if (threadIdx.x == 0) {
        if (layer == 0) mma_chain(tmem, sX, sW1, kIn, kHid);
        else if (layer == 1) mma_chain(tmem, sH, sW2, kHid, kHid);
        else mma_chain(tmem, sH, sW3, kHid, kN3);
        mma_commit(bar_a);
        if (bar_wait(bar_a, phase)) phase ^= 1u;
        else s_fail = 1;
      }
      __syncthreads();
      tc_fence_after();
      if (s_fail) break;
      // the first layer's MMAs have read X: the next tile's rows stream in behind
      // the rest of this tile
      if (layer == 0 && r0 + step < live) stage_rows_async(sX, feat, r0 + step, live);
      if (layer < 2) {
        // bias, GELU, BF16 into the next layer's A operand (H1, then H2 over it:
        // the second layer's MMAs have finished reading H1)
        char *dst = sH;
        const float *bias = layer == 0 ? sb1 : sb2;
        const int c0 = 32 * cgrp;
        float v[32];
        tmem_ld32(my_lane + (uint32_t)c0, v);
#pragma unroll
        for (int q = 0; q < 32; q += 8) {
          uint32_t w[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int c = c0 + q + 2 * t;
            w[t] = (uint32_t)f2bf(gelu(v[q + 2 * t] + bias[c])) |
                   ((uint32_t)f2bf(gelu(v[q + 2 * t + 1] + bias[c + 1])) << 16);
          }
          *reinterpret_cast<uint4 *>(dst + canon(row, c0 + q, kHid)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_async_smem();
      } else if (cgrp == 0) {  // the 4 outputs sit in the first column group
        float v[16];
        tmem_ld16(my_lane, v);
        if (row < valid) {
          float4 y = make_float4(v[0] + sb3[0], v[1] + sb3[1], v[2] + sb3[2], v[3] + sb3[3]);
          *reinterpret_cast<float4 *>(out + (r0 + row) * kOut) = y;
        }
      }
      tc_fence_before();
      __syncthreads();
    }
    if (s_fail) break;
  }
  cp_async_wait();  // a copy still in flight after a timeout lands before the CTA exits
  if (s_fail && threadIdx.x == 0) {
    if (d_status) atomicOr(d_status, FGS_DEV_TIMEOUT);
    // The timed-out chain may still be writing TMEM: wait once more (bounded) for
    // the phase that did not complete before the columns are handed back.
    (void)bar_wait(bar_a, phase);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace tc

// Inference of n feature rows (or *d_count of them when d_count is not NULL).
fgs_status launch_infer_tc(const fgs_mlp *mlp, const uint16_t *feat, int64_t n, const int64_t *d_count, float *out,
                           int32_t *d_status, cudaStream_t st) {
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(feat) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(mlp->w1) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(mlp->w2) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(mlp->w3) & 15) == 0,
                "prior inference: features, outputs and weights must be 16-byte aligned");
  FGS_CUDA(cudaFuncSetAttribute(tc::k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes),
           "prior inference shared memory");
  const int64_t tiles = (n + tc::kRows - 1) / tc::kRows;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms()));
  tc::k_infer_tc<<<grid, tc::kThreads, tc::kSmemBytes, st>>>(*mlp, feat, n, d_count, out, d_status);
  count_launch();
  FGS_CHECK_LAUNCH("prior inference");
  return FGS_OK;
}

}  // namespace fgs
