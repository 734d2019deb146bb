// prior.cu -- learned seeding prior (an extension of eq11, not in the paper).
//
// Features of a seed pixel: the 16x16 gray patch around it (clamped), its 2D DFT
// magnitude log(1 + |F|) (256), the depth, zero padding -> 272 BF16 values.
// MLP 272 -> 128 -> 128 -> 4 (GELU, erf form), BF16 operands, FP32 accumulation,
// activations rounded to BF16 before each product.
//
// Inference (the per-frame hot call) runs on tcgen05 with TMEM accumulators, in
// prior_tc.cu.  The training step here uses mma.sync m16n8k16 (BF16 in, FP32
// out): its small per-CTA batches (32 rows) and the three GEMM orientations of the
// backward pass favour register fragments.  Operands stay row-major in shared memory (activations [rows][features],
// weights [out][in]); ldmatrix (plain or .trans) builds each fragment, so the
// forward (X W^T), the input gradients (dZ W) and the weight gradients (dZ^T H)
// all read the same tiles.  Row strides are padded (280 / 136 / 24 halves) so the
// eight 16-byte rows of every ldmatrix hit distinct shared-memory banks.
#include <cmath>

#include "common.cuh"

namespace fgs {

constexpr int kIn = FGS_PRIOR_IN;    // 272
constexpr int kHid = FGS_PRIOR_HID;  // 128
constexpr int kOutP = 8;             // output rows padded to one n-tile
constexpr int kOut = FGS_PRIOR_OUT;  // 4
constexpr int kXS = 280;             // row stride (halves) of X and W1
constexpr int kHS = 136;             // row stride of H1, H2, W2, W3, dZ
constexpr int kYS = 24;              // row stride of dY (16 used)
constexpr int kNumParams = kHid * kIn + kHid + kHid * kHid + kHid + kOutP * kHid + kOutP;

// packed parameter offsets (Adam moments and gradients use this order)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOutP * kHid;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[16 x 8 NT] += A[16 x 16 KS] B[16 KS x 8 NT] for one warp.
//   A_T = false: A stored [m][k] (row m at a + m * as);  true: stored [k][m].
//   B_T = false: B stored [n][k] (a weight [out][in]);   true: stored [k][n].
// NT must be even (two n-tiles per ldmatrix.x4).
template <int NT, int KS, bool A_T, bool B_T>
__device__ __forceinline__ void warp_gemm(float (&acc)[NT][4], const uint16_t *a, int as, const uint16_t *b,
                                          int bs) {
  const int lane = threadIdx.x & 31;
  const int r8 = lane & 7, j = lane >> 3;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = ks * 16;
    uint32_t a0, a1, a2, a3;
    if (!A_T) {
      ldsm_x4(smem_u32(a + (lane & 15) * as + k0 + (lane >> 4) * 8), a0, a1, a2, a3);
    } else {
      ldsm_x4_t(smem_u32(a + (k0 + r8 + (lane >> 4) * 8) * as + (j & 1) * 8), a0, a1, a2, a3);
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt += 2) {
      const int n0 = nt * 8;
      uint32_t b0, b1, b2, b3;
      if (!B_T) {
        ldsm_x4(smem_u32(b + (n0 + (j >> 1) * 8 + r8) * bs + k0 + (j & 1) * 8), b0, b1, b2, b3);
      } else {
        ldsm_x4_t(smem_u32(b + (k0 + (j & 1) * 8 + r8) * bs + n0 + (j >> 1) * 8), b0, b1, b2, b3);
      }
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
      mma_bf16(acc[nt + 1], a0, a1, a2, a3, b2, b3);
    }
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)f2bf(lo) | ((uint32_t)f2bf(hi) << 16);
}

// accumulator fragment element (e) of n-tile nt -> (row, col) inside the warp's 16 rows
__device__ __forceinline__ void frag_pos(int nt, int e, int &row, int &col) {
  const int lane = threadIdx.x & 31;
  row = (lane >> 2) + ((e >> 1) << 3);
  col = nt * 8 + 2 * (lane & 3) + (e & 1);
}

struct MlpSmem {
  uint16_t *w1, *w2, *w3;  // [128][280], [128][136], [16][136] (rows 8..15 zero)
  float *b1, *b2, *b3;
};

__device__ void load_weights(const fgs_mlp &m, MlpSmem &s) {
  for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) {
    const int r = e / kIn, c = e - r * kIn;
    s.w1[r * kXS + c] = m.w1[e];
  }
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int r = e / kHid, c = e - r * kHid;
    s.w2[r * kHS + c] = m.w2[e];
  }
  for (int e = threadIdx.x; e < 16 * kHid; e += blockDim.x) {
    const int r = e / kHid, c = e - r * kHid;
    s.w3[r * kHS + c] = r < kOutP ? m.w3[e] : (uint16_t)0;
  }
  for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
    s.b1[e] = m.b1[e];
    s.b2[e] = m.b2[e];
  }
  for (int e = threadIdx.x; e < kOutP; e += blockDim.x) s.b3[e] = m.b3[e];
}

// Forward of 16 rows held by this warp.  x: [16][280] BF16.  Writes h1, h2 (BF16)
// and optionally z1, z2 (FP32 [16][128]); returns y in acc3 fragments.
__device__ __forceinline__ void warp_forward(const MlpSmem &s, const uint16_t *x, uint16_t *h1, uint16_t *h2,
                                             float *z1, float *z2, float (&y)[1][4]) {
  {
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<16, kIn / 16, false, false>(acc, x, kXS, s.w1, kXS);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 4; e += 2) {
        int row, col;
        frag_pos(nt, e, row, col);
        const float za = acc[nt][e] + s.b1[col], zb = acc[nt][e + 1] + s.b1[col + 1];
        if (z1) {
          z1[row * kHid + col] = za;
          z1[row * kHid + col + 1] = zb;
        }
        *reinterpret_cast<uint32_t *>(h1 + row * kHS + col) = pack_bf16(gelu(za), gelu(zb));
      }
  }
  __syncwarp();
  {
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<16, kHid / 16, false, false>(acc, h1, kHS, s.w2, kHS);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 4; e += 2) {
        int row, col;
        frag_pos(nt, e, row, col);
        const float za = acc[nt][e] + s.b2[col], zb = acc[nt][e + 1] + s.b2[col + 1];
        if (z2) {
          z2[row * kHid + col] = za;
          z2[row * kHid + col + 1] = zb;
        }
        *reinterpret_cast<uint32_t *>(h2 + row * kHS + col) = pack_bf16(gelu(za), gelu(zb));
      }
  }
  __syncwarp();
  {
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    warp_gemm<2, kHid / 16, false, false>(acc, h2, kHS, s.w3, kHS);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int row, col;
      frag_pos(0, e, row, col);
      y[0][e] = acc[0][e] + s.b3[col];
    }
  }
}

// ---------------------------------------------------------------------------------
// features

__global__ void __launch_bounds__(256) k_features(const float *__restrict__ rgb, const float *__restrict__ depth,
                                                  int W, int H, const int32_t *__restrict__ xy, int64_t n,
                                                  const int64_t *d_count, uint16_t *__restrict__ feat) {
  __shared__ float P[16][17];
  __shared__ float2 R[16][17];
  __shared__ float2 tw[16];
  const int64_t live = d_count ? min(*d_count, n) : n;
  const int tid = threadIdx.x;
  if (tid < 16) {
    float sn, cs;
    sincospif(-2.0f * (float)tid / 16.0f, &sn, &cs);
    tw[tid] = make_float2(cs, sn);
  }
  const int64_t HW = (int64_t)W * H;
  for (int64_t s = blockIdx.x; s < live; s += gridDim.x) {
    const int x = xy[2 * s], y = xy[2 * s + 1];
    {
      const int r = tid >> 4, c = tid & 15;
      const int yy = min(max(y - 8 + r, 0), H - 1), xx = min(max(x - 8 + c, 0), W - 1);
      const int64_t p = (int64_t)yy * W + xx;
      P[r][c] = 0.299f * rgb[p] + 0.587f * rgb[HW + p] + 0.114f * rgb[2 * HW + p];
    }
    __syncthreads();
    {  // DFT along x: R[r][k] = sum_c P[r][c] w^(k c)
      const int r = tid >> 4, k = tid & 15;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float2 w = tw[(k * c) & 15];
        acc.x += P[r][c] * w.x;
        acc.y += P[r][c] * w.y;
      }
      R[r][k] = acc;
    }
    __syncthreads();
    {  // DFT along y: F[v][k] = sum_r R[r][k] w^(v r)
      const int v = tid >> 4, k = tid & 15;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const float2 w = tw[(v * r) & 15], a = R[r][k];
        acc.x += a.x * w.x - a.y * w.y;
        acc.y += a.x * w.y + a.y * w.x;
      }
      feat[s * kIn + v * 16 + k] = f2bf(log1pf(hypotf(acc.x, acc.y)));
    }
    if (tid < kIn - 256) feat[s * kIn + 256 + tid] = tid == 0 ? f2bf(depth[(int64_t)y * W + x]) : (uint16_t)0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// weights staged in shared memory (padded rows for conflict-free fragment loads)

constexpr size_t kWeightSmem = sizeof(uint16_t) * (kHid * kXS + kHid * kHS + 16 * kHS) + sizeof(float) * (2 * kHid + kOutP);

__device__ __forceinline__ void carve_weights(char *base, MlpSmem &s) {
  s.w1 = reinterpret_cast<uint16_t *>(base);
  s.w2 = s.w1 + kHid * kXS;
  s.w3 = s.w2 + kHid * kHS;
  s.b1 = reinterpret_cast<float *>(s.w3 + 16 * kHS);
  s.b2 = s.b1 + kHid;
  s.b3 = s.b2 + kHid;
}

// ---------------------------------------------------------------------------------
// training: one CTA per 32 rows (2 warps), forward with stored activations, MSE,
// backward, and FP32 gradient accumulation with global atomics

constexpr int kTrainRows = 32;
constexpr size_t kTrainSmem = kWeightSmem +
                              sizeof(uint16_t) * kTrainRows * (kXS + 2 * kHS + kYS + 2 * kHS) +
                              sizeof(float) * kTrainRows * 2 * kHid;

__global__ void __launch_bounds__(64) k_train(fgs_mlp m, const uint16_t *__restrict__ feat,
                                              const float *__restrict__ target, int64_t n, float *__restrict__ grad,
                                              float *__restrict__ d_loss) {
  extern __shared__ __align__(16) char smem[];
  MlpSmem s;
  carve_weights(smem, s);
  uint16_t *X = reinterpret_cast<uint16_t *>(smem + kWeightSmem);  // [32][280]
  uint16_t *H1 = X + kTrainRows * kXS;                               // [32][136]
  uint16_t *H2 = H1 + kTrainRows * kHS;
  uint16_t *DY = H2 + kTrainRows * kHS;                              // [32][24]
  uint16_t *DZ2 = DY + kTrainRows * kYS;                             // [32][136]
  uint16_t *DZ1 = DZ2 + kTrainRows * kHS;
  float *Z1 = reinterpret_cast<float *>(DZ1 + kTrainRows * kHS);     // [32][128]
  float *Z2 = Z1 + kTrainRows * kHid;
  __shared__ float s_loss[2];
  load_weights(m, s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kTrainRows;
  for (int e = threadIdx.x; e < kTrainRows * (kIn / 2); e += blockDim.x) {
    const int r = e / (kIn / 2), c = (e - r * (kIn / 2)) * 2;
    const int64_t row = row0 + r;
    *reinterpret_cast<uint32_t *>(X + r * kXS + c) =
        row < n ? *reinterpret_cast<const uint32_t *>(feat + row * kIn + c) : 0u;
  }
  __syncthreads();
  const int wr = warp * 16;  // this warp's first row
  float y[1][4];
  warp_forward(s, X + wr * kXS, H1 + wr * kHS, H2 + wr * kHS, Z1 + wr * kHid, Z2 + wr * kHid, y);
  // MSE: L = mean over n x 4 of (y - t)^2;  dY = 2 (y - t) / (4 n), rounded to BF16
  float lsum = 0.f;
  const float scale = 2.0f / (4.0f * (float)n);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int row, col;
    frag_pos(0, e, row, col);
    const int64_t g = row0 + wr + row;
    float d = 0.f;
    if (col < kOut && g < n) {
      const float diff = y[0][e] - target[g * kOut + col];
      lsum += diff * diff;
      d = scale * diff;
    }
    DY[(wr + row) * kYS + col] = f2bf(d);
    DY[(wr + row) * kYS + 8 + col] = 0;  // k padding 8..15
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) s_loss[warp] = lsum;
  __syncwarp();
  // dH2 = dY W3 (K = 16, W3 rows 8..15 zero); dZ2 = dH2 * gelu'(Z2)
  {
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<16, 1, false, true>(acc, DY + wr * kYS, kYS, s.w3, kHS);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 4; e += 2) {
        int row, col;
        frag_pos(nt, e, row, col);
        const float *z = Z2 + (wr + row) * kHid + col;
        *reinterpret_cast<uint32_t *>(DZ2 + (wr + row) * kHS + col) =
            pack_bf16(acc[nt][e] * gelu_grad(z[0]), acc[nt][e + 1] * gelu_grad(z[1]));
      }
  }
  __syncwarp();
  // dH1 = dZ2 W2; dZ1 = dH1 * gelu'(Z1)
  {
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<16, kHid / 16, false, true>(acc, DZ2 + wr * kHS, kHS, s.w2, kHS);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 4; e += 2) {
        int row, col;
        frag_pos(nt, e, row, col);
        const float *z = Z1 + (wr + row) * kHid + col;
        *reinterpret_cast<uint32_t *>(DZ1 + (wr + row) * kHS + col) =
            pack_bf16(acc[nt][e] * gelu_grad(z[0]), acc[nt][e + 1] * gelu_grad(z[1]));
      }
  }
  __syncthreads();
  // bias gradients: column sums of dY, dZ2, dZ1 (the BF16 values the GEMMs use)
  for (int c = threadIdx.x; c < 2 * kHid + kOutP; c += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < kTrainRows; ++r) {
      if (c < kHid) acc += bf2f(DZ1[r * kHS + c]);
      else if (c < 2 * kHid) acc += bf2f(DZ2[r * kHS + c - kHid]);
      else acc += bf2f(DY[r * kYS + c - 2 * kHid]);
    }
    if (acc != 0.f) {
      if (c < kHid) atomicAdd(grad + kOffB1 + c, acc);
      else if (c < 2 * kHid) atomicAdd(grad + kOffB2 + c - kHid, acc);
      else atomicAdd(grad + kOffB3 + c - 2 * kHid, acc);
    }
  }
  // dW3 = dY^T H2 (M = 16 padded outputs, K = 32 rows, N = 128); warp w: n-tiles 8w..8w+7
  {
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<8, kTrainRows / 16, true, true>(acc, DY, kYS, H2 + warp * 64, kHS);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int row, col;
        frag_pos(nt, e, row, col);
        if (row < kOutP) atomicAdd(grad + kOffW3 + row * kHid + warp * 64 + col, acc[nt][e]);
      }
  }
  // dW2 = dZ2^T H1 (M = 128, K = 32, N = 128); warp w: m-tiles 4w..4w+3
  for (int mt = warp * 4; mt < warp * 4 + 4; ++mt) {
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    warp_gemm<16, kTrainRows / 16, true, true>(acc, DZ2 + mt * 16, kHS, H1, kHS);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int row, col;
        frag_pos(nt, e, row, col);
        atomicAdd(grad + kOffW2 + (mt * 16 + row) * kHid + col, acc[nt][e]);
      }
  }
  // dW1 = dZ1^T X (M = 128, K = 32, N = 272 in two halves of 136)
  for (int mt = warp * 4; mt < warp * 4 + 4; ++mt) {
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      float acc[18][4];
#pragma unroll
      for (int i = 0; i < 18; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
      warp_gemm<18, kTrainRows / 16, true, true>(acc, DZ1 + mt * 16, kHS, X + half * 136, kXS);
#pragma unroll
      for (int nt = 0; nt < 18; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int row, col;
          frag_pos(nt, e, row, col);
          const int c = half * 136 + col;
          if (nt < 17 && c < kIn) atomicAdd(grad + kOffW1 + (mt * 16 + row) * kIn + c, acc[nt][e]);
        }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(d_loss, (s_loss[0] + s_loss[1]) / (4.0f * (float)n));
}

// Adam on the FP32 masters, then the BF16 copies.
__global__ void k_mlp_adam(fgs_mlp_master ms, const float *__restrict__ grad, fgs_train_params hp,
                           uint16_t *w1, uint16_t *w2, uint16_t *w3, float *b1, float *b2, float *b3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNumParams) return;
  float *p;
  uint16_t *bf = nullptr;
  float *fcopy = nullptr;
  int j;
  if (i < kOffB1) { j = i - kOffW1; p = ms.w1 + j; bf = w1 + j; }
  else if (i < kOffW2) { j = i - kOffB1; p = ms.b1 + j; fcopy = b1 + j; }
  else if (i < kOffB2) { j = i - kOffW2; p = ms.w2 + j; bf = w2 + j; }
  else if (i < kOffW3) { j = i - kOffB2; p = ms.b2 + j; fcopy = b2 + j; }
  else if (i < kOffB3) { j = i - kOffW3; p = ms.w3 + j; bf = w3 + j; }
  else { j = i - kOffB3; p = ms.b3 + j; fcopy = b3 + j; }
  const float g = grad[i];
  const float m = hp.beta1 * ms.m[i] + (1.f - hp.beta1) * g;
  const float v = hp.beta2 * ms.v[i] + (1.f - hp.beta2) * g * g;
  ms.m[i] = m;
  ms.v[i] = v;
  const float c1 = 1.f - powf(hp.beta1, (float)hp.step), c2 = 1.f - powf(hp.beta2, (float)hp.step);
  float val = *p - hp.lr * (m / c1) / (sqrtf(v / c2) + hp.eps);
  // padded entries (w1 inputs 257.., w3/b3 rows 4..7) stay zero
  if (i < kOffB1 && (j % kIn) >= 257) val = 0.f;
  if (i >= kOffW3 && i < kOffB3 && j / kHid >= kOut) val = 0.f;
  if (i >= kOffB3 && j >= kOut) val = 0.f;
  *p = val;
  if (bf) *bf = f2bf(val);
  if (fcopy) *fcopy = val;
}

// Learned prior on freshly written high-frequency seeds: features, inference, then per seed the
// predicted opacity logit, and the predicted log-scales unless one axis lies
// further than max_dev from eq11's log-scale (then eq11's radius stays: eq11 is
// what arbitrates the scale; it says nothing about opacity).
__global__ void k_apply_prior(const float *__restrict__ pred, const int32_t *__restrict__ xy,
                              const uint8_t *__restrict__ seed_hi, const int64_t *__restrict__ base,
                              const float *__restrict__ depth, int W, float alpha_h, float alpha_l, float f,
                              float max_dev, GaussGrads g) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= base[1] || !seed_hi[s]) return;  // the prior initialises high-frequency seeds only
  const float d = depth[(int64_t)xy[2 * s + 1] * W + xy[2 * s]];
  const float ls = logf((seed_hi[s] ? alpha_h : alpha_l) * d / f);
  const float *p = pred + 4 * s;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) ok = ok && fabsf(p[k] - ls) <= max_dev;
  const int64_t i = base[0] + s, c = g.cap;
  g.logits[i] = p[3];
  if (!ok) return;
  g.log_scales[i] = p[0];
  g.log_scales[c + i] = p[1];
  g.log_scales[2 * c + i] = p[2];
}

size_t prior_apply_workspace_size(int64_t max_new) {
  return align_up((size_t)max_new * kIn * 2) + align_up((size_t)max_new * kOut * 4);
}


static fgs_status set_smem(const void *fn, size_t bytes) {
  FGS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), "prior smem");
  return FGS_OK;
}

// Inference on the tensor cores (prior_tc.cu).
fgs_status launch_infer_tc(const fgs_mlp *mlp, const uint16_t *feat, int64_t n, const int64_t *d_count, float *out,
                           int32_t *d_status, cudaStream_t st);

fgs_status prior_apply_to_seeds(const fgs_mlp *mlp, const float *rgb, const float *depth, int W, int H,
                                const int32_t *seed_xy, const uint8_t *seed_hi, const int64_t *base, int64_t max_new,
                                float alpha_h, float alpha_l, float fx, float fy, float max_dev, void *ws,
                                size_t ws_bytes, GaussGrads g, int32_t *d_status, cudaStream_t st) {
  if (max_new == 0) return FGS_OK;
  FGS_CHECK_ARG(ws_bytes >= prior_apply_workspace_size(max_new), "prior workspace");
  uint16_t *feat = static_cast<uint16_t *>(ws);
  float *pred = reinterpret_cast<float *>(static_cast<char *>(ws) + align_up((size_t)max_new * kIn * 2));
  const int64_t *count = base + 1;
  k_features<<<(unsigned)std::min<int64_t>(max_new, 8 * num_sms()), 256, 0, st>>>(rgb, depth, W, H, seed_xy,
                                                                                 max_new, count, feat);
  count_launch();
  fgs_status s = launch_infer_tc(mlp, feat, max_new, count, pred, d_status, st);
  if (s != FGS_OK) return s;
  k_apply_prior<<<(unsigned)((max_new + 255) / 256), 256, 0, st>>>(pred, seed_xy, seed_hi, base, depth, W, alpha_h,
                                                                  alpha_l, 0.5f * (fx + fy), max_dev, g);
  count_launch();
  FGS_CHECK_LAUNCH("prior on seeds");
  return FGS_OK;
}

static bool mlp_ok(const fgs_mlp *m) { return m && m->w1 && m->b1 && m->w2 && m->b2 && m->w3 && m->b3; }

}  // namespace fgs

using namespace fgs;

extern "C" int64_t fgs_prior_num_params(void) { return kNumParams; }

extern "C" size_t fgs_prior_train_workspace_size(int64_t n) {
  (void)n;
  return align_up(sizeof(float) * kNumParams);
}

extern "C" fgs_status fgs_prior_features(const float *rgb, const float *depth, int32_t width, int32_t height,
                                         const int32_t *seed_xy, int64_t n, uint16_t *features, void *stream) {
  FGS_CHECK_ARG(n >= 0, "fgs_prior_features: n < 0");
  if (n == 0) return FGS_OK;
  FGS_CHECK_ARG(rgb && depth && seed_xy && features && width > 0 && height > 0, "fgs_prior_features: bad argument");
  k_features<<<(unsigned)std::min<int64_t>(n, 8 * num_sms()), 256, 0, as_stream(stream)>>>(
      rgb, depth, width, height, seed_xy, n, nullptr, features);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_prior_features");
  return FGS_OK;
}

extern "C" fgs_status fgs_prior_infer(const fgs_mlp *mlp, const uint16_t *features, int64_t n, float *out,
                                      int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(n >= 0, "fgs_prior_infer: n < 0");
  if (n == 0) return FGS_OK;
  FGS_CHECK_ARG(mlp_ok(mlp) && features && out, "fgs_prior_infer: bad argument");
  return launch_infer_tc(mlp, features, n, nullptr, out, d_status, as_stream(stream));
}

extern "C" fgs_status fgs_prior_train(fgs_mlp *mlp, fgs_mlp_master *master, const uint16_t *features,
                                      const float *targets, int64_t n, const fgs_train_params *hp, float *d_loss,
                                      void *ws, size_t ws_bytes, void *stream) {
  FGS_CHECK_ARG(mlp_ok(mlp) && master && master->w1 && master->m && master->v && features && targets && hp &&
                    d_loss && n >= 1,
                "fgs_prior_train: bad argument");
  FGS_CHECK_ARG(hp->step >= 1, "fgs_prior_train: step must be >= 1");
  FGS_CHECK_ARG(ws && ws_bytes >= fgs_prior_train_workspace_size(n), "fgs_prior_train: workspace");
  cudaStream_t st = as_stream(stream);
  float *grad = static_cast<float *>(ws);
  FGS_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kNumParams, st), "memset grad");
  fgs_status s = set_smem((const void *)k_train, kTrainSmem);
  if (s != FGS_OK) return s;
  k_train<<<(unsigned)((n + kTrainRows - 1) / kTrainRows), 64, kTrainSmem, st>>>(*mlp, features, targets, n, grad,
                                                                                 d_loss);
  k_mlp_adam<<<(kNumParams + 255) / 256, 256, 0, st>>>(*master, grad, *hp, const_cast<uint16_t *>(mlp->w1),
                                                       const_cast<uint16_t *>(mlp->w2),
                                                       const_cast<uint16_t *>(mlp->w3), const_cast<float *>(mlp->b1),
                                                       const_cast<float *>(mlp->b2), const_cast<float *>(mlp->b3));
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_prior_train");
  return FGS_OK;
}
