// loss_tile.cuh -- one 16x16 tile of the fused eq16 loss (L1 colour, L1 depth,
// 1 - SSIM) and its gradient, shared by the loss kernel (loss.cu) and the
// persistent window (window.cu).
//
// The tile stages the colour pair with a 10-pixel halo in shared memory, forms
// the five windowed moments (mu_x, mu_y, E[x^2], E[y^2], E[xy]) with separable
// 11-tap sums on the tile plus a 5-pixel halo, evaluates SSIM and its partial
// derivatives there, and applies the adjoint window to produce dL/dC on the tile
// -- no intermediate map touches HBM.
#pragma once

#include "common.cuh"

namespace fgs {

constexpr int kLT = 16;              // output tile
constexpr int kLR = 5;               // window radius (11 taps)
constexpr int kLIn = kLT + 4 * kLR;  // 36: input with a 10-pixel halo
constexpr int kLMid = kLT + 2 * kLR; // 26: moment maps with a 5-pixel halo
constexpr int kLThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct LossViews {
  int n;
  struct V {
    int W, H, tiles_x, tile_base;
    int64_t pix_base;
  } v[FGS_MAX_VIEWS];
};

struct LossArgs {
  LossViews lv;
  const float *color, *depth, *color_gt, *depth_gt;
  float w_c, w_d, w_s;
  float *dC, *dD;
  double *partials;
  float g[11];
};

__device__ __forceinline__ float sgnf(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

// Shared memory of one loss tile (floats).
constexpr int kLossSmemFloats = 2 * kLIn * kLIn + 5 * kLIn * kLMid + 5 * kLMid * kLMid;

// Loss tile b (a 16x16 output tile of one view) by the whole CTA (any multiple of
// 32 threads); `sm` holds kLossSmemFloats floats.  Writes dL/dC, dL/dD of the tile
// and the tile's loss contribution to a.partials[b].
__device__ __forceinline__ void loss_tile(const LossArgs &a, int b, float *sm) {
  float *X = sm;                      // [kLIn][kLIn]
  float *Y = X + kLIn * kLIn;
  float *H5 = Y + kLIn * kLIn;        // [5][kLIn][kLMid]
  float *M5 = H5 + 5 * kLIn * kLMid;  // [5][kLMid][kLMid]; later [3] derivative maps
  float *H3 = H5;                     // [3][kLMid][kLT] (reuses H5)
  __shared__ double red[32];
  const int nthr = blockDim.x;
  __syncthreads();  // the previous user of the shared buffer is done
  int v = 0;
  while (v + 1 < a.lv.n && b >= a.lv.v[v + 1].tile_base) ++v;
  const auto &cv = a.lv.v[v];
  const int lt = b - cv.tile_base;
  const int ty = lt / cv.tiles_x, tx = lt - ty * cv.tiles_x;
  const int W = cv.W, H = cv.H;
  const int64_t HW = (int64_t)W * H;
  const int ox = tx * kLT - 2 * kLR, oy = ty * kLT - 2 * kLR;  // input origin
  const float inv3 = 1.0f / (3.0f * (float)HW), inv1 = 1.0f / (float)HW;
  const float dS = -a.w_s * inv3;  // dL / dSSIM(q)
  const float *C = a.color + 3 * cv.pix_base, *Cg = a.color_gt + 3 * cv.pix_base;
  float *dC = a.dC + 3 * cv.pix_base;
  float acc = 0.f;
  for (int ch = 0; ch < 3; ++ch) {
    const float *Xc = C + ch * HW, *Yc = Cg + ch * HW;
    if (a.w_s != 0.f) {
      for (int e = threadIdx.x; e < kLIn * kLIn; e += nthr) {
        const int iy = e / kLIn, ix = e - iy * kLIn;
        const int gx = ox + ix, gy = oy + iy;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        X[e] = in ? Xc[(int64_t)gy * W + gx] : 0.f;
        Y[e] = in ? Yc[(int64_t)gy * W + gx] : 0.f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLIn * kLMid; e += nthr) {
        const int r = e / kLMid, c = e - r * kLMid;
        float s1 = 0.f, s2 = 0.f, s11 = 0.f, s22 = 0.f, s12 = 0.f;
#pragma unroll
        for (int i = 0; i < 11; ++i) {
          const float x = X[r * kLIn + c + i], y = Y[r * kLIn + c + i], w = a.g[i];
          s1 += w * x;
          s2 += w * y;
          s11 += w * x * x;
          s22 += w * y * y;
          s12 += w * x * y;
        }
        const int o = r * kLMid + c;
        H5[o] = s1;
        H5[kLIn * kLMid + o] = s2;
        H5[2 * kLIn * kLMid + o] = s11;
        H5[3 * kLIn * kLMid + o] = s22;
        H5[4 * kLIn * kLMid + o] = s12;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLMid * kLMid; e += nthr) {
        const int r = e / kLMid, c = e - r * kLMid;
        float m[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < 11; ++i) s += a.g[i] * H5[k * kLIn * kLMid + (r + i) * kLMid + c];
          m[k] = s;
        }
        const int qx = ox + kLR + c, qy = oy + kLR + r;
        float d1 = 0.f, d11 = 0.f, d12 = 0.f;
        if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
          const float m1 = m[0], m2 = m[1];
          const float sx = m[2] - m1 * m1, sy = m[3] - m2 * m2, sxy = m[4] - m1 * m2;
          const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * sxy + kC2;
          const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = sx + sy + kC2;
          const float rB = 1.f / (B1 * B2);
          const float S = A1 * A2 * rB;
          d1 = dS * ((2.f * m2 * A2 - 2.f * m2 * A1) * rB - S * (2.f * m1 / B1 - 2.f * m1 / B2));
          d11 = dS * (-S / B2);
          d12 = dS * (2.f * A1 * rB);
          if (r >= kLR && r < kLR + kLT && c >= kLR && c < kLR + kLT) acc += a.w_s * (1.f - S) * inv3;
        }
        M5[e] = d1;
        M5[kLMid * kLMid + e] = d11;
        M5[2 * kLMid * kLMid + e] = d12;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLMid * kLT; e += nthr) {
        const int r = e / kLT, c = e - r * kLT;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < 11; ++i) s += a.g[i] * M5[k * kLMid * kLMid + r * kLMid + c + i];
          H3[k * kLMid * kLT + e] = s;
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < kLT * kLT; e += nthr) {
      const int r = e / kLT, c = e - r * kLT;
      const int gx = tx * kLT + c, gy = ty * kLT + r;
      if (gx < W && gy < H) {
        const int64_t p = (int64_t)gy * W + gx;
        const float xp = Xc[p], yp = Yc[p];
        float grad = 0.f;
        if (a.w_s != 0.f) {
          float vv[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 11; ++i) s += a.g[i] * H3[k * kLMid * kLT + (r + i) * kLT + c];
            vv[k] = s;
          }
          grad = vv[0] + 2.f * xp * vv[1] + yp * vv[2];
        }
        const float d = xp - yp;
        acc += a.w_c * fabsf(d) * inv3;
        grad += a.w_c * sgnf(d) * inv3;
        dC[ch * HW + p] = grad;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kLT * kLT; e += nthr) {
    const int r = e / kLT, c = e - r * kLT;
    const int gx = tx * kLT + c, gy = ty * kLT + r;
    if (gx < W && gy < H) {
      const int64_t p = cv.pix_base + (int64_t)gy * W + gx;
      const float dg = a.depth_gt[p];
      float gd = 0.f;
      if (dg > 0.f) {
        const float d = a.depth[p] - dg;
        acc += a.w_d * fabsf(d) * inv1;
        gd = a.w_d * sgnf(d) * inv1;
      }
      a.dD[p] = gd;
    }
  }
  double s = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nthr / 32; ++w) t += red[w];
    a.partials[b] = t;
  }
}




}  // namespace fgs
